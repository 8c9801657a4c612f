"""The multi-rank bookkeeping of bench.py on CPU (world size 2, gloo): the
single-scene path does not shard, so ranks fuse independently seeded scenes
and share only a barrier and max / sum reductions of their timings and unit
counts. Each rank here renders its own seeded input and reduces through the
same Dist class the GPU runs use (there with NCCL)."""

import os
import socket
import sys
from types import SimpleNamespace

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from dataclasses import replace
    from synthdepth import make_sequence, workload_kinect
    d = bench.Dist(backend="gloo")
    d.barrier()
    base = workload_kinect(n_frames=2)
    w = replace(base, seed=bench.rank_seed(base.seed, d.rank))
    seq = make_sequence(w)
    units = float((seq.depth > 0).sum())       # this rank's work
    seconds = 1.0 + rank                        # this rank's time
    res = dict(rank=d.rank, world=d.world, seed=w.seed, depth_sum=float(seq.depth.sum()),
               units=units, max_t=d.max(seconds), sum_units=d.sum(units))
    d.barrier()
    d.close()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), res, allow_pickle=True)


def test_two_ranks_reduce_and_fuse_independent_scenes(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [np.load(tmp_path / f"rank{i}.npy", allow_pickle=True).item() for i in range(2)]
    assert [x["rank"] for x in r] == [0, 1] and all(x["world"] == 2 for x in r)
    # every rank sees the same reductions: the slowest rank's time and the
    # units of the whole job
    assert all(x["max_t"] == 2.0 for x in r)
    assert all(x["sum_units"] == r[0]["units"] + r[1]["units"] for x in r)
    # independent inputs: rank 0 keeps the base seed, rank 1 renders another scene
    from synthdepth import workload_kinect
    assert r[0]["seed"] == workload_kinect().seed and r[1]["seed"] != r[0]["seed"]
    assert r[0]["depth_sum"] != r[1]["depth_sum"]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = SimpleNamespace(workload="kinect", frames=3, steps=1, warmup=0, gpus=2,
                           cpu_seconds=1.0)
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK"):
        monkeypatch.delenv(k, raising=False)
    d = bench.Dist(backend="gloo")
    assert d.world == 1 and d.rank == 0 and d.dist is None
    assert d.max(3.5) == 3.5 and d.sum(2.0) == 2.0
    d.barrier()
    d.close()
