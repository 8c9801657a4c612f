#!/usr/bin/env python
"""Benchmark of the fusion hot path on the Kinect-sized workload.

One *step* fuses the whole 300-frame 640x480 sequence (5 mm voxels, mu 2 cm,
hash 2^20 + 2^17, pool 2^18, float32 sdf) into a freshly reset scene: for
every frame the allocation, commit, block initialisation, visible-list and
integration kernels. The step is captured once into a CUDA graph and
replayed; depth frames (368 MB) and the voxel pool (671 MB) stay resident in
HBM, so inputs are larger than L2.

Printed JSON line (rank 0):
  value     voxel-updates/s (voxels whose (sdf, w) a frame wrote), whole job
  e2e       the same metric through the public API with the depth frames in
            pinned host memory (copied every frame inside tsdf_integrate) and
            the step's counters read back to the host at the end of the step
  roofline  the integration kernel: algorithmic bytes per launch
            (10 B per updated f32 voxel + 32 B per visible-block record + the
            depth image) over its mean duration from two CUDA events around
            every integration launch, recorded in a second timed pass of the
            same graph (the headline pass carries no events)
  cpu_baseline  the FP64 oracle, single-threaded, on the first frames of the
            same sequence (about 15 s of CPU work)

--impl reference times the oracle instead (the CPU definition; there is no
other implementation of this path to install).
--gpus N (N > 1, under torchrun): every rank fuses its own independently
seeded sequence on its own GPU (no collective on the data path); value is
the sum of updates over ranks divided by the slowest rank's time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-updates/s (640x480, 5 mm, f32 sdf)"
UNIT = "voxel-updates/s"
PROFILE = os.path.join(ROOT, "profiles", "integrate_kinect_640x480_5mm.md")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-frames", type=int, default=0,
                    help="profiling driver: fuse the first N frames eagerly, one sync per "
                         "frame, and print each frame's counters (no timing)")
    return ap.parse_args()


def seq_cache_path(w, n):
    d = os.environ.get("TSDF_SEQ_CACHE", "/tmp/tsdf_seq_cache")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"{w.name}_{w.seed}_{n}.npz")


def load_sequence(w, n):
    from synthdepth import make_sequence
    path = seq_cache_path(w, n)
    if os.path.exists(path):
        z = np.load(path)
        from synthdepth.configs import Sequence
        return Sequence(workload=w, depth=z["depth"], poses=z["poses"], first_frame=0)
    seq = make_sequence(w, n_frames=n)
    try:
        np.savez(path + ".tmp.npz", depth=seq.depth, poses=seq.poses)
        os.replace(path + ".tmp.npz", path)
    except OSError:
        pass
    return seq


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def integrate_profile_traffic():
    """dram bytes per launch of the integration kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h:
        return None
    src = open(os.path.join(ROOT, "paper_1410_0925_gb300", "csrc", "integrate.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest() != h.group(1):
        return None
    return float(m.group(1))


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(w, seq, seconds: float) -> dict:
    """The FP64 oracle, as it stands, single-threaded, on the first frames of
    the sequence until about `seconds` of CPU time have been spent."""
    import oracle
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                          max_weight=w.max_weight, storage=w.storage))
    intr = [f32(v) for v in (w.fx, w.fy, w.cx, w.cy)]
    t0 = time.perf_counter()
    n = 0
    while n < seq.depth.shape[0] and time.perf_counter() - t0 < seconds:
        o.integrate(seq.depth[n], intr, seq.poses[n])
        n += 1
    dt = time.perf_counter() - t0
    upd = o.total_updates()
    return {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {seq.depth.shape[0]} frames of the same sequence, "
                      f"{upd} voxel updates in {dt:.1f} s (FP64 C oracle, 1 thread, "
                      f"host nproc {os.cpu_count()})",
            "frames_per_s": n / dt}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synthdepth import workload_kinect
    import oracle
    w = workload_kinect()
    n_frames = 3
    seq = load_sequence(w, args.frames)
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    intr = [f32(v) for v in (w.fx, w.fy, w.cx, w.cy)]

    def step():
        o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                              max_weight=w.max_weight, storage=w.storage))
        for i in range(n_frames):
            o.integrate(seq.depth[i], intr, seq.poses[i])
        return o.total_updates()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    upd = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = upd / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": w.name, "frames_per_step": n_frames,
                      "note": "bounded sample: each step fuses the first 3 frames of the "
                              "300-frame sequence into a fresh oracle scene"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"first {n_frames} frames per step, {args.steps} steps"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out, default=float), flush=True)


def run_ours(args):
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_kinect

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    w = workload_kinect()
    if rank:
        w = replace(w, seed=w.seed + 7919 * rank)
    seq = load_sequence(w, args.frames)
    nf = seq.depth.shape[0]
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth_dev = torch.from_numpy(seq.depth).to(dev)
    stream = torch.cuda.Stream(device=dev)
    scene = Scene.from_workload(w, stream=stream)

    def enqueue_step(src):
        scene.reset()
        for i in range(nf):
            scene.integrate(src[i], intr, seq.poses[i])

    # eager warm-up (also the reference counters of one step)
    with torch.cuda.stream(stream):
        enqueue_step(depth_dev)
    st_step = scene.stats()
    upd_step = st_step["total_updated_voxels"]
    vis_step = st_step["total_visible_blocks"]
    launches_per_step = None

    def capture(timing: bool, integration_only: bool = False):
        nonlocal launches_per_step
        if timing:
            scene.timing_begin(nf, integration_only)
        l0 = scene.stats()["kernel_launches"]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            enqueue_step(depth_dev)
        launches_per_step = scene.stats()["kernel_launches"] - l0
        return g

    def replay(g):
        # CUDAGraph.replay launches on the current stream: make it the scene's
        with torch.cuda.stream(stream):
            g.replay()

    g_plain = capture(False)
    for _ in range(args.warmup):
        replay(g_plain)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    # --- pass A: headline (graph replay, device-resident inputs) -------------
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        replay(g_plain)
    e1.record(stream)
    barrier()
    clock_info = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    st = scene.stats()
    assert st["total_updated_voxels"] == upd_step, "graph replay disagrees with eager step"
    ms_max = max_over_ranks(ms_total)
    upd_all = sum_over_ranks(float(upd_step * args.steps))
    value = upd_all / (ms_max * 1e-3)
    frames_per_s = sum_over_ranks(float(nf * args.steps)) / (ms_max * 1e-3)

    # --- pass B: two events around every integration launch (roofline) ------
    from paper_1410_0925_gb300.tsdf import STAGES

    def timed_pass(integration_only):
        g = capture(True, integration_only)
        replay(g)
        torch.cuda.synchronize()
        out = []
        barrier()
        for _ in range(args.steps):
            replay(g)
            out.append(scene.timing_read())
        barrier()
        scene.timing_end()
        return np.concatenate(out)                 # (steps * frames, stages)

    ib = STAGES.index("integrate")
    marks = timed_pass(True)                       # boundaries 3 and 4 only
    steps_marks = marks.reshape(args.steps, nf, -1)
    integ_ms = (steps_marks[:, :, ib + 1] - steps_marks[:, :, ib]).reshape(-1)
    # per-frame latency: period between consecutive frame ends inside a step
    frame_ms = np.diff(steps_marks[:, :, ib + 1], axis=1).reshape(-1)
    # --- pass C: events around every stage (stage shares) --------------------
    full = timed_pass(False)
    stage_ms = np.diff(full, axis=1)               # (steps * frames, stages)
    W, H = w.width, w.height
    upd_per_launch = upd_step / nf
    vis_per_launch = vis_step / nf
    integ_bytes = 10.0 * upd_per_launch + 32.0 * vis_per_launch + 4.0 * W * H
    achieved = integ_bytes / (integ_ms.mean() * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = integrate_profile_traffic()
    stage_share = {name: float(stage_ms[:, i].sum() / stage_ms.sum())
                   for i, name in enumerate(STAGES)}

    # --- pass D: end to end through the public API with host buffers ---------
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(seq.depth).pin_memory()
        with torch.cuda.stream(stream):
            enqueue_step(pinned)
        scene.stats()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                enqueue_step(pinned)
            st_e = scene.stats()           # device -> host read of the step's counters
        barrier()
        dt = time.perf_counter() - t0
        assert st_e["total_updated_voxels"] == upd_step
        dt_max = max_over_ranks(dt)
        e2e = {"value": upd_all / dt_max, "unit": UNIT,
               "h2d_bytes_per_step": int(seq.depth.nbytes),
               "d2h_bytes_per_step": 64,
               "frames_per_s": sum_over_ranks(float(nf * args.steps)) / dt_max}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, seq, args.cpu_seconds)

    if rank == 0:
        bytes_step = (10.0 * upd_step + 32.0 * vis_step + 8.0 * W * H * nf)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "frames_per_step": nf, "image": f"{W}x{H}",
                       "voxel_size_m": w.voxel_size, "mu_m": w.mu,
                       "hash": f"2^{w.hash_buckets_log2}x{w.entries_per_bucket}+{w.excess_entries}",
                       "pool_blocks": w.pool_blocks, "storage": "f32 sdf + u8 weight",
                       "l2": "inputs larger than L2: depth frames 368 MB + voxel pool 671 MB resident",
                       "graph": "one CUDA graph per step (reset + 300 frames)",
                       "allocated_blocks_end": st_step["allocated_blocks"],
                       "seed": w.seed},
            "frames_per_s": frames_per_s,
            "hbm_gbs_effective": bytes_step * args.steps * world / (ms_max * 1e-3) / 1e9,
            "p50_frame_ms": float(np.percentile(frame_ms, 50)),
            "p99_frame_ms": float(np.percentile(frame_ms, 99)),
            "stage_share": stage_share,
            "roofline": {"kernel": "integrate_kernel<f32>", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": f"{peak_kind} (copy, burst)",
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": integ_bytes,
                         "mean_launch_us": float(integ_ms.mean() * 1e3)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clock_info,
        }
        print(json.dumps(out, default=float), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_profile_driver(args):
    """Small, deterministic case for ncu: frames 0..N-1 of the Kinect
    sequence, launched eagerly; prints per-frame updated voxels and visible
    blocks so a capture of launch k can be scaled by its own counts."""
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_kinect
    torch.cuda.set_device(0)
    w = workload_kinect()
    seq = load_sequence(w, args.frames)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(seq.depth[:args.profile_frames]).cuda()
    scene = Scene.from_workload(w)
    per = []
    for i in range(args.profile_frames):
        scene.integrate(depth[i], intr, seq.poses[i])
        st = scene.stats()
        per.append({"frame": i, "updated": st["last_updated_voxels"],
                    "visible": st["last_visible_blocks"], "new": st["last_new_blocks"],
                    "allocated": st["allocated_blocks"]})
    print(json.dumps({"profile_frames": per}))


def main():
    args = parse_args()
    if args.profile_frames:
        run_profile_driver(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
