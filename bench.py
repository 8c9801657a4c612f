#!/usr/bin/env python
"""Benchmark of the fusion hot path on the Kinect-sized workload.

One *step* fuses the whole 300-frame 640x480 sequence (5 mm voxels, mu 2 cm,
hash 2^20 + 2^17, pool 2^18, float32 sdf) into a freshly reset scene: for
every frame the allocation kernel (band allocation, find-or-insert, commit)
and the integration kernel (block selection, new-block initialisation, rule
U), as one pipelined sequence (tsdf_integrate_frames: frame t + 1's
allocation overlaps frame t's integration). The step is captured once into a
CUDA graph and replayed; depth frames (368 MB) and the voxel pool (671 MB)
stay resident in HBM, so inputs are larger than L2.

Printed JSON line (rank 0):
  value     voxel-updates/s (voxels whose (sdf, w) a frame wrote), whole job
  e2e       the same metric through the public API with the depth frames in
            pinned host memory (copied to the device every step, then fused
            as one pipelined sequence) and the step's counters read back to
            the host at the end of the step
  roofline  the integration kernel: algorithmic bytes per launch
            (10 B per updated f32 voxel + 32 B per visible-block record + the
            depth image) over its mean duration from two CUDA events around
            every integration launch, recorded in a second timed pass of the
            same graph (the headline pass carries no events)
  cpu_baseline  the FP64 oracle, single-threaded, on the first frames of the
            same sequence (about 15 s of CPU work)

Other workloads (their own JSON line, same keys; the default line above is
the headline):
  --workload hd       1280x720, 4 mm, 500 frames, int16 sdf (headline of the
                      line) beside FP16 and float32 on the same GPU, with the
                      storage forms' deviation from float32 over all voxels
  --workload batch64  64 independent scenes (images 160x120 / 320x240 /
                      640x480, voxels 4 / 5 / 10 mm, pools 2^14..2^18), 100
                      frames each; one step = reset + 100 batched launches in
                      one CUDA graph with autotuned launch shapes; int16
                      beside FP16 and float32
  --workload serve    Poisson session arrivals (200/s for 2 s), 50-400 frames
                      each at 320x240 / 640x480 / 1280x720 with 4-10 mm
                      voxels, admitted by device memory (120 GB) and fused by
                      continuous batching; p50 / p99 per-frame latency
  --workload raycast  the raycast (Section 4.4): the 300-frame Kinect
                      sequence fused first, then one step renders the scene
                      from each of the 300 poses (rays/s); also the per-frame
                      loop fuse + render (frames/s)
  --workload colour   the Kinect sequence with registered colour images, every
                      frame through tsdf_integrate_rgb (colour averaged into
                      the voxels rule U updates), beside the same loop without
                      colour
  --workload icp      the depth tracker's terms (Section 4.1): every frame
                      against the raycast maps of the frame before (pixels/s),
                      and a tracking loop (raycast, normals, 10 Gauss-Newton
                      iterations per frame) end to end
  --workload engine   the whole pipeline of one camera (tsdf_engine_process:
                      track against the model, fuse, render) over the
                      sequence from its first pose (frames/s)
These render their depth on the device (same scene and trajectory recipe).

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

from synthdepth.cache import load_sequence  # noqa: E402
from paper_1410_0925_gb300.workloads import (SWAP_CAPACITY, SWAP_MARGIN_PX, Z_NEAR,  # noqa: E402
                                             swap_step_ops)

METRIC = "voxel-updates/s (640x480, 5 mm, f32 sdf)"
UNIT = "voxel-updates/s"
PROFILE = os.path.join(ROOT, "profiles", "integrate_kinect_640x480_5mm.md")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload",
                    choices=["kinect", "hd", "batch64", "serve", "raycast", "colour", "icp",
                             "engine", "swap"],
                    default="kinect")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--scenes", type=int, default=64)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the int16 / FP16 storage forms beside float32")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload: skip the HD and batch sub-records")
    ap.add_argument("--form-oracle-frames", type=int, default=16,
                    help="frames fused by the FP64 oracle per storage form for its error")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons every 50 ms, from
    the warm-up through the timed region."""

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
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed work starts once sampling runs
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.lines.clear()

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


def profile_traffic(profile: str, source: str, unit_key: str, units_per_launch: float):
    """DRAM bytes (read + write) of an average launch of a kernel, from its
    committed ncu summary if that was taken on the current kernel source
    (else None). The summary holds one captured launch; its traffic is scaled
    to the average launch by the ratio of the work units named by unit_key."""
    try:
        text = open(profile).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    u = re.search(unit_key + r":\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not u or not h:
        return None
    src = open(os.path.join(ROOT, "paper_1410_0925_gb300", "csrc", source), "rb").read()
    if hashlib.sha256(src).hexdigest() != h.group(1):
        return None
    return float(m.group(1)) * units_per_launch / float(u.group(1))


def integrate_profile_traffic(updates_per_launch: float):
    """Integration launch traffic, scaled by voxel updates (the voxel data
    dominates)."""
    return profile_traffic(PROFILE, "integrate.cu", "traffic_updated_voxels", updates_per_launch)


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_sample(seq, k):
    """The first k frames of a sequence (host or device rendered) as host arrays: the
    oracle's input, from the seeded input generator (not from the library)."""
    from types import SimpleNamespace
    k = min(k, seq.depth.shape[0])
    d = seq.depth[:k]
    d = d if isinstance(d, np.ndarray) else d.cpu().numpy()
    return SimpleNamespace(depth=d, poses=np.asarray(seq.poses[:k]))


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


def form_error_vs_oracle(w, seq, k: int) -> dict:
    """Fuse the first k frames of the sequence with the library and with the
    FP64 oracle in the workload's storage form; on the oracle's unflagged
    voxels of unflagged blocks, the largest |sdf - sdf_oracle| and the
    weights that differ (the parity protocol's strict set)."""
    import oracle
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    hs = host_sample(seq, k)
    o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                          max_weight=w.max_weight, storage=w.storage))
    intr = [f32(v) for v in (w.fx, w.fy, w.cx, w.cy)]
    for i in range(len(hs.depth)):
        o.integrate(hs.depth[i], intr, hs.poses[i])
    ref = o.read()
    sc = Scene.from_workload(w)
    dev = torch.from_numpy(hs.depth).cuda()
    for i in range(len(hs.depth)):
        sc.integrate(dev[i], make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height),
                     hs.poses[i])
    got = sc.read_blocks()
    sc.close()
    gvals = got.sdf_values()
    idx = {tuple(kk): i for i, kk in enumerate(got.keys.tolist())}
    max_err, bad_w, strict, flagged, missing = 0.0, 0, 0, 0, 0
    for b, kk in enumerate(ref["keys"].tolist()):
        m = ref["vflag"][b] == 0
        if ref["bflag"][b]:
            flagged += 512
            continue
        g = idx.get(tuple(kk))
        if g is None:
            missing += 1
            continue
        flagged += int((~m).sum())
        strict += int(m.sum())
        if m.any():
            max_err = max(max_err, float(np.abs(gvals[g][m] - ref["sdf"][b][m]).max()))
            bad_w += int((got.w[g][m] != ref["w"][b][m]).sum())
    total = 512 * len(ref["keys"])
    return {"frames": len(hs.depth), "max_abs_sdf_err": max_err, "tolerance": FORM_TOL[w.storage],
            "within_tolerance": bool(max_err <= FORM_TOL[w.storage] and bad_w == 0 and
                                     missing == 0),
            "weights_differing": bad_w, "oracle_blocks_missing": missing,
            "strict_voxels": strict, "flagged_fraction": flagged / max(total, 1)}


def run_reference_raycast(args):
    """--workload raycast --impl reference: the raycast oracle as it stands,
    each step the raycast of one pose of the sequence (every pixel) from the
    oracle's volume of the first 3 frames."""
    from synthdepth import workload_kinect
    import oracle
    w = workload_kinect()
    seq = load_sequence(w, args.frames)
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    intr = [f32(v) for v in (w.fx, w.fy, w.cx, w.cy)]
    o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                          max_weight=w.max_weight, storage=w.storage))
    for i in range(3):
        o.integrate(seq.depth[i], intr, seq.poses[i])
    r = o.read()
    vol = oracle.Volume(r["keys"], r["sdf"].astype(np.float32).astype(np.float64))
    p = oracle.RayParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu), z_near=f32(Z_NEAR))
    for i in range(args.warmup):
        vol.raycast(w.width, w.height, intr, seq.poses[i], p)
    t0 = time.perf_counter()
    for i in range(args.steps):
        vol.raycast(w.width, w.height, intr, seq.poses[i % seq.depth.shape[0]], p)
    dt = time.perf_counter() - t0
    v = args.steps * w.width * w.height / dt
    out = {"impl": "reference", "metric": RAY_METRIC, "value": v, "unit": RAY_UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name + "-raycast", "raycasts_per_step": 1,
                      "note": "bounded sample: each step renders one pose of the sequence "
                              "from the oracle's volume of the first 3 frames"},
           "cpu_baseline": {"value": v, "unit": RAY_UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} raycasts of 640x480"},
           "e2e": {"value": v, "unit": RAY_UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out, default=float), flush=True)


def run_reference_sampled(args):
    """--impl reference for the colour, tracker, swapping and pipeline
    workloads: the oracle as it stands, one thread; each step is that
    workload's CPU sample (a few frames' worth, about cpu_seconds / steps of
    CPU time)."""
    from synthdepth import workload_kinect
    w = workload_kinect()
    per_step = max(2.0, args.cpu_seconds / max(1, args.steps))
    if args.workload == "colour":
        seq = load_sequence(w, args.frames, colour=True)
        metric, unit, fn = COLOUR_METRIC, UNIT, lambda: colour_cpu_baseline(w, seq, per_step)
    elif args.workload == "icp":
        seq = load_sequence(w, args.frames)
        metric, unit, fn = ICP_METRIC, ICP_UNIT, lambda: icp_cpu_baseline(w, seq, per_step)
    elif args.workload == "engine":
        seq = load_sequence(w, args.frames)
        metric, unit = ENGINE_METRIC, "frames/s"
        fn = lambda: engine_cpu_baseline(w, seq, per_step)  # noqa: E731
    else:
        seq = load_sequence(w, args.frames)
        metric, unit, fn = SWAP_METRIC, UNIT, lambda: swap_cpu_baseline(w, seq, per_step)
    t0 = time.perf_counter()
    vals = [fn()["value"] for _ in range(args.steps)]
    dt = time.perf_counter() - t0
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": metric, "value": v, "unit": unit,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{w.name}-{args.workload}",
                      "note": f"bounded sample: each step runs the oracle on the first frames "
                              f"of the sequence for about {per_step:.0f} s"},
           "cpu_baseline": {"value": v, "unit": unit, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} samples of about {per_step:.0f} s"},
           "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out, default=float), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "raycast":
        run_reference_raycast(args)
        return
    if args.workload in ("colour", "icp", "swap", "engine"):
        run_reference_sampled(args)
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


def bytes_per_update(storage: int) -> float:
    """Algorithmic HBM bytes of one voxel update: read and write the sdf (4 B
    float32, 2 B int16 / FP16) and the uint8 weight."""
    return 2.0 * (4.0 if storage == STORAGE_F32 else 2.0) + 2.0


STORAGE_F32, STORAGE_I16, STORAGE_F16 = 0, 1, 2
STORAGE_NAME = {STORAGE_F32: "f32", STORAGE_I16: "i16", STORAGE_F16: "f16"}


def integ_kernel_name(storage: int, pipelined: bool) -> str:
    """The integration kernel the library launches for a depth-only scene of
    these workloads (images below 2^24 pixels, mu above 2^-20 m): the staged
    kernel, 512 threads alone and 256 beside the next frame's allocation,
    except 16-bit storage in a pipelined sequence, which takes the general
    kernel."""
    name = STORAGE_NAME[storage]
    if not pipelined:
        return f"integrate_staged_kernel<{name}, 512>"
    if storage == STORAGE_F32:
        return f"integrate_staged_kernel<{name}, 256>"
    return f"integrate_kernel<{name}>"
# frames of the 1280x720 sequence fused by the oracle for the per-form errors
HD_ORACLE_FRAMES = 6
# tolerances of the parity protocol per storage form (normalised sdf units)
FORM_TOL = {STORAGE_F32: 1e-5, STORAGE_I16: 1.0 / 32767.0 + 1e-5, STORAGE_F16: 1e-3}


def rank_seed(seed: int, rank: int) -> int:
    """The input seed of a rank: every rank fuses its own, independently
    seeded scene (weak scaling, no shared data)."""
    return seed + 7919 * rank


class Dist:
    """Rank bookkeeping: barrier + max / sum over ranks (NCCL when N > 1; the
    host-only gloo backend, with no device, serves the CPU tests of this
    logic). No collective touches the data path: ranks fuse independent
    scenes."""

    def __init__(self, backend: str = "nccl"):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.cuda = backend == "nccl"
        if self.world > 1:
            import torch.distributed as dist
            if self.cuda:
                torch.cuda.set_device(local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            else:
                dist.init_process_group(backend)
            self.dist = dist
        elif self.cuda:
            torch.cuda.set_device(0)
        self.dev = (torch.device("cuda", torch.cuda.current_device()) if self.cuda
                    else torch.device("cpu"))

    def barrier(self):
        import torch
        if self.dist is not None:
            self.dist.barrier()
        if self.cuda:
            torch.cuda.synchronize()

    def _reduce(self, x, op):
        import torch
        if self.dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=self.dev)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return x if self.dist is None else self._reduce(x, self.dist.ReduceOp.MAX)

    def sum(self, x):
        return x if self.dist is None else self._reduce(x, self.dist.ReduceOp.SUM)

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def graph_replayer(stream):
    import torch

    def replay(g):
        # CUDAGraph.replay launches on the current stream: make it the scene's
        with torch.cuda.stream(stream):
            g.replay()
    return replay


def measure_scene(w, depth_dev, poses, args, d: Dist, clocks=None) -> dict:
    """Time one single-scene step (reset + every frame) captured in a CUDA
    graph: pass A (headline, no events: the frames as one pipelined sequence,
    tsdf_integrate_frames, where frame t + 1's allocation overlaps frame t's
    integration), pass B (frame by frame, events around every integration
    launch), pass C (frame by frame, events around every stage)."""
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from paper_1410_0925_gb300.tsdf import STAGES
    nf = depth_dev.shape[0]
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    stream = torch.cuda.Stream(device=d.dev)
    scene = Scene.from_workload(w, stream=stream)
    replay = graph_replayer(stream)

    def enqueue_frames(src):
        scene.reset()
        for i in range(nf):
            scene.integrate(src[i], intr, poses[i])

    def enqueue_step(src):
        scene.reset()
        scene.integrate_frames(src, intr, poses)

    with torch.cuda.stream(stream):
        enqueue_frames(depth_dev)                  # eager warm-up and reference counts
    st_step = scene.stats()
    with torch.cuda.stream(stream):
        enqueue_step(depth_dev)
    st_seq = scene.stats()
    assert st_seq["total_updated_voxels"] == st_step["total_updated_voxels"], \
        "pipelined sequence disagrees with frame-by-frame fusion"
    launches = {}

    def capture(timing: bool, integration_only: bool = False):
        if timing:
            scene.timing_begin(nf, integration_only)
        l0 = scene.stats()["kernel_launches"]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            if timing:
                enqueue_frames(depth_dev)
            else:
                enqueue_step(depth_dev)
        launches["per_step"] = scene.stats()["kernel_launches"] - l0
        return g

    g_plain = capture(False)
    if clocks is not None:
        clocks.start()
    for _ in range(args.warmup):
        replay(g_plain)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    d.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        replay(g_plain)
    e1.record(stream)
    d.barrier()
    clock_info = clocks.stop() if clocks is not None else None
    ms_total = e0.elapsed_time(e1)
    st = scene.stats()
    assert st["total_updated_voxels"] == st_step["total_updated_voxels"], \
        "graph replay disagrees with the eager step"
    launches_per_step = launches["per_step"]
    del g_plain

    def timed_pass(integration_only):
        g = capture(True, integration_only)
        replay(g)
        torch.cuda.synchronize()
        out = []
        d.barrier()
        for _ in range(args.steps):
            replay(g)
            out.append(scene.timing_read())
        d.barrier()
        scene.timing_end()
        return np.concatenate(out)

    ib = STAGES.index("integrate")
    marks = timed_pass(True).reshape(args.steps, nf, -1)
    integ_ms = (marks[:, :, ib + 1] - marks[:, :, ib]).reshape(-1)
    frame_ms = np.diff(marks[:, :, ib + 1], axis=1).reshape(-1)
    full = timed_pass(False)
    stage_ms = np.diff(full, axis=1)
    stage_share = {name: float(stage_ms[:, i].sum() / stage_ms.sum())
                   for i, name in enumerate(STAGES)}
    upd = st_step["total_updated_voxels"]
    vis = st_step["total_visible_blocks"]
    integ_bytes = (bytes_per_update(w.storage) * upd / nf + 32.0 * vis / nf
                   + 4.0 * w.width * w.height)
    return dict(scene=scene, stream=stream, enqueue_step=enqueue_step, nf=nf,
                ms_total=ms_total, st_step=st_step, upd_step=upd, vis_step=vis,
                launches_per_step=launches_per_step, integ_ms=integ_ms,
                frame_ms=frame_ms, stage_share=stage_share, integ_bytes=integ_bytes,
                clocks=clock_info)


def roofline_entry(kernel, integ_bytes, integ_ms, traffic):
    peak, peak_kind = measured_peak_hbm()
    achieved = integ_bytes / (float(np.mean(integ_ms)) * 1e-3) / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} (copy, burst)",
            "traffic": traffic, "algorithmic_bytes_per_launch": integ_bytes,
            "mean_launch_us": float(np.mean(integ_ms) * 1e3)}


def e2e_sequence(m, pinned, steps, upd_step, d) -> dict:
    """The step through the public API with the depth frames in pinned host
    memory: tsdf_integrate_frames copies each frame to the device itself (its
    own copy stream, ahead of the allocation stream), and the step's counters
    are read back to the host at the end of every step. The step's calls are
    captured once into a CUDA graph, as for the device-resident step: the
    frames' host-to-device copies are nodes of that graph, so every replay
    copies the pinned buffer's current contents (eager calls are also timed:
    cross-stream event waits between eager launches cost the GPU several
    microseconds per frame)."""
    import torch
    scene, stream = m["scene"], m["stream"]
    with torch.cuda.stream(stream):
        m["enqueue_step"](pinned)    # eager: allocates the staging ring
    scene.stats()

    def timed(step):
        step()
        scene.stats()
        d.barrier()
        t0 = time.perf_counter()
        st = None
        for _ in range(steps):
            step()
            st = scene.stats()       # device -> host read of the step's counters
        d.barrier()
        dt = time.perf_counter() - t0
        assert st["total_updated_voxels"] == upd_step
        return d.max(dt)

    def eager():
        with torch.cuda.stream(stream):
            m["enqueue_step"](pinned)

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        m["enqueue_step"](pinned)

    def replay():
        with torch.cuda.stream(stream):
            g.replay()

    dt_graph = timed(replay)
    dt_eager = timed(eager)
    del g
    rate = lambda dt: d.sum(float(upd_step * steps)) / dt  # noqa: E731
    return {"value": rate(dt_graph), "unit": UNIT,
            "h2d_bytes_per_step": int(pinned.numel() * pinned.element_size()),
            "d2h_bytes_per_step": 64,
            "frames_per_s": d.sum(float(pinned.shape[0] * steps)) / dt_graph,
            "launch": "the step's API calls captured once in a CUDA graph, replayed per step",
            "eager_value": rate(dt_eager)}


def run_ours(args):
    import torch
    from dataclasses import replace
    from synthdepth import workload_kinect

    d = Dist()
    w = workload_kinect()
    if d.rank:
        w = replace(w, seed=rank_seed(w.seed, d.rank))
    seq = load_sequence(w, args.frames)
    nf = seq.depth.shape[0]
    depth_dev = torch.from_numpy(seq.depth).to(d.dev)
    clocks = ClockSampler(torch.cuda.current_device())
    m = measure_scene(w, depth_dev, seq.poses, args, d, clocks)
    ms_max = d.max(m["ms_total"])
    upd_step = m["upd_step"]
    upd_all = d.sum(float(upd_step * args.steps))
    value = upd_all / (ms_max * 1e-3)
    frames_per_s = d.sum(float(nf * args.steps)) / (ms_max * 1e-3)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(seq.depth).pin_memory()
        e2e = e2e_sequence(m, pinned, args.steps, upd_step, d)

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, seq, args.cpu_seconds)

    # the storage forms on the same sequence and GPU: the pipelined step's
    # throughput, the integration roofline on each form's byte basis, and the
    # error against the FP64 oracle (first frames, same storage form)
    forms = {}
    if not args.no_forms:
        for storage in (STORAGE_F32, STORAGE_I16, STORAGE_F16):
            wf = replace(w, storage=storage)
            mf = m if storage == STORAGE_F32 else measure_scene(wf, depth_dev, seq.poses, args, d)
            msf = d.max(mf["ms_total"])
            ent = {"value": d.sum(float(mf["upd_step"] * args.steps)) / (msf * 1e-3),
                   "ms_per_step": msf / args.steps,
                   "bytes_per_update": bytes_per_update(storage),
                   "roofline_frac": roofline_entry("", mf["integ_bytes"], mf["integ_ms"],
                                                   None)["frac"],
                   "mean_integrate_us": float(np.mean(mf["integ_ms"]) * 1e3)}
            if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
                ent["err_vs_oracle"] = form_error_vs_oracle(wf, seq, args.form_oracle_frames)
            forms[STORAGE_NAME[storage]] = ent
            if storage != STORAGE_F32:
                mf["scene"].close()

    # compact sub-records: the 1280x720 int16 sequence and the 64-scene int16
    # batch, measured in the same run (fewer steps; no end-to-end leg or CPU
    # baseline, which their own workloads report)
    sub = None
    if not args.no_sub:
        sa = argparse.Namespace(**vars(args))
        sa.steps = min(args.steps, SUB_STEPS)
        hd = hd_line(sa, d, (STORAGE_I16,), complete=False)
        bt = batch_line(sa, d, (STORAGE_I16,), complete=False)
        if d.rank == 0:
            sub = {"hd_1280x720_4mm_i16": sub_record(hd), "batch64_mixed_i16": sub_record(bt)}

    if d.rank == 0:
        W, H = w.width, w.height
        bytes_step = (10.0 * upd_step + 32.0 * m["vis_step"] + 8.0 * W * H * nf)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "frames_per_step": nf, "image": f"{W}x{H}",
                       "voxel_size_m": w.voxel_size, "mu_m": w.mu,
                       "hash": f"2^{w.hash_buckets_log2}x{w.entries_per_bucket}+{w.excess_entries}",
                       "pool_blocks": w.pool_blocks, "storage": "f32 sdf + u8 weight",
                       "l2": "inputs larger than L2: depth frames 368 MB + voxel pool 671 MB resident",
                       "graph": "one CUDA graph per step (reset + the 300 frames as one "
                                "pipelined sequence)",
                       "allocated_blocks_end": m["st_step"]["allocated_blocks"],
                       "seed": w.seed},
            "frames_per_s": frames_per_s,
            "visited_voxels_per_s": d.sum(float(512 * m["vis_step"] * args.steps)) / (ms_max * 1e-3),
            "hbm_gbs_effective": bytes_step * args.steps * d.world / (ms_max * 1e-3) / 1e9,
            "p50_frame_ms": float(np.percentile(m["frame_ms"], 50)),
            "p99_frame_ms": float(np.percentile(m["frame_ms"], 99)),
            "stage_share": m["stage_share"],
            "roofline": roofline_entry(integ_kernel_name(STORAGE_F32, True), m["integ_bytes"],
                                       m["integ_ms"],
                                       integrate_profile_traffic(upd_step / nf)),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "forms": forms or None,
            "sub": sub,
            "gpu_launches": int(m["launches_per_step"] * args.steps),
            "clocks": m["clocks"],
        }
        print(json.dumps(out, default=float), flush=True)
    d.close()


SUB_STEPS = 5


def sub_record(line: dict) -> dict:
    """The fields of a workload's line that the default line carries."""
    keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "frames_per_s",
            "p50_frame_ms", "p99_frame_ms", "stage_share", "roofline", "config",
            "gpu_launches", "clocks")
    rec = {k: line[k] for k in keep if k in line}
    form = next(iter(line["forms"].values()))
    rec["err_vs_oracle"] = form.get("err_vs_oracle")
    if "autotuned" in form:
        rec["autotuned"] = form["autotuned"]
    return rec


def storage_accuracy(reads: dict) -> dict:
    """Max |sdf - sdf_f32| (normalised units) of the int16 / FP16 forms over
    voxels with w > 0; block sets and weights must coincide."""
    ref = reads[STORAGE_F32]
    out = {}
    for s, rb in reads.items():
        if s == STORAGE_F32:
            continue
        assert np.array_equal(rb.keys, ref.keys), "block sets differ between storage forms"
        assert np.array_equal(rb.w, ref.w), "weights differ between storage forms"
        m = ref.w > 0
        diff = np.abs(rb.sdf_values()[m] - ref.sdf_values()[m])
        out[STORAGE_NAME[s]] = {"max_abs_vs_f32": float(diff.max()) if diff.size else 0.0,
                                "mean_abs_vs_f32": float(diff.mean()) if diff.size else 0.0,
                                "voxels": int(m.sum())}
    return out


def run_hd(args):
    d = Dist()
    out = hd_line(args, d)
    if out is not None:
        print(json.dumps(out, default=float), flush=True)
    d.close()


def hd_line(args, d, storages=(STORAGE_I16, STORAGE_F16, STORAGE_F32), complete=True):
    """The precision form: 1280x720, 4 mm, 500 frames, fused with int16, FP16
    and float32 sdf on the same GPU (the JSON line on rank 0, else None).
    complete=False (a sub-record of the default line): the given storage forms
    only, no end-to-end leg and no CPU baseline."""
    import torch
    from dataclasses import replace
    from synthdepth import workload_hd
    from synthdepth.render_torch import make_sequence_torch

    nf = args.frames if args.frames != 300 else 500
    base = workload_hd()
    if d.rank:
        base = replace(base, seed=rank_seed(base.seed, d.rank))
    seq = make_sequence_torch(base, n_frames=nf, device=d.dev)
    forms = {}
    reads = {}
    e2e = None
    clocks = ClockSampler(torch.cuda.current_device())
    for storage in storages:
        w = replace(base, storage=storage)
        m = measure_scene(w, seq.depth, seq.poses, args, d,
                          clocks if storage == STORAGE_I16 else None)
        ms_max = d.max(m["ms_total"])
        upd_all = d.sum(float(m["upd_step"] * args.steps))
        forms[STORAGE_NAME[storage]] = {
            "value": upd_all / (ms_max * 1e-3), "ms_per_step": ms_max / args.steps,
            "frames_per_s": d.sum(float(nf * args.steps)) / (ms_max * 1e-3),
            "p50_frame_ms": float(np.percentile(m["frame_ms"], 50)),
            "p99_frame_ms": float(np.percentile(m["frame_ms"], 99)),
            "stage_share": m["stage_share"],
            "roofline": roofline_entry(integ_kernel_name(storage, True),
                                       m["integ_bytes"], m["integ_ms"], None),
            "gpu_launches": int(m["launches_per_step"] * args.steps),
            "clocks": m["clocks"]}
        if storage == STORAGE_I16 and complete and not args.no_e2e:
            pinned = seq.depth.cpu().pin_memory()
            e2e = e2e_sequence(m, pinned, args.steps, m["upd_step"], d)
            del pinned
        if d.rank == 0:
            reads[storage] = m["scene"].read_blocks()
        del m
        torch.cuda.empty_cache()
    if d.rank == 0:
        if not args.no_forms:
            # each form against the FP64 oracle on the first frames (the
            # oracle fuses a 1280x720 frame in about a second)
            for storage in storages:
                k = min(args.form_oracle_frames, HD_ORACLE_FRAMES)
                forms[STORAGE_NAME[storage]]["err_vs_oracle"] = form_error_vs_oracle(
                    replace(base, storage=storage), seq, k)
        cpu = None
        if d.world == 1 and complete and not args.no_cpu_baseline:
            cpu = cpu_baseline(replace(base, storage=STORAGE_I16), host_sample(seq, 40),
                               args.cpu_seconds)
            cpu["sample"] += f" (of the {nf}-frame sequence; int16 storage)"
        head = forms["i16"]
        out = {
            "metric": "voxel-updates/s (1280x720, 4 mm, i16 sdf)", "value": head["value"],
            "unit": UNIT, "n_gpus": d.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 arithmetic, i16 storage", "data": "synthetic",
            "config": {"workload": base.name, "frames_per_step": nf, "image": "1280x720",
                       "voxel_size_m": base.voxel_size, "mu_m": base.mu,
                       "pool_blocks": base.pool_blocks,
                       "render": "device ray cast of the seeded room sequence",
                       "graph": f"one CUDA graph per step (reset + {nf} frames)",
                       "l2": "inputs larger than L2"},
            "frames_per_s": head["frames_per_s"], "p50_frame_ms": head["p50_frame_ms"],
            "p99_frame_ms": head["p99_frame_ms"], "stage_share": head["stage_share"],
            "roofline": head["roofline"], "forms": forms,
            "vs_f32": ({k: forms[k]["value"] / forms["f32"]["value"] for k in ("i16", "f16")}
                       if "f32" in forms else None),
            "accuracy": storage_accuracy(reads) if STORAGE_F32 in reads else None,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"]}
        return out
    return None


def run_batch(args):
    d = Dist()
    out = batch_line(args, d)
    if out is not None:
        print(json.dumps(out, default=float), flush=True)
    d.close()


def batch_line(args, d, storages=(STORAGE_I16, STORAGE_F16, STORAGE_F32),
               complete=True):
    """The batched form: 64 independent scenes of uneven image and voxel
    sizes, 100 frames each; one step = reset + 100 batched launches (one per
    stage for all scenes) in one CUDA graph, shapes from the autotuner (the
    JSON line on rank 0, else None). complete=False (a sub-record of the default
    line): the given storage forms only, no end-to-end leg and no CPU
    baseline."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Batch, Scene, make_intrinsics
    from paper_1410_0925_gb300.tsdf import STAGES
    from synthdepth import batched_workloads
    from synthdepth.render_torch import make_sequence_torch

    nf = args.frames if args.frames != 300 else 100
    base = batched_workloads(n_scenes=args.scenes, n_frames=nf,
                             seed=rank_seed(1410_0925_4, d.rank))
    seqs = [make_sequence_torch(w, device=d.dev) for w in base]
    intrs = [make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height) for w in base]
    stream = torch.cuda.Stream(device=d.dev)
    replay = graph_replayer(stream)
    forms, reads = {}, {}
    e2e_batch = None
    n_check = min(8, len(base))
    clocks = ClockSampler(torch.cuda.current_device())
    for storage in storages:
        ws = [replace(w, storage=storage) for w in base]
        scenes = [Scene.from_workload(w, stream=stream) for w in ws]
        batch = Batch(len(ws), tables=nf, stream=stream)

        def items(i):
            return [(sc, s.depth[i], it, s.poses[i]) for sc, s, it in zip(scenes, seqs, intrs)]

        batch.prepare(items(0))
        best, tune_ms = batch.autotune(steps=3)
        # (pipelined launches do not pay at 64 scenes: each launch fills the GPU)
        batch.cursor = 0

        def capture(timing=False, integration_only=False):
            if timing:
                batch.timing_begin(nf, integration_only)
            l0 = batch.kernel_launches() + sum(sc.stats()["kernel_launches"] for sc in scenes)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for sc in scenes:
                    sc.reset()
                for i in range(nf):
                    batch.prepare(items(i))
                    batch.launch()
                batch.join()
            l1 = batch.kernel_launches() + sum(sc.stats()["kernel_launches"] for sc in scenes)
            return g, l1 - l0

        g, launches_per_step = capture()
        replay(g)
        stream.synchronize()
        stats = [sc.stats() for sc in scenes]
        upd_step = sum(s["total_updated_voxels"] for s in stats)
        vis_step = sum(s["total_visible_blocks"] for s in stats)
        if storage == STORAGE_I16:
            clocks.start()
        for _ in range(args.warmup):
            replay(g)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        d.barrier()
        e0.record(stream)
        for _ in range(args.steps):
            replay(g)
        e1.record(stream)
        d.barrier()
        clock_info = clocks.stop() if storage == STORAGE_I16 else None
        ms_total = e0.elapsed_time(e1)
        assert sum(sc.stats()["total_updated_voxels"] for sc in scenes) == upd_step
        del g

        def timed_pass(integration_only):
            gt, _ = capture(True, integration_only)
            replay(gt)
            stream.synchronize()
            out = []
            for _ in range(args.steps):
                replay(gt)
                out.append(batch.timing_read())
            batch.timing_end()
            return np.concatenate(out)

        ib = STAGES.index("integrate")
        marks = timed_pass(True).reshape(args.steps, nf, -1)
        integ_ms = (marks[:, :, ib + 1] - marks[:, :, ib]).reshape(-1)
        launch_ms = np.diff(marks[:, :, ib + 1], axis=1).reshape(-1)
        full = timed_pass(False)
        stage_ms = np.diff(full, axis=1)
        pixels = sum(w.width * w.height for w in ws)
        integ_bytes = (bytes_per_update(storage) * upd_step / nf + 32.0 * vis_step / nf
                       + 4.0 * pixels)
        ms_max = d.max(ms_total)
        upd_all = d.sum(float(upd_step * args.steps))
        forms[STORAGE_NAME[storage]] = {
            "value": upd_all / (ms_max * 1e-3), "ms_per_step": ms_max / args.steps,
            "frames_per_s": d.sum(float(len(ws) * nf * args.steps)) / (ms_max * 1e-3),
            "p50_launch_ms": float(np.percentile(launch_ms, 50)),
            "p99_launch_ms": float(np.percentile(launch_ms, 99)),
            "stage_share": {n: float(stage_ms[:, i].sum() / stage_ms.sum())
                            for i, n in enumerate(STAGES)},
            "roofline": roofline_entry(
                f"integrate_batch_{best['integrate_kernel']}_kernel<{STORAGE_NAME[storage]}>",
                integ_bytes, integ_ms, None),
            "autotuned": best, "autotune_step_ms": tune_ms,
            "gpu_launches": int(launches_per_step * args.steps), "clocks": clock_info}
        if storage == STORAGE_I16 and complete and not args.no_e2e:
            # the step through the public API from pinned host memory: every
            # launch copies its frames into the scenes' staging buffers
            # (tsdf_batch_prepare with host depth), eager prepare + launch, the
            # scenes' counters read back at the end of the step
            pinned = [s.depth.cpu().pin_memory() for s in seqs]
            hitems = lambda i: [(sc, p[i], it, s.poses[i])  # noqa: E731
                                for sc, p, s, it in zip(scenes, pinned, seqs, intrs)]

            def e2e_step():
                with torch.cuda.stream(stream):
                    for sc in scenes:
                        sc.reset()
                    for i in range(nf):
                        batch.prepare(hitems(i))
                        batch.launch()
                    batch.join()
                return sum(sc.stats()["total_updated_voxels"] for sc in scenes)

            def timed_e2e(step):
                step()
                d.barrier()
                t0 = time.perf_counter()
                for _ in range(args.steps):
                    got = step()
                d.barrier()
                assert got == upd_step
                return d.max(time.perf_counter() - t0)

            batch.cursor = 0
            dt_eager = timed_e2e(e2e_step)
            # the same calls captured once in a CUDA graph (the frames'
            # host-to-device copies are nodes of it), replayed every step
            batch.cursor = 0
            ge = torch.cuda.CUDAGraph()
            with torch.cuda.graph(ge, stream=stream):
                for sc in scenes:
                    sc.reset()
                for i in range(nf):
                    batch.prepare(hitems(i))
                    batch.launch()
                batch.join()

            def e2e_replay():
                replay(ge)
                return sum(sc.stats()["total_updated_voxels"] for sc in scenes)

            dt_graph = timed_e2e(e2e_replay)
            del ge
            # the faster of the two ways of issuing the same calls (the host
            # copies, one per scene and frame on the batch's stream, bound
            # both)
            dt = min(dt_graph, dt_eager)
            e2e_batch = {"value": d.sum(float(upd_step * args.steps)) / dt, "unit": UNIT,
                         "h2d_bytes_per_step": int(sum(p.numel() * 4 for p in pinned)),
                         "d2h_bytes_per_step": 64 * len(scenes),
                         "frames_per_s": d.sum(float(len(ws) * nf * args.steps)) / dt,
                         "launch": ("the step's API calls captured once in a CUDA graph, "
                                    "replayed per step") if dt == dt_graph else
                                   "eager API calls per step",
                         "graph_value": d.sum(float(upd_step * args.steps)) / dt_graph,
                         "eager_value": d.sum(float(upd_step * args.steps)) / dt_eager}
            del pinned
        if d.rank == 0:
            reads[storage] = [sc.read_blocks() for sc in scenes[:n_check]]
        del batch, scenes
        torch.cuda.empty_cache()
    if d.rank == 0:
        acc = {}
        for k in range(n_check if STORAGE_F32 in reads else 0):
            a = storage_accuracy({s: reads[s][k] for s in reads})
            for name, v in a.items():
                cur = acc.setdefault(name, {"max_abs_vs_f32": 0.0, "scenes": n_check})
                cur["max_abs_vs_f32"] = max(cur["max_abs_vs_f32"], v["max_abs_vs_f32"])
        if not args.no_forms:
            # each form against the FP64 oracle: scene 0 of the mix, fused
            # alone (batched fusion equals it bit for bit, tested)
            for storage in storages:
                err = form_error_vs_oracle(replace(base[0], storage=storage), seqs[0],
                                           args.form_oracle_frames)
                err["scene"] = 0
                forms[STORAGE_NAME[storage]]["err_vs_oracle"] = err
        cpu = None
        if d.world == 1 and complete and not args.no_cpu_baseline:
            w0 = base[0]
            cpu = cpu_baseline(replace(w0, storage=STORAGE_I16), host_sample(seqs[0], 40),
                               args.cpu_seconds)
            cpu["sample"] += (f" (scene 0 of {len(base)}: {w0.width}x{w0.height}, "
                              f"{w0.voxel_size * 1000:.0f} mm, int16 storage)")
        head = forms["i16"]
        mix = {}
        for w in base:
            key = f"{w.width}x{w.height}/{int(round(w.voxel_size * 1000))}mm"
            mix[key] = mix.get(key, 0) + 1
        out = {
            "metric": f"voxel-updates/s ({len(base)} scenes batched, i16 sdf)",
            "value": head["value"], "unit": UNIT, "n_gpus": d.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 arithmetic, i16 storage",
            "data": "synthetic",
            "config": {"workload": f"batch{len(base)}_mixed", "scenes": len(base),
                       "frames_per_scene": nf, "mix": mix,
                       "render": "device ray cast of the seeded room sequences",
                       "graph": f"one CUDA graph per step (reset + {nf} batched launches)",
                       "l2": "inputs larger than L2"},
            "frames_per_s": head["frames_per_s"], "p50_launch_ms": head["p50_launch_ms"],
            "p99_launch_ms": head["p99_launch_ms"], "stage_share": head["stage_share"],
            "roofline": head["roofline"], "forms": forms,
            "vs_f32": ({k: forms[k]["value"] / forms["f32"]["value"] for k in ("i16", "f16")}
                       if "f32" in forms else None),
            "accuracy": acc or None, "cpu_baseline": cpu, "e2e": e2e_batch,
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"]}
        return out
    return None


def run_serve(args):
    """The serving form: Poisson session arrivals (200 sessions/s by default
    for 2 s), each a 50-400-frame sequence at 320x240 / 640x480 / 1280x720
    with 4-10 mm voxels (int16 sdf), admitted while the admitted sessions'
    device bytes stay within the budget (120 GB by default) and fused by
    continuous batching. Each client keeps up to two frames queued. Reports
    per-frame latency (submission to device completion of the fusing step)
    and the aggregate voxel updates per second of wall time from the first
    arrival to the last completion."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Server, make_intrinsics
    from paper_1410_0925_gb300.tsdf import SESSION_FINISHED, TsdfError
    from synthdepth.configs import serving_sessions
    from synthdepth.render_torch import make_sequence_torch

    d = Dist()
    sessions = serving_sessions(rate_per_s=args.serve_rate, duration_s=args.serve_seconds,
                                seed=rank_seed(1410_0925_5, d.rank))
    longest = {}
    for _, w in sessions:
        k = (w.width, w.height, w.seed)
        longest[k] = max(longest.get(k, 0), w.n_frames)
    bank = {}
    for _, w in sessions:
        k = (w.width, w.height, w.seed)
        if k not in bank:
            bank[k] = make_sequence_torch(replace(w, n_frames=longest[k]), device=d.dev)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=d.dev)

    def serve(items, budget):
        srv = Server(budget, max_active=1024, max_queued_frames=2, max_inflight_steps=2,
                     stream=stream)
        order = sorted(range(len(items)), key=lambda i: items[i][0])
        sid, nxt, info_done = {}, {}, {}
        lat, steps_batch = [], []
        t0 = time.perf_counter()
        i_arr = 0
        live = []
        while len(info_done) < len(items):
            now = time.perf_counter() - t0
            while i_arr < len(order) and items[order[i_arr]][0] <= now:
                j = order[i_arr]
                sid[j] = srv.open_workload(items[j][1])
                nxt[j] = 0
                live.append(j)
                i_arr += 1
            still = []
            for j in live:
                w = items[j][1]
                seq = bank[(w.width, w.height, w.seed)]
                info = srv.session_info(sid[j])
                if info["state"] == SESSION_FINISHED:
                    info_done[j] = info
                    srv.release(sid[j])
                    continue
                still.append(j)
                intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
                queued = info["frames_submitted"] - info["frames_launched"]
                while nxt[j] < w.n_frames and queued < 2:
                    srv.submit(sid[j], seq.depth[nxt[j]], intr, seq.poses[nxt[j]])
                    nxt[j] += 1
                    queued += 1
                    if nxt[j] == w.n_frames:
                        srv.close_session(sid[j])
            live = still
            st = srv.step()
            if st["launched_frames"]:
                steps_batch.append(st["launched_frames"])
            for _, _, t_sub, t_done in srv.poll():
                lat.append(t_done - t_sub)
            if not st["launched_frames"] and not st["inflight_steps"] and i_arr < len(order):
                time.sleep(max(0.0, min(0.002, items[order[i_arr]][0] - now)))
        wall = time.perf_counter() - t0
        launches = srv.step()["launches"]
        srv.close()
        return wall, lat, steps_batch, info_done, launches

    # warm-up: a few short sessions through the same path
    warm = [(0.0, replace(w, n_frames=min(w.n_frames, 10))) for _, w in sessions[:max(3, args.warmup)]]
    serve(warm, int(args.serve_budget_gb * 1e9))
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    d.barrier()
    wall, lat, steps_batch, infos, launches = serve(sessions, int(args.serve_budget_gb * 1e9))
    d.barrier()
    clock_info = clocks.stop()
    upd = sum(i["updated_voxels"] for i in infos.values())
    frames = sum(i["frames_done"] for i in infos.values())
    bad = sum(1 for i in infos.values() if i["device_status"] != 0)
    wall_max = d.max(wall)
    value = d.sum(float(upd)) / wall_max
    lat = np.asarray(lat)
    waits = np.asarray([i["admit_ms"] - i["open_ms"] for i in infos.values()])
    if d.rank == 0:
        cpu = None
        if d.world == 1 and not args.no_cpu_baseline:
            w0 = sessions[0][1]
            cpu = cpu_baseline(w0, host_sample(bank[(w0.width, w0.height, w0.seed)], 40),
                               args.cpu_seconds)
            cpu["sample"] += (f" (the first session's sequence: {w0.width}x{w0.height}, "
                              f"{w0.voxel_size * 1000:.0f} mm, int16 storage)")
        mix = {}
        for _, w in sessions:
            key = f"{w.width}x{w.height}"
            mix[key] = mix.get(key, 0) + 1
        out = {
            "metric": "voxel-updates/s (serving: Poisson sessions, continuous batching, i16 sdf)",
            "value": value, "unit": UNIT, "n_gpus": d.world, "steps": len(steps_batch),
            "warmup": len(warm), "ms_per_step": 1e3 * wall / max(1, len(steps_batch)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 arithmetic, i16 storage", "data": "synthetic",
            "config": {"workload": "serving_poisson", "rate_sessions_per_s": args.serve_rate,
                       "arrival_window_s": args.serve_seconds, "sessions": len(sessions),
                       "frames": int(frames), "images": mix,
                       "budget_gb": args.serve_budget_gb, "queue_per_client": 2,
                       "render": "device ray cast, one bank of sequences per image size",
                       "l2": "inputs larger than L2"},
            "frames_per_s": d.sum(float(frames)) / wall_max,
            "wall_s": wall_max,
            "p50_frame_ms": float(np.percentile(lat, 50)),
            "p99_frame_ms": float(np.percentile(lat, 99)),
            "admission_wait_ms": {"p50": float(np.percentile(waits, 50)),
                                  "p99": float(np.percentile(waits, 99))},
            "mean_frames_per_step": float(np.mean(steps_batch)),
            "sessions_with_device_status": bad,
            "roofline": None, "cpu_baseline": cpu, "e2e": None,
            "gpu_launches": int(launches), "clocks": clock_info}
        print(json.dumps(out, default=float), flush=True)
    d.close()


RAY_METRIC = "rays/s (640x480, 5 mm, f32 sdf: raycast of the fused scene)"
RAY_UNIT = "rays/s"
RAY_PROFILE = os.path.join(ROOT, "profiles", "raycast_kinect_640x480_5mm.md")


def ray_cpu_baseline(w, seq, seconds: float, n_fuse: int = 3) -> dict:
    """The FP64 raycast oracle, as it stands, single-threaded: it fuses the
    first n_fuse frames of the sequence (not timed), then casts every pixel's
    ray from the sequence's poses in order until about `seconds` of CPU time
    have been spent."""
    import oracle
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                          max_weight=w.max_weight, storage=w.storage))
    intr = [f32(v) for v in (w.fx, w.fy, w.cx, w.cy)]
    for i in range(n_fuse):
        o.integrate(seq.depth[i], intr, seq.poses[i])
    r = o.read()
    vol = oracle.Volume(r["keys"], r["sdf"].astype(np.float32).astype(np.float64))
    p = oracle.RayParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu), z_near=f32(Z_NEAR))
    t0 = time.perf_counter()
    n = 0
    while n < seq.depth.shape[0] and time.perf_counter() - t0 < seconds:
        vol.raycast(w.width, w.height, intr, seq.poses[n], p)
        n += 1
    dt = time.perf_counter() - t0
    rays = n * w.width * w.height
    return {"value": rays / dt, "unit": RAY_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"raycasts from the first {n} poses of the sequence (every pixel, with "
                      f"the search range) of the oracle's volume of its first {n_fuse} frames "
                      f"({r['keys'].shape[0]} blocks), {dt:.1f} s (FP64 C oracle, 1 thread, "
                      f"host nproc {os.cpu_count()})"}


def run_raycast(args):
    """The raycast (Section 4.4): the 300-frame Kinect sequence is fused
    (untimed), then one step renders the fused scene from each of the 300
    poses (300 tsdf_raycast calls in one CUDA graph)."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_kinect

    d = Dist()
    w = workload_kinect()
    if d.rank:
        w = replace(w, seed=rank_seed(w.seed, d.rank))
    seq = load_sequence(w, args.frames)
    nf = seq.depth.shape[0]
    W, H = w.width, w.height
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, W, H)
    depth_dev = torch.from_numpy(seq.depth).to(d.dev)
    stream = torch.cuda.Stream(device=d.dev)
    scene = Scene.from_workload(w, stream=stream)
    replay = graph_replayer(stream)
    pts = torch.empty((H, W, 4), dtype=torch.float32, device=d.dev)
    with torch.cuda.stream(stream):
        scene.integrate_frames(depth_dev, intr, seq.poses)
    fused = scene.stats()

    def raycast_all():
        for i in range(nf):
            scene.raycast(intr, seq.poses[i], Z_NEAR, points=pts)

    # eager pass: per-raycast counters
    samples = hits = wide = 0
    for i in range(nf):
        with torch.cuda.stream(stream):
            scene.raycast(intr, seq.poses[i], Z_NEAR, points=pts)
        rs = scene.raycast_stats()
        assert rs["guard_stops"] == 0
        samples += rs["steps"]
        hits += rs["hits"]
        wide += rs["wide_footprints"]
    last = rs
    l0 = scene.stats()["kernel_launches"]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        raycast_all()
    launches_per_step = scene.stats()["kernel_launches"] - l0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        replay(g)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    d.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        replay(g)
    e1.record(stream)
    d.barrier()
    clock_info = clocks.stop()
    ms_max = d.max(e0.elapsed_time(e1))
    assert scene.raycast_stats() == last, "graph replay disagrees with the eager raycasts"

    # march kernel durations: events around every march launch
    scene.timing_begin(nf, True)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=stream):
        raycast_all()
    replay(g2)
    torch.cuda.synchronize()
    marks = []
    for _ in range(args.steps):
        replay(g2)
        marks.append(scene.timing_read())
    scene.timing_end()
    marks = np.concatenate(marks)
    march_ms = marks[:, 2] - marks[:, 1]
    del g2

    # the per-frame loop of the pipeline: fuse frame t, then render pose t
    g3 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g3, stream=stream):
        scene.reset()
        for i in range(nf):
            scene.integrate(depth_dev[i], intr, seq.poses[i])
            scene.raycast(intr, seq.poses[i], Z_NEAR, points=pts)
    replay(g3)
    torch.cuda.synchronize()
    d.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        replay(g3)
    e1.record(stream)
    d.barrier()
    loop_ms = d.max(e0.elapsed_time(e1))
    del g3

    # end to end: every raycast through the public API, its point image read
    # back to pinned host memory
    e2e = None
    if not args.no_e2e:
        host = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()

        def e2e_step():
            with torch.cuda.stream(stream):
                for i in range(nf):
                    scene.raycast(intr, seq.poses[i], Z_NEAR, points=pts)
                    host.copy_(pts, non_blocking=True)
            stream.synchronize()

        e2e_step()
        d.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        d.barrier()
        dt_max = d.max(time.perf_counter() - t0)
        e2e = {"value": d.sum(float(nf * W * H * args.steps)) / dt_max, "unit": RAY_UNIT,
               "h2d_bytes_per_step": 128 * nf, "d2h_bytes_per_step": 16 * W * H * nf,
               "note": "h2d: the 4x4 FP64 pose of each raycast (carried into the kernels' "
                       "parameters); d2h: each point image"}

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        cpu = ray_cpu_baseline(w, seq, args.cpu_seconds)

    if d.rank == 0:
        rays_all = d.sum(float(nf * W * H * args.steps))
        # algorithmic bytes of one march launch: the point image written and,
        # per sample, the eight sdf values of its cell
        march_bytes = 16.0 * W * H + 8.0 * 4.0 * samples / nf
        peak, peak_kind = measured_peak_hbm()
        achieved = march_bytes / (float(np.mean(march_ms)) * 1e-3) / 1e9
        out = {
            "metric": RAY_METRIC, "value": rays_all / (ms_max * 1e-3), "unit": RAY_UNIT,
            "n_gpus": d.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name + "-raycast", "raycasts_per_step": nf,
                       "image": f"{W}x{H}", "voxel_size_m": w.voxel_size, "mu_m": w.mu,
                       "z_near_m": Z_NEAR, "pool_blocks": w.pool_blocks,
                       "storage": "f32 sdf + u8 weight",
                       "scene": f"the {nf}-frame sequence fused first (untimed), "
                                f"{fused['allocated_blocks']} blocks",
                       "graph": f"one CUDA graph per step ({nf} raycasts, one per pose)",
                       "l2": "inputs larger than L2: a step reads the whole fused scene "
                             f"({fused['allocated_blocks'] * 2560 / 1e6:.0f} MB of voxel data); "
                             "consecutive poses share blocks through L2 as consecutive "
                             "frames do",
                       "seed": w.seed},
            "raycasts_per_s": d.sum(float(nf * args.steps)) / (ms_max * 1e-3),
            "samples_per_ray": samples / (nf * W * H), "hit_fraction": hits / (nf * W * H),
            "wide_footprints_per_raycast": wide / nf,
            "march_us": float(np.mean(march_ms) * 1e3),
            "fuse_and_raycast_frames_per_s": d.sum(float(nf * args.steps)) / (loop_ms * 1e-3),
            "roofline": {"kernel": "raycast_kernel<f32>", "bound": "hbm", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": f"{peak_kind} (copy, burst)",
                         "traffic": profile_traffic(RAY_PROFILE, "raycast.cu",
                                                    "traffic_samples", samples / nf),
                         "algorithmic_bytes_per_launch": march_bytes,
                         "mean_launch_us": float(np.mean(march_ms) * 1e3)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clock_info,
        }
        print(json.dumps(out, default=float), flush=True)
    d.close()


COLOUR_METRIC = "voxel-updates/s (640x480, 5 mm, f32 sdf + colour)"
COLOUR_PROFILE = os.path.join(ROOT, "profiles", "integrate_colour_kinect_640x480_5mm.md")


def colour_cpu_baseline(w, seq, seconds: float) -> dict:
    """The FP64 oracle with colour, as it stands, single-threaded, on the
    first frames of the sequence until about `seconds` of CPU time."""
    import oracle
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                          max_weight=w.max_weight, storage=w.storage))
    intr = [f32(v) for v in (w.fx, w.fy, w.cx, w.cy)]
    t0 = time.perf_counter()
    n = 0
    while n < seq.depth.shape[0] and time.perf_counter() - t0 < seconds:
        o.integrate_rgb(seq.depth[n], seq.colour[n], intr, seq.poses[n])
        n += 1
    dt = time.perf_counter() - t0
    upd = o.total_updates()
    return {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {seq.depth.shape[0]} frames with colour, {upd} voxel "
                      f"updates in {dt:.1f} s (FP64 C oracle, 1 thread, host nproc {os.cpu_count()})"}


def run_colour(args):
    """Colour fusion (voxel clr / w_color, Section 3.1): the Kinect sequence
    with registered RGBX colour images; one step = reset + every frame through
    tsdf_integrate_rgb, in one CUDA graph. The same step without colour
    (tsdf_integrate frame by frame) is timed beside it."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from paper_1410_0925_gb300.tsdf import STAGES
    from synthdepth import workload_kinect

    d = Dist()
    w = workload_kinect()
    if d.rank:
        w = replace(w, seed=rank_seed(w.seed, d.rank))
    seq = load_sequence(w, args.frames, colour=True)
    nf = seq.depth.shape[0]
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth_dev = torch.from_numpy(seq.depth).to(d.dev)
    col_dev = torch.from_numpy(seq.colour).to(d.dev)
    stream = torch.cuda.Stream(device=d.dev)
    replay = graph_replayer(stream)
    scene = Scene.from_workload(w, stream=stream)
    scene.enable_colour()
    plain = Scene.from_workload(w, stream=stream)

    def step_colour():
        scene.reset()
        for i in range(nf):
            scene.integrate_rgb(depth_dev[i], col_dev[i], intr, seq.poses[i])

    def step_plain():
        plain.reset()
        for i in range(nf):
            plain.integrate(depth_dev[i], intr, seq.poses[i])

    with torch.cuda.stream(stream):
        step_colour()
        step_plain()
    st_c, st_p = scene.stats(), plain.stats()
    assert st_c["total_updated_voxels"] == st_p["total_updated_voxels"]
    upd = st_c["total_updated_voxels"]

    def timed(step, clocks=None):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        if clocks is not None:
            clocks.start()
        for _ in range(args.warmup):
            replay(g)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        d.barrier()
        e0.record(stream)
        for _ in range(args.steps):
            replay(g)
        e1.record(stream)
        d.barrier()
        info = clocks.stop() if clocks is not None else None
        return d.max(e0.elapsed_time(e1)), info

    l0 = scene.stats()["kernel_launches"]
    clocks = ClockSampler(torch.cuda.current_device())
    ms_c, clock_info = timed(step_colour, clocks)
    # the counter counts calls into the library, made once at capture
    launches_per_step = scene.stats()["kernel_launches"] - l0
    ms_p, _ = timed(step_plain)
    assert scene.stats()["total_updated_voxels"] == upd

    # integration kernel durations with colour: events around every launch
    scene.timing_begin(nf, True)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step_colour()
    replay(g)
    torch.cuda.synchronize()
    marks = []
    for _ in range(args.steps):
        replay(g)
        marks.append(scene.timing_read())
    scene.timing_end()
    marks = np.concatenate(marks)
    ib = STAGES.index("integrate")
    integ_ms = marks[:, ib + 1] - marks[:, ib]
    vis = st_c["total_visible_blocks"]
    # per updated voxel: sdf + weight read and written (10 B), its colour word
    # read and written (8 B) and its pixel's colour (4 B); per visible block
    # its 32 B record; per pixel the depth (4 B)
    integ_bytes = (22.0 * upd + 32.0 * vis) / nf + 4.0 * w.width * w.height

    e2e = None
    if not args.no_e2e:
        pin_d = torch.from_numpy(seq.depth).pin_memory()
        pin_c = torch.from_numpy(seq.colour).pin_memory()
        sd, sc_ = torch.empty_like(depth_dev), torch.empty_like(col_dev)

        def e2e_step():
            with torch.cuda.stream(stream):
                sd.copy_(pin_d, non_blocking=True)
                sc_.copy_(pin_c, non_blocking=True)
                scene.reset()
                for i in range(nf):
                    scene.integrate_rgb(sd[i], sc_[i], intr, seq.poses[i])
            return scene.stats()

        e2e_step()
        d.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st_e = e2e_step()
        d.barrier()
        dt = d.max(time.perf_counter() - t0)
        assert st_e["total_updated_voxels"] == upd
        e2e = {"value": d.sum(float(upd * args.steps)) / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(seq.depth.nbytes + seq.colour.nbytes),
               "d2h_bytes_per_step": 64}

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        cpu = colour_cpu_baseline(w, seq, args.cpu_seconds)

    if d.rank == 0:
        value = d.sum(float(upd * args.steps)) / (ms_c * 1e-3)
        plain_value = d.sum(float(upd * args.steps)) / (ms_p * 1e-3)
        peak, peak_kind = measured_peak_hbm()
        achieved = integ_bytes / (float(np.mean(integ_ms)) * 1e-3) / 1e9
        out = {
            "metric": COLOUR_METRIC, "value": value, "unit": UNIT, "n_gpus": d.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_c / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 sdf, u8 colour", "data": "synthetic",
            "config": {"workload": w.name + "-colour", "frames_per_step": nf,
                       "image": f"{w.width}x{w.height} depth + RGBX colour",
                       "voxel_size_m": w.voxel_size, "mu_m": w.mu,
                       "pool_blocks": w.pool_blocks,
                       "storage": "f32 sdf + u8 weight + u8x4 colour",
                       "graph": f"one CUDA graph per step (reset + {nf} frames, frame by frame)",
                       "l2": "inputs larger than L2: depth 368 MB + colour 368 MB + voxels "
                             "1.2 GB resident", "seed": w.seed},
            "frames_per_s": d.sum(float(nf * args.steps)) / (ms_c * 1e-3),
            "depth_only_same_loop": {"value": plain_value,
                                     "frames_per_s": d.sum(float(nf * args.steps)) / (ms_p * 1e-3)},
            "colour_cost": ms_c / ms_p,
            "roofline": {"kernel": "integrate_kernel<f32, colour>", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": f"{peak_kind} (copy, burst)",
                         "traffic": profile_traffic(COLOUR_PROFILE, "integrate.cu",
                                                    "traffic_updated_voxels", upd / nf),
                         "algorithmic_bytes_per_launch": integ_bytes,
                         "mean_launch_us": float(np.mean(integ_ms) * 1e3)},
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clock_info,
        }
        print(json.dumps(out, default=float), flush=True)
    d.close()


ICP_METRIC = "pixels/s (640x480 point-to-plane terms of the depth tracker)"
ICP_PROFILE = os.path.join(ROOT, "profiles", "icp_reduce_kinect_640x480.md")
ICP_UNIT = "pixels/s"
ICP_ITERS = 10


def icp_cpu_baseline(w, seq, seconds: float) -> dict:
    """The FP64 tracker oracle, as it stands, single-threaded: normals and
    terms of frames 1, 2, ... against the exact synthetic view of the frame
    before (its point map built outside the timed part), until about
    `seconds` of CPU time."""
    import oracle
    from synthdepth.configs import sequence_geometry
    from synthdepth.scene import raycast_depth
    scene, _, world_from_room = sequence_geometry(w, 1)
    intr = [float(np.float32(v)) for v in (w.fx, w.fy, w.cx, w.cy)]
    u, v = np.meshgrid(np.arange(w.width, dtype=np.float64), np.arange(w.height, dtype=np.float64))
    rays = np.stack([(u - w.cx) / w.fx, (v - w.cy) / w.fy, np.ones_like(u)], -1)
    spent, n = 0.0, 0
    while n + 1 < seq.depth.shape[0] and spent < seconds:
        pose = seq.poses[n]
        dref = raycast_depth(scene, pose @ world_from_room, w.width, w.height, w.fx, w.fy,
                             w.cx, w.cy)
        Minv = np.linalg.inv(pose)
        Vh = np.zeros((w.height, w.width, 4), np.float32)
        ok = dref > 0
        Vh[ok, :3] = ((rays * dref[..., None]) @ Minv[:3, :3].T + Minv[:3, 3])[ok]
        Vh[ok, 3] = 1.0
        t1 = time.perf_counter()
        No = oracle.icp_normals(Vh)
        oracle.icp_reduce(seq.depth[n + 1], intr, pose, pose, Vh, No, 0.1)
        spent += time.perf_counter() - t1
        n += 1
    px = n * w.width * w.height
    return {"value": px / spent, "unit": ICP_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"normals + terms of frames 1..{n} against the exact view of the frame "
                      f"before, {spent:.1f} s (FP64 C oracle, 1 thread, host nproc "
                      f"{os.cpu_count()})"}


def run_icp(args):
    """The depth tracker's terms (Section 4.1): the 300-frame Kinect sequence
    is fused (untimed) and rendered from every pose (tsdf_raycast) into
    reference point maps with normal maps (tsdf_icp_normals); one step
    reduces the terms of every frame t against the maps of frame t - 1,
    from that pose (299 tsdf_icp_reduce calls in one CUDA graph). The
    tracking loop (raycast, normals, 10 Gauss-Newton iterations on the
    device) is timed end to end."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Icp, Scene, make_intrinsics
    from synthdepth import workload_kinect

    d = Dist()
    w = workload_kinect()
    if d.rank:
        w = replace(w, seed=rank_seed(w.seed, d.rank))
    seq = load_sequence(w, args.frames)
    nf = seq.depth.shape[0]
    W, H = w.width, w.height
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, W, H)
    depth_dev = torch.from_numpy(seq.depth).to(d.dev)
    stream = torch.cuda.Stream(device=d.dev)
    replay = graph_replayer(stream)
    scene = Scene.from_workload(w, stream=stream)
    icp = Icp(stream=stream)
    V = torch.empty((nf, H, W, 4), dtype=torch.float32, device=d.dev)
    N = torch.empty_like(V)
    S = torch.zeros((nf, Icp.TERMS), dtype=torch.float64, device=d.dev)
    with torch.cuda.stream(stream):
        scene.integrate_frames(depth_dev, intr, seq.poses)
        for t in range(nf):
            scene.raycast(intr, seq.poses[t], Z_NEAR, points=V[t])
            icp.normals(V[t], out=N[t])
    stream.synchronize()

    def step():
        for t in range(1, nf):
            icp.reduce(depth_dev[t], intr, seq.poses[t - 1], seq.poses[t - 1], V[t - 1], N[t - 1],
                       0.1, sums=S[t])

    with torch.cuda.stream(stream):
        step()
    stream.synchronize()
    ref = S.clone()
    l0 = icp.kernel_launches()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step()
    launches_per_step = icp.kernel_launches() - l0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        replay(g)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    d.barrier()
    # a step takes ~3 ms: at least 150 of them, so that the clock sampler
    # (50 ms) sees the timed region several times
    steps = max(args.steps, 150)
    e0.record(stream)
    for _ in range(steps):
        replay(g)
    e1.record(stream)
    d.barrier()
    clock_info = clocks.stop()
    ms = d.max(e0.elapsed_time(e1))
    assert torch.equal(S, ref), "graph replay disagrees with the eager reductions"
    inliers = float(S[1:, 28].sum().item())
    reduce_us = ms * 1e3 / (steps * (nf - 1))

    # the tracking loop, end to end: per frame the depth from pinned host
    # memory, the raycast from the previous estimate, normals, and 10
    # Gauss-Newton iterations on the device (tsdf_icp_track: terms, 6x6
    # solve and pose update without a host round trip); the estimate is read
    # back once per frame for the next raycast
    e2e = None
    loop_frames = min(nf - 1, 60)
    if not args.no_e2e:
        pinned = torch.from_numpy(seq.depth).pin_memory()
        staging = torch.empty((H, W), dtype=torch.float32, device=d.dev)
        Vr = torch.empty((H, W, 4), dtype=torch.float32, device=d.dev)
        Nr = torch.empty_like(Vr)
        pose_dev = torch.empty((4, 4), dtype=torch.float64, device=d.dev)
        pose_host = torch.empty((4, 4), dtype=torch.float64).pin_memory()

        def track():
            est = seq.poses[0].copy()
            drift = 0.0
            for t in range(1, loop_frames + 1):
                pose_host.copy_(torch.from_numpy(est))
                with torch.cuda.stream(stream):
                    staging.copy_(pinned[t], non_blocking=True)
                    pose_dev.copy_(pose_host, non_blocking=True)
                    scene.raycast(intr, est, Z_NEAR, points=Vr)
                    icp.normals(Vr, out=Nr)
                    icp.track(staging, intr, pose_dev, est, Vr, Nr, 0.1, iterations=ICP_ITERS)
                    pose_host.copy_(pose_dev, non_blocking=True)
                stream.synchronize()
                est = pose_host.numpy().copy()
                drift = max(drift, float(np.linalg.norm((np.linalg.inv(est) @ seq.poses[t])[:3, 3])))
            assert icp.status() == 0, "a tracking step was skipped or singular"
            return drift

        track()
        d.barrier()
        t0 = time.perf_counter()
        drift = track()
        d.barrier()
        dt = d.max(time.perf_counter() - t0)
        e2e = {"value": d.sum(float(loop_frames * ICP_ITERS * W * H)) / dt, "unit": ICP_UNIT,
               "h2d_bytes_per_step": int(loop_frames * (W * H * 4 + 128)),
               "d2h_bytes_per_step": int(loop_frames * 128),
               "tracking_frames_per_s": d.sum(float(loop_frames)) / dt,
               "max_translation_error_m": drift,
               "note": f"{loop_frames} frames tracked from the first pose: per frame the depth "
                       f"and pose copies, a raycast from the current estimate, normals and "
                       f"{ICP_ITERS} Gauss-Newton iterations on the device (terms, 6x6 solve, "
                       "pose update), the pose read back once"}

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        cpu = icp_cpu_baseline(w, seq, args.cpu_seconds)

    if d.rank == 0:
        # bytes of one reduction: every pixel's depth, and for each associated
        # pixel the reference point and normal (16 B each)
        bytes_launch = 4.0 * W * H + 32.0 * inliers / (nf - 1)
        peak, peak_kind = measured_peak_hbm()
        achieved = bytes_launch / (reduce_us * 1e-6) / 1e9
        out = {
            "metric": ICP_METRIC, "value": d.sum(float((nf - 1) * W * H * steps)) / (ms * 1e-3),
            "unit": ICP_UNIT, "n_gpus": d.world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 terms, f64 sums", "data": "synthetic",
            "config": {"workload": w.name + "-icp", "reductions_per_step": nf - 1,
                       "image": f"{W}x{H}", "max_dist_m": 0.1,
                       "reference": "raycast of the fused 300-frame scene from the previous pose",
                       "graph": f"one CUDA graph per step ({nf - 1} reductions)",
                       "l2": "inputs larger than L2: 300 depth frames (368 MB) + point and "
                             "normal maps (2.9 GB) resident", "seed": w.seed},
            "reductions_per_s": d.sum(float((nf - 1) * steps)) / (ms * 1e-3),
            "inliers_per_reduction": inliers / (nf - 1),
            "roofline": {"kernel": "icp_reduce_kernel", "bound": "hbm", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": f"{peak_kind} (copy, burst)",
                         "traffic": profile_traffic(ICP_PROFILE, "icp.cu", "traffic_pixels",
                                                    float(W * H)),
                         "algorithmic_bytes_per_launch": bytes_launch,
                         "mean_launch_us": reduce_us},
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches_per_step * steps),
            "clocks": clock_info,
        }
        print(json.dumps(out, default=float), flush=True)
    d.close()


SWAP_METRIC = "voxel-updates/s (640x480, 5 mm, f32 sdf, swapping every frame)"
def swap_cpu_baseline(w, seq, seconds: float) -> dict:
    """The FP64 oracle with the same swap schedule, as it stands, one thread,
    on the first frames until about `seconds` of CPU time."""
    import oracle
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                          max_weight=w.max_weight, storage=w.storage,
                                          pool_blocks=w.pool_blocks))
    intr = [f32(v) for v in (w.fx, w.fy, w.cx, w.cy)]
    t0 = time.perf_counter()
    n = 0
    while n < seq.depth.shape[0] and time.perf_counter() - t0 < seconds:
        P = seq.poses[n]
        o.swap_in(w.width, w.height, intr, P, SWAP_MARGIN_PX, 0.0, SWAP_CAPACITY)
        o.integrate(seq.depth[n], intr, P)
        o.swap_out(w.width, w.height, intr, P, SWAP_MARGIN_PX, 0.0, SWAP_CAPACITY)
        n += 1
    dt = time.perf_counter() - t0
    upd = o.total_updates()
    return {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {seq.depth.shape[0]} frames with the swap schedule, "
                      f"{upd} voxel updates in {dt:.1f} s (FP64 C oracle, 1 thread, "
                      f"host nproc {os.cpu_count()})"}


def run_swap(args):
    """Swapping (Section 5) on the 300-frame Kinect sequence: every frame
    swaps in what the view sees (16 px margin), fuses, and swaps out what it
    does not, at most 4096 blocks per call, the host copies in mapped pinned
    host memory. One step = reset + the whole sequence in one CUDA graph. The
    same loop without swapping is timed beside it."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from paper_1410_0925_gb300.tsdf import STAGES
    from synthdepth import workload_kinect

    d = Dist()
    w = workload_kinect()
    if d.rank:
        w = replace(w, seed=rank_seed(w.seed, d.rank))
    seq = load_sequence(w, args.frames)
    nf = seq.depth.shape[0]
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth_dev = torch.from_numpy(seq.depth).to(d.dev)
    stream = torch.cuda.Stream(device=d.dev)
    replay = graph_replayer(stream)
    scene = Scene.from_workload(w, stream=stream)
    scene.enable_swapping(SWAP_CAPACITY)
    plain = Scene.from_workload(w, stream=stream)

    def step_swap():
        scene.reset()
        swap_step_ops(scene, depth_dev, intr, seq.poses)

    def step_plain():
        plain.reset()
        for i in range(nf):
            plain.integrate(depth_dev[i], intr, seq.poses[i])

    with torch.cuda.stream(stream):
        step_swap()
        step_plain()
    st_s, st_p = scene.stats(), plain.stats()
    sw = scene.swap_stats()
    upd = st_s["total_updated_voxels"]

    def timed(step, clocks=None):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        if clocks is not None:
            clocks.start()
        for _ in range(args.warmup):
            replay(g)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        d.barrier()
        e0.record(stream)
        for _ in range(args.steps):
            replay(g)
        e1.record(stream)
        d.barrier()
        info = clocks.stop() if clocks is not None else None
        return d.max(e0.elapsed_time(e1)), info

    l0 = scene.stats()["kernel_launches"]
    clocks = ClockSampler(torch.cuda.current_device())
    ms_s, clock_info = timed(step_swap, clocks)
    launches_per_step = scene.stats()["kernel_launches"] - l0
    ms_p, _ = timed(step_plain)
    assert scene.stats()["total_updated_voxels"] == upd

    # integration kernel durations inside the swapping step
    scene.timing_begin(nf, True)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step_swap()
    replay(g)
    torch.cuda.synchronize()
    marks = []
    for _ in range(args.steps):
        replay(g)
        marks.append(scene.timing_read())
    scene.timing_end()
    marks = np.concatenate(marks)
    ib = STAGES.index("integrate")
    integ_ms = marks[:, ib + 1] - marks[:, ib]
    vis = st_s["total_visible_blocks"]
    integ_bytes = (bytes_per_update(w.storage) * upd + 32.0 * vis) / nf + 4.0 * w.width * w.height

    e2e = None
    if not args.no_e2e:
        pin_d = torch.from_numpy(seq.depth).pin_memory()
        sd = torch.empty_like(depth_dev)

        def e2e_step():
            with torch.cuda.stream(stream):
                sd.copy_(pin_d, non_blocking=True)
                scene.reset()
                swap_step_ops(scene, sd, intr, seq.poses)
            return scene.stats()

        e2e_step()
        d.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st_e = e2e_step()
        d.barrier()
        dt = d.max(time.perf_counter() - t0)
        assert st_e["total_updated_voxels"] == upd
        e2e = {"value": d.sum(float(upd * args.steps)) / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(seq.depth.nbytes), "d2h_bytes_per_step": 64}

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        cpu = swap_cpu_baseline(w, seq, args.cpu_seconds)

    if d.rank == 0:
        value = d.sum(float(upd * args.steps)) / (ms_s * 1e-3)
        peak, peak_kind = measured_peak_hbm()
        achieved = integ_bytes / (float(np.mean(integ_ms)) * 1e-3) / 1e9
        block_bytes = 512 * 5  # f32 sdf + u8 weight
        moved = sw["total_out"] + sw["total_in"]
        out = {
            "metric": SWAP_METRIC, "value": value, "unit": UNIT, "n_gpus": d.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name + "-swap", "frames_per_step": nf,
                       "transfer_blocks": SWAP_CAPACITY, "margin_px": SWAP_MARGIN_PX,
                       "host_store": "mapped pinned host memory, one block slot per hash entry",
                       "graph": f"one CUDA graph per step (reset + {nf} x (swap in, fuse, "
                                f"swap out))",
                       "l2": "inputs larger than L2: depth 368 MB + voxels 1.2 GB resident",
                       "seed": w.seed},
            "frames_per_s": d.sum(float(nf * args.steps)) / (ms_s * 1e-3),
            "without_swapping": {"value": d.sum(float(st_p["total_updated_voxels"] * args.steps))
                                 / (ms_p * 1e-3),
                                 "frames_per_s": d.sum(float(nf * args.steps)) / (ms_p * 1e-3)},
            "swap_cost": ms_s / ms_p,
            "updates_equal_without_swapping": upd == st_p["total_updated_voxels"],
            "swap": {"blocks_out_per_step": sw["total_out"], "blocks_in_per_step": sw["total_in"],
                     "merged_per_step": sw["total_merged"],
                     "host_blocks_at_end": sw["host_blocks"],
                     "device_blocks_at_end": st_s["allocated_blocks"],
                     "bytes_moved_per_step": moved * block_bytes,
                     "extra_ms_per_frame": (ms_s - ms_p) / args.steps / nf},
            "roofline": {"kernel": integ_kernel_name(STORAGE_F32, False), "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": f"{peak_kind} (copy, burst)",
                         "traffic": None,
                         "algorithmic_bytes_per_launch": integ_bytes,
                         "mean_launch_us": float(np.mean(integ_ms) * 1e3)},
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clock_info,
        }
        print(json.dumps(out, default=float), flush=True)
    d.close()


ENGINE_METRIC = "frames/s (640x480 sequence through the whole pipeline: track, fuse, render)"
ENGINE_LEVELS, ENGINE_ITERATIONS, ENGINE_MAX_DIST = 3, (4, 4, 6), 0.1


def _rodrigues(wv):
    th = float(np.linalg.norm(wv))
    if th < 1e-15:
        return np.eye(3)
    k = wv / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def engine_cpu_baseline(w, seq, seconds: float) -> dict:
    """The pipeline of one camera composed from the FP64 oracles as they
    stand, one thread: per frame the depth hierarchy, the oracle's raycast of
    its own fused volume from the last pose at every level, normals, the
    point-to-plane terms with a host Gauss-Newton step per iteration (coarse
    to fine, the engine's iteration counts), then fusion at the tracked pose;
    until about `seconds` of CPU time."""
    import oracle
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    o = oracle.Oracle(oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                                          max_weight=w.max_weight, storage=w.storage))
    rp = oracle.RayParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu), z_near=f32(Z_NEAR))
    levels = []
    fx, fy, cx, cy, W, H = (f32(w.fx), f32(w.fy), f32(w.cx), f32(w.cy), w.width, w.height)
    for lvl in range(ENGINE_LEVELS):
        if lvl:
            fx, fy, cx, cy, W, H = fx / 2, fy / 2, (cx - 0.5) / 2, (cy - 0.5) / 2, W // 2, H // 2
        levels.append(((fx, fy, cx, cy), W, H))
    pose = np.array(seq.poses[0], np.float64)
    t0 = time.perf_counter()
    n = 0
    worst = 0.0
    while n < seq.depth.shape[0] and time.perf_counter() - t0 < seconds:
        depth = seq.depth[n]
        if n > 0:
            pyr = [depth]
            for _ in range(1, ENGINE_LEVELS):
                pyr.append(oracle.icp_downsample(pyr[-1]))
            r = o.read()
            vol = oracle.Volume(r["keys"], r["sdf"])
            ref, cur = pose.copy(), pose.copy()
            for lvl in reversed(range(ENGINE_LEVELS)):
                intr_l, W_l, H_l = levels[lvl]
                V = vol.raycast(W_l, H_l, intr_l, ref, rp)["points"].reshape(H_l, W_l, 4)
                V = V.astype(np.float32)
                N = oracle.icp_normals(V)
                for _ in range(ENGINE_ITERATIONS[lvl]):
                    out = oracle.icp_reduce(pyr[lvl], intr_l, cur, ref, V, N, ENGINE_MAX_DIST)
                    Hm, g = oracle.icp_system(out["sums"])
                    if out["sums"][28] < 6:
                        break
                    try:
                        np.linalg.cholesky(Hm)
                    except np.linalg.LinAlgError:
                        break
                    xi = -np.linalg.solve(Hm, g)
                    step = np.eye(4)
                    step[:3, :3] = _rodrigues(xi[:3])
                    step[:3, 3] = xi[3:]
                    cur = cur @ np.linalg.inv(step)
            vol.close()
            pose = cur
        o.integrate(depth, levels[0][0], pose)
        worst = max(worst, float(np.linalg.norm((np.linalg.inv(pose) @ seq.poses[n])[:3, 3])))
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {seq.depth.shape[0]} frames through the oracle pipeline "
                      f"(raycast at {ENGINE_LEVELS} levels, {sum(ENGINE_ITERATIONS)} host "
                      f"Gauss-Newton steps, fusion) in {dt:.1f} s, largest translation error "
                      f"{worst * 1e3:.1f} mm (FP64 C oracles, 1 thread, host nproc "
                      f"{os.cpu_count()})"}


def run_engine(args):
    """The processing pipeline of one camera (tsdf_engine_process, Section
    2.1) on the 300-frame Kinect sequence from its first pose: per frame the
    depth hierarchy, the model rendered from the last pose at 3 levels, 14
    Gauss-Newton iterations on the device (4 + 4 + 6, coarse to fine), one
    pose read-back, and the fusion at the tracked pose. One step = the whole
    sequence from an emptied model (host clock: every frame synchronises)."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Engine, make_intrinsics
    from synthdepth import workload_kinect

    d = Dist()
    w = workload_kinect()
    if d.rank:
        w = replace(w, seed=rank_seed(w.seed, d.rank))
    seq = load_sequence(w, args.frames)
    nf = seq.depth.shape[0]
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth_dev = torch.from_numpy(seq.depth).to(d.dev)
    stream = torch.cuda.Stream(device=d.dev)
    eng = Engine(w.scene_desc(), intr, seq.poses[0], levels=ENGINE_LEVELS,
                 iterations=ENGINE_ITERATIONS, max_dist=ENGINE_MAX_DIST, stream=stream)

    def one_pass(src, host=None):
        eng.reset(seq.poses[0])
        worst = 0.0
        with torch.cuda.stream(stream):
            for i in range(nf):
                if host is not None:
                    src[i % 2].copy_(host[i], non_blocking=True)
                    pose = eng.process(src[i % 2])
                else:
                    pose = eng.process(src[i])
                worst = max(worst, float(np.linalg.norm((np.linalg.inv(pose) @ seq.poses[i])[:3, 3])))
        return worst

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        one_pass(depth_dev)
    d.barrier()
    l0 = eng.kernel_launches()
    t0 = time.perf_counter()
    worst = 0.0
    for _ in range(args.steps):
        worst = max(worst, one_pass(depth_dev))
    d.barrier()
    dt = d.max(time.perf_counter() - t0)
    launches = eng.kernel_launches() - l0
    clock_info = clocks.stop()
    assert eng.tracker_status() == 0, "a tracking step was skipped or singular"
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(seq.depth).pin_memory()
        staging = torch.empty((2, w.height, w.width), dtype=torch.float32, device=d.dev)
        one_pass(staging, pinned)
        d.barrier()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            one_pass(staging, pinned)
        d.barrier()
        dte = d.max(time.perf_counter() - t1)
        e2e = {"value": d.sum(float(nf * args.steps)) / dte, "unit": "frames/s",
               "h2d_bytes_per_step": int(seq.depth.nbytes), "d2h_bytes_per_step": 128 * nf}
    if d.rank == 0:
        cpu = None
        if d.world == 1 and not args.no_cpu_baseline:
            cpu = engine_cpu_baseline(w, seq, args.cpu_seconds)
        fps = d.sum(float(nf * args.steps)) / dt
        out = {
            "metric": ENGINE_METRIC, "value": fps, "unit": "frames/s", "n_gpus": d.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name + "-engine", "frames_per_step": nf,
                       "tracker": "3 levels, 4 + 4 + 6 Gauss-Newton iterations on the device, "
                                  "max_dist 0.1 m",
                       "timing": "host clock around whole passes (each frame reads its pose back)",
                       "l2": "inputs larger than L2: depth frames 368 MB + voxels 671 MB",
                       "seed": w.seed},
            "max_translation_error_m": worst,
            "roofline": None, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clock_info,
        }
        print(json.dumps(out, default=float), flush=True)
    d.close()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "hd":
        run_hd(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "raycast":
        run_raycast(args)
    elif args.workload == "colour":
        run_colour(args)
    elif args.workload == "icp":
        run_icp(args)
    elif args.workload == "engine":
        run_engine(args)
    elif args.workload == "swap":
        run_swap(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
