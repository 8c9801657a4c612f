"""Python binding of libtsdf (include/tsdf.h): argument marshalling only.

Every step of the fusion path runs in the library's CUDA kernels; this module
converts arguments (torch tensors, numpy arrays, Python numbers) into the
pointers and structs of the C ABI and turns status codes into exceptions.
There is no fallback: if the library cannot be loaded or no CUDA device is
usable, the calls raise.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsdf.so")

TSDF_OK = 0
TSDF_ERR_INVALID_ARG = -1
TSDF_ERR_OUT_OF_MEMORY = -2
TSDF_ERR_POOL_EXHAUSTED = -3
TSDF_ERR_EXCESS_EXHAUSTED = -4
TSDF_ERR_CUDA = -5
TSDF_ERR_TIMEOUT = -6
TSDF_ERR_CAPACITY = -7
TSDF_ERR_KEY_RANGE = -8
TSDF_ERR_INTERNAL = -9

STORAGE_F32, STORAGE_I16, STORAGE_F16 = 0, 1, 2
SDF_DTYPE = {STORAGE_F32: np.float32, STORAGE_I16: np.int16, STORAGE_F16: np.float16}

EXPORTED = ["tsdf_scene_create", "tsdf_scene_destroy", "tsdf_scene_reset",
            "tsdf_scene_set_stream", "tsdf_scene_device", "tsdf_integrate", "tsdf_sync",
            "tsdf_get_stats", "tsdf_num_blocks", "tsdf_read_blocks",
            "tsdf_load_blocks", "tsdf_lookup_blocks", "tsdf_status_string",
            "tsdf_timing_begin", "tsdf_timing_read", "tsdf_timing_end",
            "tsdf_read_blocks_device_noalloc", "tsdf_batch_create", "tsdf_batch_destroy",
            "tsdf_batch_prepare", "tsdf_batch_launch", "tsdf_batch_integrate",
            "tsdf_batch_set_config", "tsdf_batch_get_config", "tsdf_batch_autotune",
            "tsdf_batch_kernel_launches", "tsdf_batch_cursor", "tsdf_batch_set_cursor",
            "tsdf_batch_timing_begin", "tsdf_batch_timing_read", "tsdf_batch_timing_end",
            "tsdf_admission_create", "tsdf_admission_destroy", "tsdf_admission_enqueue",
            "tsdf_admission_cancel", "tsdf_admission_admit", "tsdf_admission_release",
            "tsdf_admission_stats", "tsdf_scene_device_bytes", "tsdf_server_create",
            "tsdf_server_destroy", "tsdf_server_open", "tsdf_server_submit", "tsdf_server_close",
            "tsdf_server_step", "tsdf_server_poll", "tsdf_server_session_info",
            "tsdf_server_scene", "tsdf_server_release", "tsdf_server_trim",
            "tsdf_integrate_frames", "tsdf_batch_join", "tsdf_raycast",
            "tsdf_get_raycast_stats", "tsdf_scene_enable_colour", "tsdf_integrate_rgb",
            "tsdf_read_colour", "tsdf_icp_create", "tsdf_icp_destroy", "tsdf_icp_normals",
            "tsdf_icp_reduce", "tsdf_icp_kernel_launches", "tsdf_icp_solve", "tsdf_icp_track",
            "tsdf_icp_status", "tsdf_icp_downsample", "tsdf_icp_level_intrinsics", "tsdf_engine_create", "tsdf_engine_destroy",
            "tsdf_engine_process", "tsdf_engine_scene", "tsdf_engine_tracker_status",
            "tsdf_engine_reset", "tsdf_scene_enable_swapping", "tsdf_swap_out", "tsdf_swap_in",
            "tsdf_get_swap_stats", "tsdf_read_host_blocks", "tsdf_swap_visibility",
            "tsdf_engine_kernel_launches", "tsdf_swap_merge_voxels"]

READ_NOALLOC_MAX_BLOCKS = 1 << 18

STAGES = ["alloc", "integrate"]  # kernels of one fusion step, in order


class TsdfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class SceneDesc(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("mu", ctypes.c_float),
                ("max_weight", ctypes.c_int32),
                ("hash_buckets_log2", ctypes.c_int32),
                ("entries_per_bucket", ctypes.c_int32),
                ("excess_entries", ctypes.c_int32),
                ("pool_blocks", ctypes.c_int32), ("storage", ctypes.c_int32)]


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Frame(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("pitch_elems", ctypes.c_int64), ("intr", Intrinsics),
                ("world_to_cam", ctypes.c_double * 16), ("depth_on_host", ctypes.c_int32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("integrate_ctas_per_sm", ctypes.c_int32), ("pipelined", ctypes.c_int32),
                ("integrate_kernel", ctypes.c_int32), ("integrate_threads", ctypes.c_int32),
                ("alloc_tile", ctypes.c_int32)]

    KERNELS = {0: "staged", 1: "general"}
    TILES = {0: "16x16", 1: "16x8", 2: "32x8"}

    def as_dict(self) -> dict:
        return {"integrate_kernel": self.KERNELS.get(int(self.integrate_kernel), "?"),
                "integrate_threads": int(self.integrate_threads),
                "integrate_ctas_per_sm": int(self.integrate_ctas_per_sm),
                "alloc_tile": self.TILES.get(int(self.alloc_tile), "?"),
                "pipelined": bool(self.pipelined)}


class ServerConfig(ctypes.Structure):
    _fields_ = [("pool_budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("max_queued_frames", ctypes.c_int32), ("max_inflight_steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class StepInfo(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int32), ("launched_frames", ctypes.c_int32),
                ("active_sessions", ctypes.c_int32), ("queued_sessions", ctypes.c_int32),
                ("inflight_steps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("active_bytes", ctypes.c_int64), ("cached_bytes", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "reserved"}


class FrameDone(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("session", ctypes.c_int64),
                ("submit_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class SessionInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("frames_submitted", ctypes.c_int64),
                ("frames_launched", ctypes.c_int64), ("frames_done", ctypes.c_int64),
                ("open_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("finish_ms", ctypes.c_double), ("updated_voxels", ctypes.c_int64),
                ("allocated_blocks", ctypes.c_int64), ("device_status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


SESSION_QUEUED, SESSION_ACTIVE, SESSION_FINISHED, SESSION_FAILED = 0, 1, 2, 3


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "frames", "allocated_blocks", "last_new_blocks", "last_visible_blocks",
        "last_updated_voxels", "total_updated_voxels", "total_visible_blocks",
        "excess_used", "kernel_launches")]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class EngineConfig(ctypes.Structure):
    _fields_ = [("scene", SceneDesc), ("intr", Intrinsics), ("levels", ctypes.c_int32),
                ("iterations", ctypes.c_int32 * 4), ("max_dist", ctypes.c_float),
                ("z_near", ctypes.c_float), ("colour", ctypes.c_int32),
                ("swap_blocks", ctypes.c_int32), ("swap_margin_px", ctypes.c_float)]


class RaycastStats(ctypes.Structure):
    _fields_ = [("footprints", ctypes.c_int64), ("wide_footprints", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("hits", ctypes.c_int64),
                ("guard_stops", ctypes.c_int64)]


class SwapStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "host_blocks", "transfer_blocks", "last_out_candidates", "last_out",
        "last_in_candidates", "last_in", "last_merged", "total_out", "total_in",
        "total_merged")]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtsdf.so (built by paper_1410_0925_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtsdf.so not built ({path}); run paper_1410_0925_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "tsdf_scene_create": [P(SceneDesc), vp, P(vp)],
        "tsdf_scene_destroy": [vp],
        "tsdf_scene_reset": [vp],
        "tsdf_scene_set_stream": [vp, vp],
        "tsdf_scene_device": [vp, vp],
        "tsdf_icp_level_intrinsics": [vp, i32, vp],
        "tsdf_integrate": [vp, vp, i64, i32, P(Intrinsics), vp],
        "tsdf_sync": [vp],
        "tsdf_get_stats": [vp, P(Stats)],
        "tsdf_num_blocks": [vp, P(i64)],
        "tsdf_read_blocks": [vp, vp, vp, vp, i64, P(i64)],
        "tsdf_load_blocks": [vp, vp, vp, vp, i64],
        "tsdf_lookup_blocks": [vp, vp, i64, vp],
        "tsdf_timing_begin": [vp, ctypes.c_int32, ctypes.c_int32],
        "tsdf_timing_read": [vp, vp, i64, P(i64)],
        "tsdf_timing_end": [vp],
        "tsdf_read_blocks_device_noalloc": [vp, vp, vp, vp, i64, P(i64)],
        "tsdf_batch_create": [ctypes.c_int32, ctypes.c_int32, vp, P(vp)],
        "tsdf_batch_cursor": [vp, P(ctypes.c_int32)],
        "tsdf_batch_set_cursor": [vp, ctypes.c_int32],
        "tsdf_batch_timing_begin": [vp, ctypes.c_int32, ctypes.c_int32],
        "tsdf_batch_timing_read": [vp, vp, i64, P(i64)],
        "tsdf_batch_timing_end": [vp],
        "tsdf_admission_create": [i64, ctypes.c_int32, P(vp)],
        "tsdf_admission_destroy": [vp],
        "tsdf_admission_enqueue": [vp, i64, i64],
        "tsdf_admission_cancel": [vp, i64],
        "tsdf_admission_admit": [vp, vp, ctypes.c_int32, P(ctypes.c_int32)],
        "tsdf_admission_release": [vp, i64],
        "tsdf_admission_stats": [vp, P(i64), P(ctypes.c_int32), P(ctypes.c_int32)],
        "tsdf_scene_device_bytes": [P(SceneDesc), ctypes.c_int32, ctypes.c_int32, P(i64)],
        "tsdf_server_create": [P(ServerConfig), vp, P(vp)],
        "tsdf_server_destroy": [vp],
        "tsdf_server_open": [vp, P(SceneDesc), ctypes.c_int32, ctypes.c_int32, P(i64)],
        "tsdf_server_submit": [vp, i64, vp, i64, P(Intrinsics), vp, P(i64)],
        "tsdf_server_close": [vp, i64],
        "tsdf_server_step": [vp, P(StepInfo)],
        "tsdf_server_poll": [vp, ctypes.c_int32, vp, ctypes.c_int32, P(ctypes.c_int32)],
        "tsdf_server_session_info": [vp, i64, P(SessionInfo)],
        "tsdf_server_scene": [vp, i64, P(vp)],
        "tsdf_server_release": [vp, i64],
        "tsdf_server_trim": [vp],
        "tsdf_integrate_frames": [vp, vp, ctypes.c_int32],
        "tsdf_batch_join": [vp],
        "tsdf_batch_destroy": [vp],
        "tsdf_batch_prepare": [vp, vp, ctypes.c_int32],
        "tsdf_batch_launch": [vp],
        "tsdf_batch_integrate": [vp, vp, ctypes.c_int32],
        "tsdf_batch_set_config": [vp, P(BatchConfig)],
        "tsdf_batch_get_config": [vp, P(BatchConfig)],
        "tsdf_batch_autotune": [vp, ctypes.c_int32, P(BatchConfig), P(ctypes.c_float)],
        "tsdf_batch_kernel_launches": [vp, P(i64)],
        "tsdf_raycast": [vp, P(Intrinsics), vp, ctypes.c_float, vp, vp],
        "tsdf_get_raycast_stats": [vp, P(RaycastStats)],
        "tsdf_scene_enable_colour": [vp],
        "tsdf_integrate_rgb": [vp, vp, i64, i32, vp, P(Intrinsics), vp],
        "tsdf_read_colour": [vp, vp, i64, P(i64)],
        "tsdf_icp_create": [vp, P(vp)],
        "tsdf_icp_destroy": [vp],
        "tsdf_icp_normals": [vp, vp, vp, ctypes.c_int32, ctypes.c_int32],
        "tsdf_icp_reduce": [vp, vp, i64, P(Intrinsics), vp, vp, vp, vp, ctypes.c_float, vp],
        "tsdf_icp_kernel_launches": [vp, P(i64)],
        "tsdf_icp_solve": [vp, vp, vp],
        "tsdf_icp_track": [vp, vp, i64, P(Intrinsics), vp, vp, vp, vp, ctypes.c_float,
                           ctypes.c_int32, vp],
        "tsdf_icp_status": [vp, P(ctypes.c_int32)],
        "tsdf_icp_downsample": [vp, vp, i64, ctypes.c_int32, ctypes.c_int32, vp],
        "tsdf_engine_create": [P(EngineConfig), vp, vp, P(vp)],
        "tsdf_engine_destroy": [vp],
        "tsdf_engine_process": [vp, vp, i64, vp, vp],
        "tsdf_engine_scene": [vp, P(vp)],
        "tsdf_engine_tracker_status": [vp, P(ctypes.c_int32)],
        "tsdf_engine_reset": [vp, vp],
        "tsdf_engine_kernel_launches": [vp, P(i64)],
        "tsdf_swap_merge_voxels": [ctypes.c_int32, ctypes.c_int32, i64, vp, vp, vp, vp, vp, vp],
        "tsdf_scene_enable_swapping": [vp, ctypes.c_int32],
        "tsdf_swap_out": [vp, P(Intrinsics), vp, ctypes.c_double, ctypes.c_double],
        "tsdf_swap_in": [vp, P(Intrinsics), vp, ctypes.c_double, ctypes.c_double],
        "tsdf_get_swap_stats": [vp, P(SwapStats)],
        "tsdf_read_host_blocks": [vp, vp, vp, vp, vp, i64, P(i64)],
        "tsdf_swap_visibility": [ctypes.c_float, P(Intrinsics), vp, ctypes.c_double,
                                 ctypes.c_double, vp, i64, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.tsdf_status_string.argtypes = [ctypes.c_int]
    lib.tsdf_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def swap_visibility(voxel_size: float, intrinsics: Intrinsics, pose, keys,
                    margin_px: float = 0.0, max_depth: float = 0.0) -> np.ndarray:
    """The swapping visibility rule for block keys (n, 3) on the host (the
    swap kernels' code, compiled for the CPU): (n,) bool."""
    lib = load_library()
    k = np.ascontiguousarray(keys, dtype=np.int16).reshape(-1, 3)
    out = np.zeros(len(k), np.uint8)
    pose_arr = _pose_array(pose)
    _check(lib.tsdf_swap_visibility(float(voxel_size), ctypes.byref(intrinsics),
                                    pose_arr.ctypes.data_as(ctypes.c_void_p), float(margin_px),
                                    float(max_depth), k.ctypes.data_as(ctypes.c_void_p), len(k),
                                    out.ctypes.data_as(ctypes.c_void_p)), "tsdf_swap_visibility")
    return out.astype(bool)


def swap_merge_voxels(storage: int, max_weight: int, host_sdf, host_w, sdf, w,
                      host_rgbw=None, rgbw=None):
    """The secondary integration of swapping on the host (the swap-in
    kernel's per-voxel code, compiled for the CPU). Returns the merged
    (sdf, w, rgbw or None); the inputs are not modified."""
    lib = load_library()
    dt = SDF_DTYPE.get(storage, np.uint16)  # an unknown storage is the library's to refuse
    hs = np.ascontiguousarray(host_sdf, dtype=dt).ravel()
    hw = np.ascontiguousarray(host_w, dtype=np.uint8).ravel()
    ds = np.array(sdf, dtype=dt).ravel()
    dw = np.array(w, dtype=np.uint8).ravel()
    if not (len(hs) == len(hw) == len(ds) == len(dw)):
        raise ValueError("voxel arrays of different lengths")
    vp = ctypes.c_void_p
    hc = dc = None
    if host_rgbw is not None:
        hc = np.ascontiguousarray(host_rgbw, dtype=np.uint32).ravel()
        dc = np.array(rgbw, dtype=np.uint32).ravel()
    _check(lib.tsdf_swap_merge_voxels(int(storage), int(max_weight), len(hs),
                                      hs.ctypes.data_as(vp), hw.ctypes.data_as(vp),
                                      hc.ctypes.data_as(vp) if hc is not None else None,
                                      ds.ctypes.data_as(vp), dw.ctypes.data_as(vp),
                                      dc.ctypes.data_as(vp) if dc is not None else None),
           "tsdf_swap_merge_voxels")
    return ds, dw, dc


def status_string(status: int) -> str:
    return load_library().tsdf_status_string(int(status)).decode()


def _check(rc: int, where: str):
    if rc != TSDF_OK:
        raise TsdfError(rc, where)


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def make_intrinsics(fx, fy, cx, cy, width, height) -> Intrinsics:
    return Intrinsics(float(fx), float(fy), float(cx), float(cy), int(width), int(height))


def _pose_array(pose) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(4, 4))
    return p


@dataclass
class Blocks:
    keys: np.ndarray   # (n, 3) int16, sorted by (x, y, z)
    sdf: np.ndarray    # (n, 512) float32 / int16 / float16
    w: np.ndarray      # (n, 512) uint8

    def sdf_values(self) -> np.ndarray:
        """Stored sdf as real numbers (int16: q / 32767)."""
        if self.sdf.dtype == np.int16:
            return self.sdf.astype(np.float64) / 32767.0
        return self.sdf.astype(np.float64)


def scene_device_bytes(width: int = 0, height: int = 0, **desc) -> int:
    """Device bytes of a scene with these parameters plus the depth buffer of
    a width x height image (tsdf_scene_device_bytes; host only)."""
    lib = load_library()
    d = SceneDesc(**{**dict(max_weight=100, hash_buckets_log2=20, entries_per_bucket=2,
                            excess_entries=1 << 17, pool_blocks=1 << 18, storage=STORAGE_F32),
                     **desc})
    n = ctypes.c_int64()
    _check(lib.tsdf_scene_device_bytes(ctypes.byref(d), int(width), int(height), ctypes.byref(n)),
           "tsdf_scene_device_bytes")
    return int(n.value)


class Admission:
    """FIFO admission by byte budget (tsdf_admission_*; host only)."""

    def __init__(self, budget_bytes: int, max_active: int):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_admission_create(int(budget_bytes), int(max_active),
                                               ctypes.byref(h)), "tsdf_admission_create")
        self._h = h

    def __del__(self):
        try:
            if self._h.value:
                self._lib.tsdf_admission_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass

    def enqueue(self, sid: int, nbytes: int) -> None:
        _check(self._lib.tsdf_admission_enqueue(self._h, int(sid), int(nbytes)),
               "tsdf_admission_enqueue")

    def cancel(self, sid: int) -> None:
        _check(self._lib.tsdf_admission_cancel(self._h, int(sid)), "tsdf_admission_cancel")

    def admit(self, capacity: int = 1024) -> list:
        ids = (ctypes.c_int64 * max(capacity, 1))()
        n = ctypes.c_int32()
        _check(self._lib.tsdf_admission_admit(self._h, ctypes.cast(ids, ctypes.c_void_p),
                                              int(capacity), ctypes.byref(n)),
               "tsdf_admission_admit")
        return [int(ids[i]) for i in range(n.value)]

    def release(self, sid: int) -> None:
        _check(self._lib.tsdf_admission_release(self._h, int(sid)), "tsdf_admission_release")

    def stats(self) -> dict:
        b = ctypes.c_int64()
        a = ctypes.c_int32()
        q = ctypes.c_int32()
        _check(self._lib.tsdf_admission_stats(self._h, ctypes.byref(b), ctypes.byref(a),
                                              ctypes.byref(q)), "tsdf_admission_stats")
        return {"active_bytes": int(b.value), "active": int(a.value), "queued": int(q.value)}


class Scene:
    """One TSDF scene on the current CUDA device (tsdf_scene_* calls)."""

    def __init__(self, voxel_size: float, mu: float, max_weight: int = 100,
                 hash_buckets_log2: int = 20, entries_per_bucket: int = 2,
                 excess_entries: int = 1 << 17, pool_blocks: int = 1 << 18,
                 storage: int = STORAGE_F32, stream=None):
        self._lib = load_library()
        self.desc = SceneDesc(voxel_size, mu, max_weight, hash_buckets_log2,
                              entries_per_bucket, excess_entries, pool_blocks,
                              storage)
        self.storage = storage
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_scene_create(ctypes.byref(self.desc),
                                           ctypes.c_void_p(_stream_handle(stream)),
                                           ctypes.byref(h)), "tsdf_scene_create")
        self._h = h
        self._keep = []   # host buffers that must outlive enqueued copies

    @classmethod
    def from_workload(cls, w, stream=None, **over):
        d = dict(w.scene_desc())
        d.update(over)
        return cls(stream=stream, **d)

    @classmethod
    def borrowed(cls, handle: int, storage: int):
        """A view of a scene owned elsewhere (a server session's): every
        scene call but destruction."""
        self = cls.__new__(cls)
        self._lib = load_library()
        self._h = ctypes.c_void_p(handle)
        self.storage = storage
        self._keep = []
        self._borrowed = True
        return self

    @property
    def handle(self) -> int:
        return self._h.value

    @property
    def device(self) -> int:
        """The CUDA device index the scene lives on."""
        d = ctypes.c_int32()
        _check(self._lib.tsdf_scene_device(self._h, ctypes.byref(d)), "tsdf_scene_device")
        return int(d.value)

    def close(self):
        if getattr(self, "_borrowed", False):
            self._h = ctypes.c_void_p()
            return
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tsdf_scene_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check(self._lib.tsdf_scene_reset(self._h), "tsdf_scene_reset")

    def set_stream(self, stream):
        _check(self._lib.tsdf_scene_set_stream(self._h, ctypes.c_void_p(_stream_handle(stream))),
               "tsdf_scene_set_stream")

    def integrate(self, depth, intrinsics: Intrinsics, pose) -> None:
        """Fuse one frame. ``depth``: a CUDA torch tensor (H, W) float32
        (device path, row pitch from its stride), or a CPU tensor / numpy
        array (host path: copied to the device inside the call)."""
        pitch, ptr, on_host = _depth_pointer(depth, self._keep)
        pose_arr = _pose_array(pose)
        _check(self._lib.tsdf_integrate(self._h, ctypes.c_void_p(ptr), pitch, on_host,
                                        ctypes.byref(intrinsics),
                                        pose_arr.ctypes.data_as(ctypes.c_void_p)),
               "tsdf_integrate")
        if len(self._keep) > 64:
            self._keep = self._keep[-64:]

    def integrate_frames(self, depth, intrinsics, poses) -> None:
        """Fuse a sequence of frames with the allocation of frame t + 1
        overlapping the integration of frame t (tsdf_integrate_frames).
        ``depth``: a tensor (N, H, W) float32 (or a list of (H, W) tensors),
        on the scene's device, or in (pinned) host memory, which the library
        copies to the device frame by frame; ``intrinsics``: one Intrinsics
        or a list of N; ``poses``: (N, 4, 4) world->camera."""
        n = len(depth)
        intrs = intrinsics if isinstance(intrinsics, (list, tuple)) else [intrinsics] * n
        arr = (Frame * n)()
        for i in range(n):
            d = depth[i]
            if not hasattr(d, "data_ptr") or d.dim() != 2 or d.stride(1) != 1 or \
                    str(d.dtype) != "torch.float32":
                raise ValueError("depth frames must be float32 tensors with unit column stride")
            arr[i].scene = self.handle
            arr[i].depth = d.data_ptr()
            arr[i].pitch_elems = d.stride(0)
            arr[i].depth_on_host = 0 if d.is_cuda else 1
            arr[i].intr = intrs[i]
            p = _pose_array(poses[i]).reshape(-1)
            for j in range(16):
                arr[i].world_to_cam[j] = float(p[j])
        _check(self._lib.tsdf_integrate_frames(self._h, ctypes.cast(arr, ctypes.c_void_p), n),
               "tsdf_integrate_frames")

    def enable_colour(self) -> None:
        """Keep a colour per voxel from now on (tsdf_scene_enable_colour)."""
        _check(self._lib.tsdf_scene_enable_colour(self._h), "tsdf_scene_enable_colour")

    def integrate_rgb(self, depth, colour, intrinsics: Intrinsics, pose) -> None:
        """Fuse one frame with a registered colour image: ``colour`` is a CUDA
        uint8 tensor (H, W, 4) (r, g, b, unused), contiguous; ``depth`` as in
        integrate()."""
        import torch
        if (not getattr(colour, "is_cuda", False) or colour.dtype != torch.uint8 or
                tuple(colour.shape) != (intrinsics.height, intrinsics.width, 4) or
                not colour.is_contiguous()):
            raise ValueError("colour must be a contiguous CUDA uint8 tensor (H, W, 4)")
        pitch, ptr, on_host = _depth_pointer(depth, self._keep)
        pose_arr = _pose_array(pose)
        _check(self._lib.tsdf_integrate_rgb(self._h, ctypes.c_void_p(ptr), pitch, on_host,
                                            ctypes.c_void_p(colour.data_ptr()),
                                            ctypes.byref(intrinsics),
                                            pose_arr.ctypes.data_as(ctypes.c_void_p)),
               "tsdf_integrate_rgb")

    def read_colour(self) -> np.ndarray:
        """(n, 512, 4) uint8 (r, g, b, colour weight) in read_blocks() order."""
        n = ctypes.c_int64()
        rc = self._lib.tsdf_read_colour(self._h, None, 0, ctypes.byref(n))
        if rc not in (TSDF_OK, TSDF_ERR_CAPACITY):
            _check(rc, "tsdf_read_colour")
        out = np.zeros((n.value, 512, 4), np.uint8)
        _check(self._lib.tsdf_read_colour(self._h, out.ctypes.data_as(ctypes.c_void_p),
                                          n.value, ctypes.byref(n)), "tsdf_read_colour")
        return out

    def raycast(self, intrinsics: Intrinsics, pose, z_near: float = 0.2, points=None,
                range_out=None):
        """Render the surface from a camera (tsdf_raycast, Section 4.4).
        Returns ``points``, a CUDA float32 tensor (H, W, 4): world metres and
        1 on a surface, zeros without one (allocated here unless given).
        ``range_out``: optional CUDA float32 tensor (H, W, 2) that receives
        each pixel's search range."""
        import torch
        H, W = intrinsics.height, intrinsics.width
        if points is None:
            points = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        for t, c in ((points, 4), (range_out, 2)):
            if t is None:
                continue
            if (not t.is_cuda or t.dtype != torch.float32 or tuple(t.shape) != (H, W, c)
                    or not t.is_contiguous()):
                raise ValueError(f"expected a contiguous CUDA float32 tensor ({H}, {W}, {c})")
        pose_arr = _pose_array(pose)
        _check(self._lib.tsdf_raycast(self._h, ctypes.byref(intrinsics),
                                      pose_arr.ctypes.data_as(ctypes.c_void_p), float(z_near),
                                      ctypes.c_void_p(points.data_ptr()),
                                      ctypes.c_void_p(range_out.data_ptr()
                                                      if range_out is not None else 0)),
               "tsdf_raycast")
        return points

    def raycast_stats(self) -> dict:
        """Counters of the most recent raycast (synchronises)."""
        st = RaycastStats()
        _check(self._lib.tsdf_get_raycast_stats(self._h, ctypes.byref(st)),
               "tsdf_get_raycast_stats")
        return {k: int(getattr(st, k)) for k, _ in RaycastStats._fields_}

    def enable_swapping(self, transfer_blocks: int) -> None:
        """Keep a host copy of the map for swapping (Section 5); one swap call
        moves at most ``transfer_blocks`` blocks."""
        _check(self._lib.tsdf_scene_enable_swapping(self._h, int(transfer_blocks)),
               "tsdf_scene_enable_swapping")

    def swap_out(self, intrinsics: Intrinsics, pose, margin_px: float = 0.0,
                 max_depth: float = 0.0) -> None:
        """Move device blocks that the view does not see to the host copy
        (enqueued; tsdf_swap_out)."""
        pose_arr = _pose_array(pose)
        _check(self._lib.tsdf_swap_out(self._h, ctypes.byref(intrinsics),
                                       pose_arr.ctypes.data_as(ctypes.c_void_p),
                                       float(margin_px), float(max_depth)), "tsdf_swap_out")

    def swap_in(self, intrinsics: Intrinsics, pose, margin_px: float = 0.0,
                max_depth: float = 0.0) -> None:
        """Bring host blocks back: merged into the fresh blocks the allocation
        gave them, or (if the pool has room) copied when the view sees them
        (enqueued; tsdf_swap_in)."""
        pose_arr = _pose_array(pose)
        _check(self._lib.tsdf_swap_in(self._h, ctypes.byref(intrinsics),
                                      pose_arr.ctypes.data_as(ctypes.c_void_p),
                                      float(margin_px), float(max_depth)), "tsdf_swap_in")

    def swap_stats(self) -> dict:
        st = SwapStats()
        _check(self._lib.tsdf_get_swap_stats(self._h, ctypes.byref(st)), "tsdf_get_swap_stats")
        return {k: int(getattr(st, k)) for k, _ in SwapStats._fields_}

    def read_host_blocks(self, colour: bool = False):
        """The host copies, sorted by key: (Blocks, rgbw or None)."""
        n = ctypes.c_int64()
        rc = self._lib.tsdf_read_host_blocks(self._h, None, None, None, None, 0, ctypes.byref(n))
        if rc not in (TSDF_OK, TSDF_ERR_CAPACITY):
            _check(rc, "tsdf_read_host_blocks")
        cap = int(n.value)
        keys = np.zeros((cap, 3), np.int16)
        sdf = np.zeros((cap, 512), SDF_DTYPE[self.storage])
        w = np.zeros((cap, 512), np.uint8)
        rgbw = np.zeros((cap, 512, 4), np.uint8) if colour else None
        vp = ctypes.c_void_p
        _check(self._lib.tsdf_read_host_blocks(
            self._h, keys.ctypes.data_as(vp), sdf.ctypes.data_as(vp), w.ctypes.data_as(vp),
            rgbw.ctypes.data_as(vp) if colour else None, cap, ctypes.byref(n)),
            "tsdf_read_host_blocks")
        m = int(n.value)
        return Blocks(keys[:m], sdf[:m], w[:m]), (rgbw[:m] if colour else None)

    def sync(self):
        self._keep.clear()
        _check(self._lib.tsdf_sync(self._h), "tsdf_sync")

    def stats(self) -> dict:
        st = Stats()
        rc = self._lib.tsdf_get_stats(self._h, ctypes.byref(st))
        self._keep.clear()
        _check(rc, "tsdf_get_stats")
        return st.as_dict()

    def stats_and_status(self):
        st = Stats()
        rc = self._lib.tsdf_get_stats(self._h, ctypes.byref(st))
        self._keep.clear()
        return st.as_dict(), rc

    def num_blocks(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.tsdf_num_blocks(self._h, ctypes.byref(n)), "tsdf_num_blocks")
        return int(n.value)

    def read_blocks(self, check: bool = True) -> Blocks:
        n = ctypes.c_int64()
        rc = self._lib.tsdf_read_blocks(self._h, None, None, None, 0, ctypes.byref(n))
        if rc not in (TSDF_OK, TSDF_ERR_CAPACITY):
            if check:
                _check(rc, "tsdf_read_blocks")
        cap = int(n.value)
        keys = np.zeros((cap, 3), np.int16)
        sdf = np.zeros((cap, 512), SDF_DTYPE[self.storage])
        w = np.zeros((cap, 512), np.uint8)
        rc = self._lib.tsdf_read_blocks(self._h, keys.ctypes.data_as(ctypes.c_void_p),
                                        sdf.ctypes.data_as(ctypes.c_void_p),
                                        w.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n))
        if check:
            _check(rc, "tsdf_read_blocks")
        m = int(n.value)
        return Blocks(keys[:m], sdf[:m], w[:m])

    def load_blocks(self, blocks: Blocks) -> None:
        keys = np.ascontiguousarray(blocks.keys, np.int16)
        sdf = np.ascontiguousarray(blocks.sdf, SDF_DTYPE[self.storage])
        w = np.ascontiguousarray(blocks.w, np.uint8)
        _check(self._lib.tsdf_load_blocks(self._h, keys.ctypes.data_as(ctypes.c_void_p),
                                          sdf.ctypes.data_as(ctypes.c_void_p),
                                          w.ctypes.data_as(ctypes.c_void_p), len(keys)),
               "tsdf_load_blocks")

    def timing_begin(self, max_frames: int, integration_only: bool = False) -> None:
        _check(self._lib.tsdf_timing_begin(self._h, int(max_frames), int(bool(integration_only))),
               "tsdf_timing_begin")

    def timing_read(self) -> np.ndarray:
        """Per-frame stage boundary times in ms relative to the first one
        recorded, shape (frames, len(STAGES) + 1); NaN where not recorded."""
        n = ctypes.c_int64()
        self._lib.tsdf_timing_read(self._h, None, 0, ctypes.byref(n))
        out = np.zeros((max(int(n.value), 1), len(STAGES) + 1), np.float32)
        _check(self._lib.tsdf_timing_read(self._h, out.ctypes.data_as(ctypes.c_void_p),
                                          out.shape[0], ctypes.byref(n)), "tsdf_timing_read")
        return out[:int(n.value)]

    def timing_end(self) -> None:
        _check(self._lib.tsdf_timing_end(self._h), "tsdf_timing_end")

    def read_blocks_device_noalloc(self, keys_dev, sdf_dev, w_dev) -> int:
        """Canonical readback into caller-owned CUDA tensors without any
        allocation by the library (tsdf_read_blocks_device_noalloc).
        keys_dev int16 (cap, 3), sdf_dev (cap, 512) of the storage dtype,
        w_dev uint8 (cap, 512), all contiguous on the scene's device (sdf_dev
        and w_dev may be None); returns the number of blocks written."""
        import torch
        sdf_dtype = {STORAGE_F32: torch.float32, STORAGE_I16: torch.int16,
                     STORAGE_F16: torch.float16}[self.storage]
        cap = int(keys_dev.shape[0]) if keys_dev is not None and keys_dev.dim() == 2 else -1
        dev = torch.device("cuda", self.device)
        for name, t, dtype, cols in (("keys_dev", keys_dev, torch.int16, 3),
                                     ("sdf_dev", sdf_dev, sdf_dtype, 512),
                                     ("w_dev", w_dev, torch.uint8, 512)):
            if t is None and name != "keys_dev":
                continue
            if (t is None or t.device != dev or not t.is_contiguous() or t.dtype != dtype or
                    t.dim() != 2 or tuple(t.shape) != (cap, cols)):
                raise TsdfError(TSDF_ERR_INVALID_ARG,
                                f"read_blocks_device_noalloc: {name} must be a contiguous "
                                f"{dtype} tensor of shape ({cap}, {cols}) on {dev}")
        n = ctypes.c_int64()
        rc = self._lib.tsdf_read_blocks_device_noalloc(
            self._h, ctypes.c_void_p(keys_dev.data_ptr()),
            ctypes.c_void_p(sdf_dev.data_ptr() if sdf_dev is not None else 0),
            ctypes.c_void_p(w_dev.data_ptr() if w_dev is not None else 0), cap, ctypes.byref(n))
        if rc == TSDF_ERR_CAPACITY:
            raise TsdfError(rc, f"tsdf_read_blocks_device_noalloc: {int(n.value)} blocks allocated, "
                                f"buffers hold {cap}, fixed scratch holds {READ_NOALLOC_MAX_BLOCKS}")
        _check(rc, "tsdf_read_blocks_device_noalloc")
        return int(n.value)

    def lookup(self, keys) -> np.ndarray:
        k = np.ascontiguousarray(np.asarray(keys).reshape(-1, 3), np.int16)
        out = np.zeros(len(k), np.int32)
        _check(self._lib.tsdf_lookup_blocks(self._h, k.ctypes.data_as(ctypes.c_void_p), len(k),
                                            out.ctypes.data_as(ctypes.c_void_p)),
               "tsdf_lookup_blocks")
        return out


class Engine:
    """The processing pipeline of one camera (tsdf_engine_*, Section 2.1):
    track every frame against the model rendered from the last pose, fuse at
    the tracked pose; with ``swap_blocks`` > 0 the scene swaps (Section 5)
    around each fusion, at most that many blocks a call."""

    def __init__(self, scene_desc: dict, intrinsics: Intrinsics, initial_pose, levels: int = 3,
                 iterations=(4, 4, 6), max_dist: float = 0.1, z_near: float = 0.2,
                 colour: bool = False, swap_blocks: int = 0, swap_margin_px: float = 16.0,
                 stream=None):
        self._lib = load_library()
        d = dict(max_weight=100, hash_buckets_log2=20, entries_per_bucket=2,
                 excess_entries=1 << 17, pool_blocks=1 << 18, storage=STORAGE_F32)
        d.update(scene_desc)
        it = (ctypes.c_int32 * 4)(*(list(iterations) + [0] * (4 - len(iterations))))
        self.cfg = EngineConfig(SceneDesc(d["voxel_size"], d["mu"], d["max_weight"],
                                          d["hash_buckets_log2"], d["entries_per_bucket"],
                                          d["excess_entries"], d["pool_blocks"], d["storage"]),
                                intrinsics, int(levels), it, float(max_dist), float(z_near),
                                int(bool(colour)), int(swap_blocks), float(swap_margin_px))
        pose = _pose_array(initial_pose)
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_engine_create(ctypes.byref(self.cfg),
                                            pose.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.c_void_p(_stream_handle(stream)),
                                            ctypes.byref(h)), "tsdf_engine_create")
        self._h = h
        self.storage = d["storage"]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tsdf_engine_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def process(self, depth, colour=None) -> np.ndarray:
        """Track and fuse one frame (CUDA depth (H, W) float32, optional CUDA
        colour (H, W, 4) uint8); returns the tracked world->camera pose."""
        if not getattr(depth, "is_cuda", False) or depth.stride(1) != 1:
            raise ValueError("depth must be a CUDA tensor with unit column stride")
        out = np.zeros(16, np.float64)
        _check(self._lib.tsdf_engine_process(
            self._h, ctypes.c_void_p(depth.data_ptr()), depth.stride(0),
            ctypes.c_void_p(colour.data_ptr() if colour is not None else 0),
            out.ctypes.data_as(ctypes.c_void_p)), "tsdf_engine_process")
        return out.reshape(4, 4)

    def reset(self, initial_pose) -> None:
        """Empty the model and start again from initial_pose."""
        pose = _pose_array(initial_pose)
        _check(self._lib.tsdf_engine_reset(self._h, pose.ctypes.data_as(ctypes.c_void_p)),
               "tsdf_engine_reset")

    def scene(self) -> "Scene":
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_engine_scene(self._h, ctypes.byref(h)), "tsdf_engine_scene")
        return Scene.borrowed(h.value, self.storage)

    def kernel_launches(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.tsdf_engine_kernel_launches(self._h, ctypes.byref(n)),
               "tsdf_engine_kernel_launches")
        return int(n.value)

    def tracker_status(self) -> int:
        v = ctypes.c_int32()
        _check(self._lib.tsdf_engine_tracker_status(self._h, ctypes.byref(v)),
               "tsdf_engine_tracker_status")
        return v.value


class Icp:
    """The depth tracker's linearised point-to-plane system (tsdf_icp_*,
    Section 4.1) on one CUDA stream."""

    TERMS = 29

    def __init__(self, stream=None):
        import torch
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_icp_create(ctypes.c_void_p(_stream_handle(stream)),
                                         ctypes.byref(h)), "tsdf_icp_create")
        self._h = h
        self.sums = torch.zeros(self.TERMS, dtype=torch.float64, device="cuda")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tsdf_icp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def normals(self, points, out=None):
        """Normal map (H, W, 4) of a point map (H, W, 4), CUDA float32."""
        import torch
        H, W = points.shape[:2]
        if out is None:
            out = torch.empty_like(points)
        for t in (points, out):
            if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or \
                    tuple(t.shape) != (H, W, 4):
                raise ValueError("expected contiguous CUDA float32 (H, W, 4) tensors")
        _check(self._lib.tsdf_icp_normals(self._h, ctypes.c_void_p(points.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), W, H),
               "tsdf_icp_normals")
        return out

    def reduce(self, depth, intrinsics: Intrinsics, cur_pose, ref_pose, points, normals,
               max_dist: float = 0.1, sums=None):
        """Enqueue one reduction; returns the CUDA float64 tensor (29) that
        receives the terms (H upper triangle 21, g 6, E, count)."""
        if not getattr(depth, "is_cuda", False) or depth.stride(1) != 1:
            raise ValueError("depth must be a CUDA tensor with unit column stride")
        out = self.sums if sums is None else sums
        cur = _pose_array(cur_pose)
        ref = _pose_array(ref_pose)
        _check(self._lib.tsdf_icp_reduce(self._h, ctypes.c_void_p(depth.data_ptr()),
                                         depth.stride(0), ctypes.byref(intrinsics),
                                         cur.ctypes.data_as(ctypes.c_void_p),
                                         ref.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.c_void_p(points.data_ptr()),
                                         ctypes.c_void_p(normals.data_ptr()), float(max_dist),
                                         ctypes.c_void_p(out.data_ptr())), "tsdf_icp_reduce")
        return out

    def solve(self, sums, pose):
        """One Gauss-Newton step on the device: pose (CUDA float64 (4, 4),
        world->camera) updated in place from sums (CUDA float64 (29))."""
        _check(self._lib.tsdf_icp_solve(self._h, ctypes.c_void_p(sums.data_ptr()),
                                        ctypes.c_void_p(pose.data_ptr())), "tsdf_icp_solve")

    def track(self, depth, intrinsics: Intrinsics, pose, ref_pose, points, normals,
              max_dist: float = 0.1, iterations: int = 10, sums=None):
        """`iterations` Gauss-Newton iterations on the device; pose is a CUDA
        float64 (4, 4) tensor updated in place."""
        import torch
        if not pose.is_cuda or pose.dtype != torch.float64 or not pose.is_contiguous():
            raise ValueError("pose must be a contiguous CUDA float64 (4, 4) tensor")
        out = self.sums if sums is None else sums
        ref = _pose_array(ref_pose)
        _check(self._lib.tsdf_icp_track(self._h, ctypes.c_void_p(depth.data_ptr()),
                                        depth.stride(0), ctypes.byref(intrinsics),
                                        ctypes.c_void_p(pose.data_ptr()),
                                        ref.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.c_void_p(points.data_ptr()),
                                        ctypes.c_void_p(normals.data_ptr()), float(max_dist),
                                        int(iterations), ctypes.c_void_p(out.data_ptr())),
               "tsdf_icp_track")
        return pose

    def downsample(self, depth, out=None):
        """One level of the depth hierarchy: (H/2, W/2) CUDA float32."""
        import torch
        H, W = depth.shape
        if out is None:
            out = torch.empty((H // 2, W // 2), dtype=torch.float32, device=depth.device)
        if not getattr(depth, "is_cuda", False) or depth.stride(1) != 1 or \
                tuple(out.shape) != (H // 2, W // 2) or not out.is_contiguous():
            raise ValueError("depth must be a CUDA (H, W) tensor with unit column stride")
        _check(self._lib.tsdf_icp_downsample(self._h, ctypes.c_void_p(depth.data_ptr()),
                                             depth.stride(0), W, H,
                                             ctypes.c_void_p(out.data_ptr())),
               "tsdf_icp_downsample")
        return out

    @staticmethod
    def level_intrinsics(intr, level: int):
        """Intrinsics of hierarchy level `level` (0 = full resolution), from
        tsdf_icp_level_intrinsics."""
        out = Intrinsics()
        _check(load_library().tsdf_icp_level_intrinsics(ctypes.byref(intr), int(level),
                                                        ctypes.byref(out)),
               "tsdf_icp_level_intrinsics")
        return out

    def status(self) -> int:
        v = ctypes.c_int32()
        _check(self._lib.tsdf_icp_status(self._h, ctypes.byref(v)), "tsdf_icp_status")
        return v.value

    def kernel_launches(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.tsdf_icp_kernel_launches(self._h, ctypes.byref(n)),
               "tsdf_icp_kernel_launches")
        return n.value

    @staticmethod
    def system(sums):
        """(H 6x6, g 6) as numpy float64 from the 29 terms."""
        s = np.asarray(sums.cpu() if hasattr(sums, "cpu") else sums, np.float64)
        Hm = np.zeros((6, 6))
        t = 0
        for a in range(6):
            for b in range(a, 6):
                Hm[a, b] = Hm[b, a] = s[t]
                t += 1
        return Hm, s[21:27].copy()


class Batch:
    """Batched fusion step over many scenes (tsdf_batch_* calls). Depth is a
    CUDA tensor or a (pinned) host tensor, which the launch copies to the
    device. ``tables`` slot tables are used round-robin, one per prepare +
    launch pair."""

    def __init__(self, capacity: int, tables: int = 1, stream=None):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_batch_create(int(capacity), int(tables),
                                           ctypes.c_void_p(_stream_handle(stream)),
                                           ctypes.byref(h)), "tsdf_batch_create")
        self._h = h
        self.capacity = capacity
        self.tables = tables

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tsdf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _frame_array(self, items):
        """items: iterable of (scene, depth tensor (CUDA or host), Intrinsics,
        pose)."""
        items = list(items)
        arr = (Frame * len(items))()
        for i, (scene, depth, intr, pose) in enumerate(items):
            if not hasattr(depth, "data_ptr") or depth.dim() != 2 or \
                    str(depth.dtype) != "torch.float32":
                raise ValueError("batched depth must be a 2-D float32 tensor")
            if depth.stride(1) != 1:
                raise ValueError("depth must have unit column stride")
            arr[i].scene = scene.handle
            arr[i].depth = depth.data_ptr()
            arr[i].pitch_elems = depth.stride(0)
            arr[i].depth_on_host = 0 if depth.is_cuda else 1
            arr[i].intr = intr
            p = _pose_array(pose).reshape(-1)
            for j in range(16):
                arr[i].world_to_cam[j] = float(p[j])
        return arr

    def prepare(self, items) -> None:
        arr = self._frame_array(items)
        _check(self._lib.tsdf_batch_prepare(self._h, ctypes.cast(arr, ctypes.c_void_p), len(arr)),
               "tsdf_batch_prepare")

    def launch(self) -> None:
        _check(self._lib.tsdf_batch_launch(self._h), "tsdf_batch_launch")

    def integrate(self, items) -> None:
        self.prepare(items)
        self.launch()

    def config(self) -> dict:
        c = BatchConfig()
        _check(self._lib.tsdf_batch_get_config(self._h, ctypes.byref(c)), "tsdf_batch_get_config")
        return c.as_dict()

    def set_config(self, integrate_ctas_per_sm: int = 1, pipelined: bool = False,
                   integrate_kernel="staged", integrate_threads: int = 512,
                   alloc_tile="16x16") -> None:
        """The batch's schedule (tsdf_batch_set_config); kernel and tile by
        name ("staged" / "general", "16x16" / "16x8" / "32x8") or number."""
        kern = {v: k for k, v in BatchConfig.KERNELS.items()}.get(integrate_kernel, integrate_kernel)
        tile = {v: k for k, v in BatchConfig.TILES.items()}.get(alloc_tile, alloc_tile)
        c = BatchConfig(int(integrate_ctas_per_sm), int(bool(pipelined)), int(kern),
                        int(integrate_threads), int(tile))
        _check(self._lib.tsdf_batch_set_config(self._h, ctypes.byref(c)), "tsdf_batch_set_config")

    def autotune(self, steps: int = 3):
        c = BatchConfig()
        ms = ctypes.c_float()
        _check(self._lib.tsdf_batch_autotune(self._h, int(steps), ctypes.byref(c), ctypes.byref(ms)),
               "tsdf_batch_autotune")
        return c.as_dict(), float(ms.value)

    def timing_begin(self, max_launches: int, integration_only: bool = False) -> None:
        _check(self._lib.tsdf_batch_timing_begin(self._h, int(max_launches), int(integration_only)),
               "tsdf_batch_timing_begin")

    def timing_read(self) -> np.ndarray:
        """Per-launch stage boundary times in ms, shape (launches, 4)."""
        n = ctypes.c_int64()
        self._lib.tsdf_batch_timing_read(self._h, None, 0, ctypes.byref(n))
        out = np.zeros((max(int(n.value), 1), len(STAGES) + 1), np.float32)
        _check(self._lib.tsdf_batch_timing_read(self._h, out.ctypes.data_as(ctypes.c_void_p),
                                                out.shape[0], ctypes.byref(n)),
               "tsdf_batch_timing_read")
        return out[:int(n.value)]

    def timing_end(self) -> None:
        _check(self._lib.tsdf_batch_timing_end(self._h), "tsdf_batch_timing_end")

    def join(self) -> None:
        _check(self._lib.tsdf_batch_join(self._h), "tsdf_batch_join")

    @property
    def cursor(self) -> int:
        c = ctypes.c_int32()
        _check(self._lib.tsdf_batch_cursor(self._h, ctypes.byref(c)), "tsdf_batch_cursor")
        return int(c.value)

    @cursor.setter
    def cursor(self, value: int) -> None:
        _check(self._lib.tsdf_batch_set_cursor(self._h, int(value)), "tsdf_batch_set_cursor")

    def kernel_launches(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.tsdf_batch_kernel_launches(self._h, ctypes.byref(n)),
               "tsdf_batch_kernel_launches")
        return int(n.value)


class Server:
    """Continuous-batching fusion server (tsdf_server_* calls)."""

    def __init__(self, pool_budget_bytes: int, max_active: int = 1024,
                 max_queued_frames: int = 4, max_inflight_steps: int = 2, stream=None):
        self._lib = load_library()
        self.cfg = ServerConfig(int(pool_budget_bytes), int(max_active), int(max_queued_frames),
                                int(max_inflight_steps), 0)
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_server_create(ctypes.byref(self.cfg),
                                            ctypes.c_void_p(_stream_handle(stream)),
                                            ctypes.byref(h)), "tsdf_server_create")
        self._h = h
        self._storage = {}
        self._depth_refs = {}   # ticket -> depth tensor kept alive until done
        self._done_buf = (FrameDone * 4096)()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tsdf_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open(self, width: int, height: int, **desc) -> int:
        d = SceneDesc(**{**dict(max_weight=100, hash_buckets_log2=20, entries_per_bucket=2,
                                excess_entries=1 << 17, pool_blocks=1 << 18,
                                storage=STORAGE_F32), **desc})
        sid = ctypes.c_int64()
        _check(self._lib.tsdf_server_open(self._h, ctypes.byref(d), int(width), int(height),
                                          ctypes.byref(sid)), "tsdf_server_open")
        self._storage[int(sid.value)] = d.storage
        return int(sid.value)

    def open_workload(self, w) -> int:
        return self.open(w.width, w.height, **w.scene_desc())

    def submit(self, session: int, depth, intrinsics: Intrinsics, pose) -> int:
        if not getattr(depth, "is_cuda", False) or depth.stride(1) != 1:
            raise ValueError("server depth must be a CUDA tensor with unit column stride")
        pose_arr = _pose_array(pose)
        t = ctypes.c_int64()
        _check(self._lib.tsdf_server_submit(self._h, int(session), ctypes.c_void_p(depth.data_ptr()),
                                            depth.stride(0), ctypes.byref(intrinsics),
                                            pose_arr.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(t)), "tsdf_server_submit")
        self._depth_refs[int(t.value)] = depth
        return int(t.value)

    def close_session(self, session: int) -> None:
        _check(self._lib.tsdf_server_close(self._h, int(session)), "tsdf_server_close")

    def step(self) -> dict:
        info = StepInfo()
        _check(self._lib.tsdf_server_step(self._h, ctypes.byref(info)), "tsdf_server_step")
        return info.as_dict()

    def poll(self, wait_all: bool = False) -> list:
        """[(ticket, session, submit_ms, done_ms)] of frames fused since the
        last poll."""
        out = []
        while True:
            n = ctypes.c_int32()
            _check(self._lib.tsdf_server_poll(self._h, int(wait_all),
                                              ctypes.cast(self._done_buf, ctypes.c_void_p),
                                              len(self._done_buf), ctypes.byref(n)),
                   "tsdf_server_poll")
            for i in range(n.value):
                d = self._done_buf[i]
                out.append((int(d.ticket), int(d.session), float(d.submit_ms), float(d.done_ms)))
                self._depth_refs.pop(int(d.ticket), None)
            if n.value < len(self._done_buf):
                return out
            wait_all = False

    def session_info(self, session: int) -> dict:
        info = SessionInfo()
        _check(self._lib.tsdf_server_session_info(self._h, int(session), ctypes.byref(info)),
               "tsdf_server_session_info")
        return info.as_dict()

    def scene(self, session: int) -> "Scene":
        h = ctypes.c_void_p()
        _check(self._lib.tsdf_server_scene(self._h, int(session), ctypes.byref(h)),
               "tsdf_server_scene")
        return Scene.borrowed(h.value, self._storage[int(session)])

    def release(self, session: int) -> None:
        _check(self._lib.tsdf_server_release(self._h, int(session)), "tsdf_server_release")
        self._storage.pop(int(session), None)

    def trim(self) -> None:
        _check(self._lib.tsdf_server_trim(self._h), "tsdf_server_trim")


def _depth_pointer(depth, keep: list):
    """(row pitch in elements, pointer, on_host) of a depth image."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(depth, torch.Tensor):
        if depth.dtype != torch.float32 or depth.dim() != 2 or depth.stride(1) != 1:
            raise ValueError("depth must be a 2-D float32 tensor with unit column stride")
        if depth.is_cuda:
            return depth.stride(0), depth.data_ptr(), 0
        keep.append(depth)
        return depth.stride(0), depth.data_ptr(), 1
    a = np.asarray(depth)
    if a.dtype != np.float32 or a.ndim != 2 or a.strides[1] != 4:
        a = np.ascontiguousarray(a, np.float32)
    keep.append(a)
    return a.strides[0] // 4, a.ctypes.data, 1
