"""FP64 CPU oracle for voxel-block TSDF depth fusion -- TEST INFRASTRUCTURE.

This package is the plain, slow definition the CUDA path is checked against
(InfiniTAM report, arXiv 1410.0925: Sections 3.1-3.3 for the voxel, block and
fixed-point definitions, Section 4.2 for the allocation band, Section 4.3 for
the per-voxel update). It is written in plain C (``tsdf_oracle.c``) and
loaded with ctypes; this module only marshals arguments.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA library.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  Oracle.integrate / read      pinned: closed-form plane, translating plane,
                               weight cap, invariants, dense == block form,
                               sampled-segment brute force
  DenseOracle                  pinned against Oracle (and the plane closed form)
  block_hit_frames             pinned against Oracle's allocation frames
  voxel_candidates             pinned: equals Oracle on unflagged voxels; on a
                               planted ambiguity contains both outcomes
  float_to_i16 / round_f16     pinned against numpy's int16 cast / float16
  Oracle.integrate_rgb         pinned: constant colour on the closed-form plane,
                               hand-derived averages with round-half-up ties and
                               the weight cap, per-pixel texture lookup
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("tsdf_oracle.c", "raycast_oracle.c", "icp_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

STORAGE_F32, STORAGE_I16, STORAGE_F16 = 0, 1, 2
BLOCK_MEMBERSHIP_AMBIGUOUS, BLOCK_HISTORY_AMBIGUOUS = 1, 2
BLOCK_SWAP_AMBIGUOUS, BLOCK_SWAPPED = 4, 8
HIT_GROWN, HIT_EXACT, HIT_SHRUNK = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C11, -O2).

    The environment variable TSDF_ORACLE_LIB names a prebuilt library to use
    instead (the mutation test points it at deliberately broken copies)."""
    override = os.environ.get("TSDF_ORACLE_LIB")
    if override:
        return override
    deps = _SRCS + [os.path.join(_HERE, "tsdf_oracle.h")]
    stale = (not os.path.exists(_LIB_PATH) or
             any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(d) for d in deps))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared",
                               "-Wall", "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_double), ("mu", ctypes.c_double),
                ("max_weight", ctypes.c_int), ("storage", ctypes.c_int),
                ("pool_blocks", ctypes.c_longlong),
                ("delta_px", ctypes.c_double), ("delta_eta", ctypes.c_double),
                ("delta_b", ctypes.c_double), ("delta_z", ctypes.c_double)]


class _RayParams(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_double), ("mu", ctypes.c_double),
                ("z_near", ctypes.c_double), ("delta_px", ctypes.c_double),
                ("delta_z", ctypes.c_double), ("delta_v", ctypes.c_double),
                ("delta_sdf", ctypes.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.or_create.restype = vp
    lib.or_create.argtypes = [P(_Params)]
    lib.or_destroy.argtypes = [vp]
    lib.or_integrate.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.or_integrate_rgb.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.or_read_colour.argtypes = [vp, vp]
    lib.or_num_blocks.restype = ctypes.c_longlong
    lib.or_num_blocks.argtypes = [vp]
    lib.or_total_updates.restype = ctypes.c_longlong
    lib.or_total_updates.argtypes = [vp]
    lib.or_num_ghosts.restype = ctypes.c_longlong
    lib.or_num_ghosts.argtypes = [vp]
    lib.or_read.argtypes = [vp] * 7
    lib.or_read_ghosts.argtypes = [vp, vp]
    lib.or_swap_out.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_double,
                                ctypes.c_double, ctypes.c_longlong, vp]
    lib.or_swap_in.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_double,
                               ctypes.c_double, ctypes.c_longlong, vp, vp]
    lib.or_num_host_blocks.restype = ctypes.c_longlong
    lib.or_num_host_blocks.argtypes = [vp]
    lib.or_read_host.argtypes = [vp] * 7
    lib.or_block_visible.argtypes = [P(_Params), ctypes.c_int, ctypes.c_int, vp, vp,
                                     ctypes.c_double, ctypes.c_double, vp, vp]
    lib.or_swap_merge_voxel.argtypes = [P(_Params), ctypes.c_double, ctypes.c_int,
                                        P(ctypes.c_double), P(ctypes.c_int)]
    lib.or_swap_merge_colour.argtypes = [P(_Params), vp, vp]
    lib.or_dense_create.restype = vp
    lib.or_dense_create.argtypes = [P(_Params), vp, vp]
    lib.or_dense_destroy.argtypes = [vp]
    lib.or_dense_integrate.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.or_dense_read.argtypes = [vp, vp, vp]
    lib.or_block_hit_frames.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, vp, vp, P(_Params), vp]
    lib.or_voxel_candidates.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, vp, vp, P(_Params), vp,
                                        vp, vp, ctypes.c_int]
    lib.or_float_to_i16.restype = ctypes.c_int16
    lib.or_float_to_i16.argtypes = [ctypes.c_double]
    lib.or_i16_to_float.restype = ctypes.c_double
    lib.or_i16_to_float.argtypes = [ctypes.c_int16]
    lib.or_round_f16.restype = ctypes.c_double
    lib.or_round_f16.argtypes = [ctypes.c_double]
    lib.or_icp_normals.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    lib.or_icp_downsample.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    lib.or_icp_reduce.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp,
                                  ctypes.c_double, vp, vp, vp, vp, vp]
    lib.or_volume_create.restype = vp
    lib.or_volume_create.argtypes = [vp, vp, ctypes.c_longlong]
    lib.or_volume_destroy.argtypes = [vp]
    lib.or_volume_read.argtypes = [vp, vp, vp]
    lib.or_expected_depth.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp,
                                      P(_RayParams), vp, vp]
    lib.or_raycast.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, P(_RayParams),
                               vp, vp, vp, ctypes.c_longlong, vp, vp, vp, vp]
    _lib = lib
    return lib


@dataclass
class OracleParams:
    """Fusion parameters in FP64. Callers that compare against the CUDA path
    pass the float32-rounded values the CUDA API received."""
    voxel_size: float
    mu: float
    max_weight: int = 100
    storage: int = STORAGE_F32
    pool_blocks: int = 0
    delta_px: float = 1e-3
    delta_eta: float = 1e-6
    delta_b: float = 1e-5
    delta_z: float = 1e-6

    def c(self) -> _Params:
        return _Params(self.voxel_size, self.mu, self.max_weight, self.storage,
                       self.pool_blocks, self.delta_px, self.delta_eta,
                       self.delta_b, self.delta_z)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _depth(depth) -> np.ndarray:
    return np.ascontiguousarray(depth, dtype=np.float32)


def _intr(intr) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(intr, dtype=np.float64)[:4])


def _pose(pose) -> np.ndarray:
    return np.ascontiguousarray(pose, dtype=np.float64).reshape(-1)


class Oracle:
    """Block-form oracle scene (blocks kept sorted by block coordinate)."""

    def __init__(self, params: OracleParams):
        self.params = params
        self._p = params.c()
        self._lib = _load()
        self._h = self._lib.or_create(ctypes.byref(self._p))
        if not self._h:
            raise ValueError("invalid oracle parameters")

    def close(self):
        if self._h:
            self._lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, depth, intr, pose) -> int:
        d = _depth(depth)
        H, W = d.shape
        rc = self._lib.or_integrate(self._h, _ptr(d), W, H, _ptr(_intr(intr)),
                                    _ptr(_pose(pose)))
        if rc < 0:
            raise ValueError(f"or_integrate failed ({rc})")
        return rc

    def integrate_rgb(self, depth, rgb, intr, pose) -> int:
        """Fuse one frame with an RGBX colour image (H, W, 4) uint8."""
        d = _depth(depth)
        H, W = d.shape
        c = np.ascontiguousarray(rgb, dtype=np.uint8)
        if c.shape != (H, W, 4):
            raise ValueError("colour must be (H, W, 4) uint8 like the depth")
        rc = self._lib.or_integrate_rgb(self._h, _ptr(d), _ptr(c), W, H, _ptr(_intr(intr)),
                                        _ptr(_pose(pose)))
        if rc < 0:
            raise ValueError(f"or_integrate_rgb failed ({rc})")
        return rc

    def read_colour(self) -> np.ndarray:
        """(n, 512, 4) uint8: r, g, b, colour weight, in read()'s order."""
        out = np.zeros((self.num_blocks(), 512, 4), np.uint8)
        if out.shape[0]:
            self._lib.or_read_colour(self._h, _ptr(out))
        return out

    def num_blocks(self) -> int:
        return int(self._lib.or_num_blocks(self._h))

    def total_updates(self) -> int:
        return int(self._lib.or_total_updates(self._h))

    def read(self) -> dict:
        n = self.num_blocks()
        out = dict(keys=np.zeros((n, 3), np.int32),
                   sdf=np.zeros((n, 512), np.float64),
                   w=np.zeros((n, 512), np.uint8),
                   vflag=np.zeros((n, 512), np.uint8),
                   bflag=np.zeros(n, np.uint8),
                   t_alloc=np.zeros(n, np.int32))
        self._lib.or_read(self._h, _ptr(out["keys"]), _ptr(out["sdf"]),
                          _ptr(out["w"]), _ptr(out["vflag"]),
                          _ptr(out["bflag"]), _ptr(out["t_alloc"]))
        return out

    def swap_out(self, width, height, intr, pose, margin_px, max_depth, capacity) -> int:
        """Swapping (Section 5): move device blocks that are not visible from
        the view to the host copy; returns the number moved."""
        n = ctypes.c_longlong(0)
        rc = self._lib.or_swap_out(self._h, width, height, _ptr(_intr(intr)), _ptr(_pose(pose)),
                                   float(margin_px), float(max_depth), int(capacity),
                                   ctypes.byref(n))
        if rc < 0:
            raise ValueError(f"or_swap_out failed ({rc})")
        return n.value

    def swap_in(self, width, height, intr, pose, margin_px, max_depth, capacity):
        """Bring host blocks back (merged with a fresh device block where one
        exists); returns (moved, merged)."""
        n = ctypes.c_longlong(0)
        m = ctypes.c_longlong(0)
        rc = self._lib.or_swap_in(self._h, width, height, _ptr(_intr(intr)), _ptr(_pose(pose)),
                                  float(margin_px), float(max_depth), int(capacity),
                                  ctypes.byref(n), ctypes.byref(m))
        if rc < 0:
            raise ValueError(f"or_swap_in failed ({rc})")
        return n.value, m.value

    def num_host_blocks(self) -> int:
        return int(self._lib.or_num_host_blocks(self._h))

    def read_host(self) -> dict:
        """The host copies, sorted by key (keys, sdf, w, rgbw, vflag, bflag)."""
        n = self.num_host_blocks()
        out = dict(keys=np.zeros((n, 3), np.int32),
                   sdf=np.zeros((n, 512), np.float64),
                   w=np.zeros((n, 512), np.uint8),
                   rgbw=np.zeros((n, 512, 4), np.uint8),
                   vflag=np.zeros((n, 512), np.uint8),
                   bflag=np.zeros(n, np.uint8))
        if n:
            self._lib.or_read_host(self._h, _ptr(out["keys"]), _ptr(out["sdf"]),
                                   _ptr(out["w"]), _ptr(out["rgbw"]), _ptr(out["vflag"]),
                                   _ptr(out["bflag"]))
        return out

    def ghosts(self) -> np.ndarray:
        n = int(self._lib.or_num_ghosts(self._h))
        keys = np.zeros((n, 3), np.int32)
        if n:
            self._lib.or_read_ghosts(self._h, _ptr(keys))
        return keys


class DenseOracle:
    """Dense-volume oracle: a fixed voxel grid (Section 3.2)."""

    def __init__(self, params: OracleParams, origin, size):
        self.params = params
        self._p = params.c()
        self._lib = _load()
        self.origin = np.ascontiguousarray(origin, dtype=np.int32)
        self.size = np.ascontiguousarray(size, dtype=np.int32)
        self._h = self._lib.or_dense_create(ctypes.byref(self._p),
                                            _ptr(self.origin), _ptr(self.size))
        if not self._h:
            raise ValueError("invalid dense oracle grid")

    def close(self):
        if self._h:
            self._lib.or_dense_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, depth, intr, pose) -> int:
        d = _depth(depth)
        H, W = d.shape
        rc = self._lib.or_dense_integrate(self._h, _ptr(d), W, H,
                                          _ptr(_intr(intr)), _ptr(_pose(pose)))
        if rc < 0:
            raise ValueError(f"or_dense_integrate failed ({rc})")
        return rc

    def read(self):
        nx, ny, nz = (int(v) for v in self.size)
        sdf = np.zeros((nz, ny, nx), np.float64)
        w = np.zeros((nz, ny, nx), np.uint8)
        self._lib.or_dense_read(self._h, _ptr(sdf), _ptr(w))
        return sdf, w


def block_hit_frames(key, depth_seq, intr, poses, params: OracleParams) -> np.ndarray:
    """Per-frame HIT_* bits of one block over a whole sequence."""
    lib = _load()
    k = np.ascontiguousarray(key, dtype=np.int32)
    d = _depth(depth_seq)
    N, H, W = d.shape
    P = np.ascontiguousarray(poses, dtype=np.float64).reshape(N, 16)
    hits = np.zeros(N, np.uint8)
    p = params.c()
    rc = lib.or_block_hit_frames(_ptr(k), _ptr(d), N, W, H, _ptr(_intr(intr)),
                                 _ptr(P), ctypes.byref(p), _ptr(hits))
    if rc:
        raise ValueError(f"or_block_hit_frames failed ({rc})")
    return hits


def voxel_candidates(voxel, depth_seq, intr, poses, params: OracleParams,
                     block_hits, max_out: int = 64):
    """All admissible final (sdf, w) of one voxel; None if too many arose.
    Unallocated outcomes have w = 255 and sdf = NaN."""
    lib = _load()
    v = np.ascontiguousarray(voxel, dtype=np.int32)
    d = _depth(depth_seq)
    N, H, W = d.shape
    P = np.ascontiguousarray(poses, dtype=np.float64).reshape(N, 16)
    hits = np.ascontiguousarray(block_hits, dtype=np.uint8)
    sdf = np.zeros(max_out, np.float64)
    w = np.zeros(max_out, np.uint8)
    p = params.c()
    n = lib.or_voxel_candidates(_ptr(v), _ptr(d), N, W, H, _ptr(_intr(intr)),
                                _ptr(P), ctypes.byref(p), _ptr(hits), _ptr(sdf),
                                _ptr(w), max_out)
    if n == -1:
        return None
    if n < 0:
        raise ValueError(f"or_voxel_candidates failed ({n})")
    return sdf[:n].copy(), w[:n].copy()


def block_visible(params: OracleParams, width, height, intr, pose, key, margin_px=0.0,
                  max_depth=0.0):
    """The swapping visibility rule for one block: (visible, ambiguous)."""
    lib = _load()
    p = params.c()
    k = np.ascontiguousarray(key, dtype=np.int32)
    amb = ctypes.c_int(0)
    r = lib.or_block_visible(ctypes.byref(p), int(width), int(height), _ptr(_intr(intr)),
                             _ptr(_pose(pose)), float(margin_px), float(max_depth), _ptr(k),
                             ctypes.byref(amb))
    if r < 0:
        raise ValueError("or_block_visible: bad input")
    return bool(r), bool(amb.value)


def swap_merge_voxel(params: OracleParams, Fh, wh, Fd, wd):
    """The secondary integration of one voxel: (F, w) after merging the host
    voxel (Fh, wh) into the device voxel (Fd, wd)."""
    lib = _load()
    p = params.c()
    f = ctypes.c_double(float(Fd))
    w = ctypes.c_int(int(wd))
    if lib.or_swap_merge_voxel(ctypes.byref(p), float(Fh), int(wh), ctypes.byref(f),
                               ctypes.byref(w)):
        raise ValueError("or_swap_merge_voxel: bad input")
    return f.value, w.value


def swap_merge_colour(params: OracleParams, h, d):
    """The secondary integration of one colour word (r, g, b, weight bytes)."""
    lib = _load()
    p = params.c()
    hh = np.ascontiguousarray(h, dtype=np.uint8)
    dd = np.array(d, dtype=np.uint8)
    if lib.or_swap_merge_colour(ctypes.byref(p), _ptr(hh), _ptr(dd)):
        raise ValueError("or_swap_merge_colour: bad input")
    return dd


def float_to_i16(x: float) -> int:
    return int(_load().or_float_to_i16(float(x)))


def i16_to_float(q: int) -> float:
    return float(_load().or_i16_to_float(int(q)))


def round_f16(x: float) -> float:
    return float(_load().or_round_f16(float(x)))


# ---------------------------------------------------------------------------
# Raycast (Section 4.4), raycast_oracle.c

RAY_RANGE_AMBIGUOUS, RAY_MARCH_AMBIGUOUS = 1, 2


@dataclass
class RayParams:
    """Raycast parameters in FP64 (callers comparing with the CUDA path pass
    the float32-rounded values the CUDA API received). The margins bound the
    FP32 path's error: a pixel centre within delta_px of a projected block
    box edge, a block corner within delta_z of the near plane, a sample within
    delta_v voxels of a block or cell boundary where the answer changes, an
    interpolated value within delta_sdf (plus its cell's slope times delta_v)
    of 0."""
    voxel_size: float
    mu: float
    z_near: float = 0.2
    delta_px: float = 1e-3
    delta_z: float = 1e-5
    delta_v: float = 1e-3
    delta_sdf: float = 1e-4

    def c(self) -> _RayParams:
        return _RayParams(self.voxel_size, self.mu, self.z_near, self.delta_px,
                          self.delta_z, self.delta_v, self.delta_sdf)


class Volume:
    """A block volume for the raycast oracle: keys [n][3] and the stored sdf
    values [n][512] (voxel order x + 8y + 64z) as real numbers."""

    def __init__(self, keys, sdf):
        self._lib = _load()
        k = np.ascontiguousarray(keys, dtype=np.int32).reshape(-1, 3)
        v = np.ascontiguousarray(sdf, dtype=np.float64).reshape(-1, 512)
        if k.shape[0] != v.shape[0]:
            raise ValueError("keys and sdf disagree on the block count")
        self.n = k.shape[0]
        self._h = self._lib.or_volume_create(_ptr(k), _ptr(v), self.n)
        if not self._h:
            raise ValueError("invalid volume (duplicate keys?)")

    def close(self):
        if self._h:
            self._lib.or_volume_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def read(self, P):
        """Trilinear value at P (voxel units), or None if unreadable."""
        p = np.ascontiguousarray(P, dtype=np.float64)
        out = np.zeros(1, np.float64)
        return float(out[0]) if self._lib.or_volume_read(self._h, _ptr(p), _ptr(out)) == 1 else None

    def expected_depth(self, width, height, intr, pose, params: RayParams):
        """(range [H][W][2], flags [H][W]) of the search range."""
        rng = np.zeros((height, width, 2), np.float64)
        fl = np.zeros((height, width), np.uint8)
        p = params.c()
        rc = self._lib.or_expected_depth(self._h, width, height, _ptr(_intr(intr)),
                                         _ptr(_pose(pose)), ctypes.byref(p), _ptr(rng), _ptr(fl))
        if rc:
            raise ValueError(f"or_expected_depth failed ({rc})")
        return rng, fl

    def raycast(self, width, height, intr, pose, params: RayParams, pixels=None, rng=None):
        """Cast the rays of `pixels` (flat indices y * width + x; all pixels
        if None). Returns dict(points [n][4], flags [n], steps [n], gain [n],
        range, range_flags)."""
        if rng is None:
            rng, rfl = self.expected_depth(width, height, intr, pose, params)
        else:
            rng, rfl = rng
        rng = np.ascontiguousarray(rng, dtype=np.float64)
        rfl = np.ascontiguousarray(rfl, dtype=np.uint8)
        pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
        n = width * height if pix is None else pix.shape[0]
        pts = np.zeros((n, 4), np.float64)
        fl = np.zeros(n, np.uint8)
        st = np.zeros(n, np.int32)
        gain = np.zeros(n, np.float64)
        p = params.c()
        rc = self._lib.or_raycast(self._h, width, height, _ptr(_intr(intr)), _ptr(_pose(pose)),
                                  ctypes.byref(p), _ptr(rng), _ptr(rfl),
                                  None if pix is None else _ptr(pix), n, _ptr(pts), _ptr(fl),
                                  _ptr(st), _ptr(gain))
        if rc:
            raise ValueError(f"or_raycast failed ({rc})")
        return dict(points=pts, flags=fl, steps=st, gain=gain, range=rng, range_flags=rfl)


# ---------------------------------------------------------------------------
# Depth tracker terms (Section 4.1), icp_oracle.c

ICP_TERMS = 29


def icp_normals(points) -> np.ndarray:
    """Normal map (H, W, 4) float64 of a point map (H, W, 4) float32."""
    p = np.ascontiguousarray(points, dtype=np.float32)
    H, W = p.shape[:2]
    out = np.zeros((H, W, 4), np.float64)
    if _load().or_icp_normals(_ptr(p), W, H, _ptr(out)):
        raise ValueError("or_icp_normals failed")
    return out


def icp_reduce(depth, intr, cur_pose, ref_pose, points, normals, max_dist,
               margins=(1e-3, 1e-6, 1e-5)) -> dict:
    """The 29 terms (H upper triangle 21, g 6, E, count) with their slack,
    scale and per-pixel flags."""
    d = _depth(depth)
    H, W = d.shape
    p = np.ascontiguousarray(points, dtype=np.float32)
    n = np.ascontiguousarray(normals, dtype=np.float64)
    m = np.ascontiguousarray(margins, dtype=np.float64)
    out = {k: np.zeros(ICP_TERMS, np.float64) for k in ("sums", "slack", "scale")}
    fl = np.zeros((H, W), np.uint8)
    rc = _load().or_icp_reduce(_ptr(d), W, H, _ptr(_intr(intr)), _ptr(_pose(cur_pose)),
                               _ptr(_pose(ref_pose)), _ptr(p), _ptr(n), float(max_dist), _ptr(m),
                               _ptr(out["sums"]), _ptr(out["slack"]), _ptr(out["scale"]), _ptr(fl))
    if rc:
        raise ValueError(f"or_icp_reduce failed ({rc})")
    out["flags"] = fl
    return out


def icp_downsample(depth) -> np.ndarray:
    """One level of the tracker's depth hierarchy (H/2, W/2) float32."""
    d = _depth(depth)
    H, W = d.shape
    out = np.zeros((H // 2, W // 2), np.float32)
    if _load().or_icp_downsample(_ptr(d), W, H, _ptr(out)):
        raise ValueError("or_icp_downsample failed")
    return out


def icp_system(sums):
    """(H 6x6, g 6) from the 29 terms."""
    Hm = np.zeros((6, 6))
    t = 0
    for a in range(6):
        for b in range(a, 6):
            Hm[a, b] = Hm[b, a] = sums[t]
            t += 1
    return Hm, np.asarray(sums[21:27], np.float64)
