// raycast.cu -- the raycast of Section 4.4 on sm_103a, and its C ABI.
//
// One view is rendered in four kernels on the scene stream:
//   footprints: every allocated block's box is projected; the bounding box of
//               its corners' pixels and the corners' depth range form a
//               footprint; the footprints are counted per 16x16 pixel tile
//               (wide ones, spanning more than kRayMaxTilesPerRec tiles, go
//               to one list that every tile reads);
//   scan:       exclusive prefix of the per-tile counts;
//   scatter:    each footprint's index into the lists of its tiles (the
//               report's fragments: a block x a tile);
//   march:      one CTA per tile: every thread takes its pixel's search
//               range (the minimum and maximum depth over the footprints
//               covering it) from the tile's footprints staged in shared
//               memory, then marches the pixel's ray with the five-state
//               machine, trilinear reads and two refinement steps.
#include <cmath>
#include <cstdint>

#include "scene_impl.h"

namespace tsdf {
namespace {


__device__ __forceinline__ int high_water(const SceneView& sv) {
  return sv.pool - __ldcg(&sv.sc->free_top);
}

// ---------------------------------------------------------------------------
// footprints

// Footprint of block (bx, by, bz); false if it covers no pixel centre.
__device__ __forceinline__ bool block_footprint(const RayConst& rc, int bx, int by, int bz,
                                                RayRec& r) {
  const float vx = 8.0f * (float)bx, vy = 8.0f * (float)by, vz = 8.0f * (float)bz;
  float c0[3], ex[3], ey[3], ez[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c0[i] = fmaf(rc.A_hi[3 * i], vx, fmaf(rc.A_hi[3 * i + 1], vy, fmaf(rc.A_hi[3 * i + 2], vz, rc.t_hi[i]))) +
            fmaf(rc.A_lo[3 * i], vx, fmaf(rc.A_lo[3 * i + 1], vy, fmaf(rc.A_lo[3 * i + 2], vz, rc.t_lo[i])));
    ex[i] = 8.0f * rc.A_hi[3 * i];
    ey[i] = 8.0f * rc.A_hi[3 * i + 1];
    ez[i] = 8.0f * rc.A_hi[3 * i + 2];
  }
  float c[8][3];
  float zmin = INFINITY, zmax = -INFINITY;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
      c[k][i] = c0[i] + ((k & 1) ? ex[i] : 0.0f) + ((k & 2) ? ey[i] : 0.0f) + ((k & 4) ? ez[i] : 0.0f);
    zmin = fminf(zmin, c[k][2]);
    zmax = fmaxf(zmax, c[k][2]);
  }
  if (!(zmin >= rc.z_near)) return false;  // a corner nearer than the near plane: clipped
  float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float u = rc.fx * c[k][0] / c[k][2] + rc.cx;
    const float v = rc.fy * c[k][1] / c[k][2] + rc.cy;
    umin = fminf(umin, u);
    umax = fmaxf(umax, u);
    vmin = fminf(vmin, v);
    vmax = fmaxf(vmax, v);
  }
  const float u0 = fmaxf(ceilf(umin), 0.0f), u1 = fminf(floorf(umax), (float)(rc.width - 1));
  const float v0 = fmaxf(ceilf(vmin), 0.0f), v1 = fminf(floorf(vmax), (float)(rc.height - 1));
  if (!(u0 <= u1 && v0 <= v1)) return false;
  r.z_lo = zmin;
  r.z_hi = zmax;
  r.u0 = (unsigned short)u0;
  r.u1 = (unsigned short)u1;
  r.v0 = (unsigned short)v0;
  r.v1 = (unsigned short)v1;
  return true;
}

__device__ __forceinline__ int footprint_tiles(const RayRec& r) {
  return ((r.u1 / kRayTile) - (r.u0 / kRayTile) + 1) * ((r.v1 / kRayTile) - (r.v0 / kRayTile) + 1);
}

__global__ void __launch_bounds__(256) ray_footprint_kernel(RayConst rc, SceneView sv, RayWork w) {
  const int hw = high_water(sv);
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x; base < hw; base += gridDim.x * blockDim.x) {
    const int ptr = base + threadIdx.x;
    RayRec r;
    bool has = false;
    if (ptr < hw) {
      int bx, by, bz;
      unpack_key(__ldg(&sv.key_of_ptr[ptr]), bx, by, bz);
      has = block_footprint(rc, bx, by, bz, r);
    }
    const unsigned m = __ballot_sync(~0u, has);
    if (!m) continue;
    int slot = 0;
    const int leader = __ffs(m) - 1;
    if (lane == leader) slot = atomicAdd(&w.ctr->n_rec, __popc(m));
    slot = __shfl_sync(~0u, slot, leader) + __popc(m & ((1u << lane) - 1));
    if (!has) continue;
    w.rec[slot] = r;
    if (footprint_tiles(r) > kRayMaxTilesPerRec) {
      w.large[atomicAdd(&w.ctr->n_large, 1)] = slot;
    } else {
      for (int ty = r.v0 / kRayTile; ty <= r.v1 / kRayTile; ++ty)
        for (int tx = r.u0 / kRayTile; tx <= r.u1 / kRayTile; ++tx)
          atomicAdd(&w.tile_count[ty * rc.tiles_x + tx], 1);
    }
  }
}

// Exclusive prefix of the tile counts (one CTA of 1024 threads, each owning a
// contiguous run of tiles); the fill cursors start at the offsets.
__global__ void __launch_bounds__(1024) ray_scan_kernel(RayWork w, int n_tiles) {
  __shared__ int s_warp[32];
  const int per = (n_tiles + 1023) / 1024;
  const int b = threadIdx.x * per, e = min(b + per, n_tiles);
  int sum = 0;
  for (int i = b; i < e; ++i) sum += w.tile_count[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(~0u, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int x = s_warp[lane];
    int y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int z = __shfl_up_sync(~0u, y, o);
      if (lane >= o) y += z;
    }
    s_warp[lane] = y - x;
  }
  __syncthreads();
  int run = s_warp[wid] + incl - sum;
  for (int i = b; i < e; ++i) {
    w.tile_off[i] = run;
    w.tile_cursor[i] = run;
    run += w.tile_count[i];
  }
  if (threadIdx.x == 1023) w.tile_off[n_tiles] = run;
}

__global__ void __launch_bounds__(256) ray_scatter_kernel(RayWork w, int tiles_x) {
  const int n = __ldcg(&w.ctr->n_rec);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const RayRec r = w.rec[i];
    if (footprint_tiles(r) > kRayMaxTilesPerRec) continue;
    for (int ty = r.v0 / kRayTile; ty <= r.v1 / kRayTile; ++ty)
      for (int tx = r.u0 / kRayTile; tx <= r.u1 / kRayTile; ++tx)
        w.frag[atomicAdd(&w.tile_cursor[ty * tiles_x + tx], 1)] = i;
  }
}

// ---------------------------------------------------------------------------
// march

// Pool index of block (bx, by, bz), or -1 if it is not allocated; the last
// answer is kept (consecutive samples mostly fall in one block).
struct BlockCache {
  unsigned long long key;
  int ptr;
};

__device__ __forceinline__ int block_ptr(const SceneView& sv, BlockCache& c, int bx, int by, int bz) {
  if (bx < -32768 || bx > 32767 || by < -32768 || by > 32767 || bz < -32768 || bz > 32767)
    return -1;  // outside the key range: never allocated
  const unsigned long long k = pack_key(bx, by, bz);
  if (k == c.key) return c.ptr;
  int p = -1;
  const unsigned b = bucket_of(k, (unsigned)sv.bucket_mask);
  const int base = (int)b * sv.entries_per_bucket;
  int e = -1;
  bool full = true;  // occupied slots form a prefix; a chain hangs only off a full bucket
  for (int s = 0; s < sv.entries_per_bucket; ++s) {
    const unsigned long long kk = __ldg(&sv.entries[base + s].key);
    if (kk == k) {
      e = base + s;
      break;
    }
    if (kk == kKeyEmpty) {
      full = false;
      break;
    }
  }
  if (e < 0 && full) {
    int idx = __ldg(&sv.entries[base].next);
    for (int guard = 0; idx >= 0 && guard <= sv.excess_cap; ++guard) {
      const int x = sv.n_bucket_entries + idx;
      if (__ldg(&sv.entries[x].key) == k) {
        e = x;
        break;
      }
      idx = __ldg(&sv.entries[x].next);
    }
  }
  if (e >= 0) p = __ldg(&sv.entries[e].ptr);
  if (p < 0) p = -1;
  c.key = k;
  c.ptr = p;
  return p;
}

// Trilinear read at P (voxel units): false if one of the cell's eight voxels
// lies in a block that is not allocated. The sample's own block comes from
// `own`; a cell whose lower corner has local coordinate 7 on an axis reaches
// into the next block on that axis, and each such neighbour is looked up once
// (through `nb`, which keeps the last neighbour).
template <int S>
__device__ __forceinline__ bool read_interp(const SceneView& sv, BlockCache& own, BlockCache& nb,
                                            float px, float py, float pz, float& sdf) {
  using T = typename Storage<S>::T;
  const float fx0 = floorf(px), fy0 = floorf(py), fz0 = floorf(pz);
  const int cx = (int)fx0, cy = (int)fy0, cz = (int)fz0;
  const float fx = px - fx0, fy = py - fy0, fz = pz - fz0;
  const int bx = cx >> 3, by = cy >> 3, bz = cz >> 3;
  const int x0 = cx & 7, y0 = cy & 7, z0 = cz & 7;
  const bool sx = x0 == 7, sy = y0 == 7, sz = z0 == 7;
  const int p000 = block_ptr(sv, own, bx, by, bz);
  if (p000 < 0) return false;
  int p100 = p000, p010 = p000, p001 = p000, p110 = p000, p101 = p000, p011 = p000, p111 = p000;
  if (sx | sy | sz) {
    if (sx && (p100 = block_ptr(sv, nb, bx + 1, by, bz)) < 0) return false;
    if (sy && (p010 = block_ptr(sv, nb, bx, by + 1, bz)) < 0) return false;
    if (sz && (p001 = block_ptr(sv, nb, bx, by, bz + 1)) < 0) return false;
    p110 = sx ? (sy ? block_ptr(sv, nb, bx + 1, by + 1, bz) : p100) : p010;
    p101 = sx ? (sz ? block_ptr(sv, nb, bx + 1, by, bz + 1) : p100) : p001;
    p011 = sy ? (sz ? block_ptr(sv, nb, bx, by + 1, bz + 1) : p010) : p001;
    p111 = sx ? (sy ? (sz ? block_ptr(sv, nb, bx + 1, by + 1, bz + 1) : p110) : p101) : p011;
    if ((p110 | p101 | p011 | p111) < 0) return false;
  }
  const int x1 = sx ? 0 : x0 + 1, y1 = sy ? 0 : y0 + 1, z1 = sz ? 0 : z0 + 1;
  const T* vox = (const T*)sv.sdf;
  // storage order inside a block: x + 8 z + 64 y
  auto at = [&](int p, int x, int y, int z) {
    return Storage<S>::load(__ldg(&vox[(size_t)p * kBlockVoxels + x + 8 * z + 64 * y]));
  };
  const float v0 = at(p000, x0, y0, z0), v1 = at(p100, x1, y0, z0);
  const float v2 = at(p010, x0, y1, z0), v3 = at(p110, x1, y1, z0);
  const float v4 = at(p001, x0, y0, z1), v5 = at(p101, x1, y0, z1);
  const float v6 = at(p011, x0, y1, z1), v7 = at(p111, x1, y1, z1);
  const float x00 = fmaf(fx, v1 - v0, v0);
  const float x10 = fmaf(fx, v3 - v2, v2);
  const float x01 = fmaf(fx, v5 - v4, v4);
  const float x11 = fmaf(fx, v7 - v6, v6);
  const float y_0 = fmaf(fy, x10 - x00, x00);
  const float y_1 = fmaf(fy, x11 - x01, x01);
  sdf = fmaf(fz, y_1 - y_0, y_0);
  return true;
}

// Ray distance as an unevaluated sum hi + lo (voxel units), so that dozens
// of steps add no rounding to the sample positions.
struct RayT {
  float hi, lo;
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
  }
  __device__ __forceinline__ float value() const { return hi + lo; }
};

enum { kCoarse = 0, kFine = 1, kSurface = 2 };

struct Ray {
  float o_hi[3], o_lo[3], d[3];
  __device__ __forceinline__ void at(const RayT& t, float P[3]) const {
#pragma unroll
    for (int i = 0; i < 3; ++i) P[i] = fmaf(t.hi, d[i], o_hi[i]) + fmaf(t.lo, d[i], o_lo[i]);
  }
};

// March one ray over [t_lo, t_end]; true with the surface at P.
template <int S>
__device__ bool march(const SceneView& sv, const Ray& ray, float t_lo, float t_lo_err, float t_end,
                      float mu_v, float P[3], int& steps, bool& guard) {
  BlockCache bc{kKeyEmpty, -1}, nb{kKeyEmpty, -1};
  RayT t{t_lo, t_lo_err};
  int state = kCoarse;
  float sdf;
  for (;;) {
    if (t.value() > t_end) return false;
    if (steps >= kRayMaxSteps) {
      guard = true;
      return false;
    }
    ++steps;
    ray.at(t, P);
    if (state == kCoarse) {
      const int bx = (int)floorf(P[0] * 0.125f), by = (int)floorf(P[1] * 0.125f),
                bz = (int)floorf(P[2] * 0.125f);
      if (block_ptr(sv, bc, bx, by, bz) >= 0) {
        t.add(-8.0f);  // one step back, then the finer search
        state = kFine;
      } else {
        t.add(8.0f);
      }
      continue;
    }
    if (!read_interp<S>(sv, bc, nb, P[0], P[1], P[2], sdf)) {
      state = kFine;
      t.add(mu_v);
      continue;
    }
    if (state == kFine && sdf < 0.0f) return false;  // WRONG_SIDE
    state = kSurface;
    if (sdf < 0.0f) {  // BEHIND_SURFACE: two interpolation steps back onto it
      t.add(sdf * mu_v);
      ray.at(t, P);
      if (read_interp<S>(sv, bc, nb, P[0], P[1], P[2], sdf)) {
        t.add(sdf * mu_v);
        ray.at(t, P);
      }
      return true;
    }
    t.add(fmaxf(sdf * mu_v, 1.0f));
  }
}

// March CTAs: one 8x8 quarter of a 16x16 tile each (a warp is 8x4 pixels);
// small CTAs free an SM's slots soon after their slowest ray ends.
constexpr int kMarchSide = 8;
constexpr int kMarchThreads = kMarchSide * kMarchSide;

template <int S>
__global__ void __launch_bounds__(kMarchThreads) raycast_kernel(RayConst rc, SceneView sv, RayWork w,
                                                                float4* points, float2* range) {
  __shared__ RayRec s_rec[kMarchThreads];
  const int tile = blockIdx.x >> 2, quarter = blockIdx.x & 3;
  const int u = (tile % rc.tiles_x) * kRayTile + (quarter & 1) * kMarchSide + (threadIdx.x % kMarchSide);
  const int v = (tile / rc.tiles_x) * kRayTile + (quarter >> 1) * kMarchSide + (threadIdx.x / kMarchSide);
  float z_lo = INFINITY, z_hi = -INFINITY;
  // search range: the tile's footprints, then the wide ones
  for (int pass = 0; pass < 2; ++pass) {
    const int b = pass == 0 ? w.tile_off[tile] : 0;
    const int e = pass == 0 ? w.tile_off[tile + 1] : __ldcg(&w.ctr->n_large);
    const int* list = pass == 0 ? w.frag : w.large;
    for (int c = b; c < e; c += kMarchThreads) {
      const int m = min(kMarchThreads, e - c);
      __syncthreads();
      if ((int)threadIdx.x < m) s_rec[threadIdx.x] = w.rec[list[c + threadIdx.x]];
      __syncthreads();
      for (int i = 0; i < m; ++i) {
        const RayRec r = s_rec[i];
        if (u >= r.u0 && u <= r.u1 && v >= r.v0 && v <= r.v1) {
          z_lo = fminf(z_lo, r.z_lo);
          z_hi = fmaxf(z_hi, r.z_hi);
        }
      }
    }
  }
  int steps = 0;
  bool hit = false, guard = false;
  if (u < rc.width && v < rc.height) {
    float P[3] = {0.0f, 0.0f, 0.0f};
    if (z_lo <= z_hi) {
      // the pixel centre's ray: world voxel units per metre of camera depth
      const float qx = ((float)u - rc.cx) * rc.inv_fx, qy = ((float)v - rc.cy) * rc.inv_fy;
      float E[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) E[i] = fmaf(rc.L[3 * i], qx, fmaf(rc.L[3 * i + 1], qy, rc.L[3 * i + 2]));
      const float len = sqrtf(fmaf(E[0], E[0], fmaf(E[1], E[1], E[2] * E[2])));
      Ray ray;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        ray.o_hi[i] = rc.o_hi[i];
        ray.o_lo[i] = rc.o_lo[i];
        ray.d[i] = E[i] / len;
      }
      const float t0 = z_lo * len;
      hit = march<S>(sv, ray, t0, fmaf(z_lo, len, -t0), z_hi * len, rc.mu_v, P, steps, guard);
    }
    const size_t o = (size_t)v * rc.width + u;
    points[o] = hit ? make_float4(P[0] * rc.voxel_size, P[1] * rc.voxel_size, P[2] * rc.voxel_size, 1.0f)
                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (range) range[o] = make_float2(z_lo, z_hi);
  }
  // counters: one atomic per warp and counter (no barrier: a warp leaves as
  // soon as its rays are done)
  const unsigned ws = __reduce_add_sync(~0u, (unsigned)steps);
  const unsigned wh = __reduce_add_sync(~0u, hit ? 1u : 0u);
  const unsigned wg = __reduce_add_sync(~0u, guard ? 1u : 0u);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&w.ctr->steps, (unsigned long long)ws);
    if (wh) atomicAdd(&w.ctr->hits, (unsigned long long)wh);
    if (wg) atomicAdd(&w.ctr->guard, (unsigned long long)wg);
  }
}

}  // namespace

cudaError_t launch_raycast_range(const RayConst& rc, const SceneView& sv, const RayWork& w,
                                 int sm_count, cudaStream_t st) {
  const int n_tiles = rc.tiles_x * rc.tiles_y;
  cudaError_t e = cudaMemsetAsync(w.ctr, 0, sizeof(RayCounters) + (size_t)n_tiles * sizeof(int), st);
  if (e != cudaSuccess) return e;
  ray_footprint_kernel<<<sm_count * 8, 256, 0, st>>>(rc, sv, w);
  ray_scan_kernel<<<1, 1024, 0, st>>>(w, n_tiles);
  ray_scatter_kernel<<<sm_count * 4, 256, 0, st>>>(w, rc.tiles_x);
  return cudaGetLastError();
}

cudaError_t launch_raycast_march(const RayConst& rc, const SceneView& sv, const RayWork& w,
                                 int storage, float4* points, float2* range, cudaStream_t st) {
  const int n_tiles = rc.tiles_x * rc.tiles_y;
  switch (storage) {
    case TSDF_STORAGE_I16:
      raycast_kernel<TSDF_STORAGE_I16><<<n_tiles * 4, kMarchThreads, 0, st>>>(rc, sv, w, points, range);
      break;
    case TSDF_STORAGE_F16:
      raycast_kernel<TSDF_STORAGE_F16><<<n_tiles * 4, kMarchThreads, 0, st>>>(rc, sv, w, points, range);
      break;
    default:
      raycast_kernel<TSDF_STORAGE_F32><<<n_tiles * 4, kMarchThreads, 0, st>>>(rc, sv, w, points, range);
  }
  return cudaGetLastError();
}

}  // namespace tsdf

// ---------------------------------------------------------------------------
// C ABI

using namespace tsdf;

namespace {

void split2(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// FP64 pose handling of one raycast: world -> camera for the block corners,
// camera -> world (voxel units) for the rays.
int make_ray_const(const tsdf_scene* s, const tsdf_intrinsics* in, const double* M, float z_near,
                   RayConst* rc) {
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(M[i])) return TSDF_ERR_INVALID_ARG;
  if (M[12] != 0.0 || M[13] != 0.0 || M[14] != 0.0 || M[15] != 1.0) return TSDF_ERR_INVALID_ARG;
  const double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8], h = M[9],
               k = M[10];
  const double det = a * (e * k - f * h) - b * (d * k - f * g) + c * (d * h - e * g);
  if (!(std::fabs(det) > 1e-300) || !std::isfinite(det)) return TSDF_ERR_INVALID_ARG;
  const double Ri[9] = {(e * k - f * h) / det, (c * h - b * k) / det, (b * f - c * e) / det,
                        (f * g - d * k) / det, (a * k - c * g) / det, (c * d - a * f) / det,
                        (d * h - e * g) / det, (b * g - a * h) / det, (a * e - b * d) / det};
  const double vs = (double)s->desc.voxel_size;
  const double R[9] = {a, b, c, d, e, f, g, h, k};
  for (int i = 0; i < 9; ++i) {
    split2(vs * R[i], rc->A_hi[i], rc->A_lo[i]);
    rc->L[i] = (float)(Ri[i] / vs);
  }
  const double t[3] = {M[3], M[7], M[11]};
  for (int r = 0; r < 3; ++r) {
    split2(t[r], rc->t_hi[r], rc->t_lo[r]);
    const double o = -(Ri[3 * r] * t[0] + Ri[3 * r + 1] * t[1] + Ri[3 * r + 2] * t[2]) / vs;
    split2(o, rc->o_hi[r], rc->o_lo[r]);
  }
  rc->fx = in->fx;
  rc->fy = in->fy;
  rc->cx = in->cx;
  rc->cy = in->cy;
  rc->inv_fx = (float)(1.0 / (double)in->fx);
  rc->inv_fy = (float)(1.0 / (double)in->fy);
  rc->z_near = z_near;
  rc->mu_v = (float)((double)s->desc.mu / vs);
  rc->voxel_size = s->desc.voxel_size;
  rc->width = in->width;
  rc->height = in->height;
  rc->tiles_x = (in->width + kRayTile - 1) / kRayTile;
  rc->tiles_y = (in->height + kRayTile - 1) / kRayTile;
  return TSDF_OK;
}

// Grow the scene's raycast work buffers to its pool and n_tiles tiles.
int ensure_ray_work(tsdf_scene* s, int n_tiles) {
  RayWork& w = s->ray;
  if (w.rec && w.pool >= s->sv.pool && w.tile_cap >= n_tiles) return TSDF_OK;
  free_ray_work(s);
  const size_t pool = (size_t)s->sv.pool;
  const size_t ctr_bytes = sizeof(RayCounters) + (size_t)n_tiles * sizeof(int);
  cudaError_t e = cudaMalloc((void**)&w.rec, pool * sizeof(RayRec));
  if (e == cudaSuccess) e = cudaMalloc((void**)&w.frag, pool * kRayMaxTilesPerRec * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&w.large, pool * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&w.ctr, ctr_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&w.tile_off, ((size_t)n_tiles + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&w.tile_cursor, (size_t)n_tiles * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w.ctr, 0, ctr_bytes);
  if (e != cudaSuccess) {
    free_ray_work(s);
    return cuda_fail(e);
  }
  w.tile_count = (int*)(w.ctr + 1);
  w.tile_cap = n_tiles;
  w.pool = s->sv.pool;
  return TSDF_OK;
}

}  // namespace

namespace tsdf {

void free_ray_work(tsdf_scene* s) {
  RayWork& w = s->ray;
  cudaFree(w.rec);
  cudaFree(w.frag);
  cudaFree(w.large);
  cudaFree(w.ctr);
  cudaFree(w.tile_off);
  cudaFree(w.tile_cursor);
  w = RayWork{};
}

}  // namespace tsdf

int tsdf_raycast(tsdf_scene* s, const tsdf_intrinsics* intr, const double world_to_cam[16],
                 float z_near, float* points, float* range) {
  if (!s || !world_to_cam || !points) return TSDF_ERR_INVALID_ARG;
  int rc = validate_intr(intr);
  if (rc) return rc;
  if (!std::isfinite(z_near) || !(z_near > 0.0f)) return TSDF_ERR_INVALID_ARG;
  if (((uintptr_t)points & 15) || ((uintptr_t)range & 7)) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  RayConst c;
  if ((rc = make_ray_const(s, intr, world_to_cam, z_near, &c))) return rc;
  if ((rc = ensure_ray_work(s, c.tiles_x * c.tiles_y))) return rc;
  bool capturing = false;
  cudaEvent_t* ev = s->timer.next(s->stream, &capturing);
  TSDF_CUDA(s->timer.mark(ev, 0, s->stream, capturing));
  TSDF_CUDA(launch_raycast_range(c, s->sv, s->ray, s->sm_count, s->stream));
  TSDF_CUDA(s->timer.mark(ev, 1, s->stream, capturing));
  TSDF_CUDA(launch_raycast_march(c, s->sv, s->ray, s->desc.storage, (float4*)points,
                                 (float2*)range, s->stream));
  TSDF_CUDA(s->timer.mark(ev, 2, s->stream, capturing));
  s->launches += 4;
  return TSDF_OK;
}

int tsdf_get_raycast_stats(tsdf_scene* s, tsdf_raycast_stats* out) {
  if (!s || !out) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  RayCounters c{};
  if (s->ray.ctr) {
    TSDF_CUDA(cudaMemcpyAsync(&c, s->ray.ctr, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    TSDF_CUDA(cudaStreamSynchronize(s->stream));
  }
  out->footprints = c.n_rec;
  out->wide_footprints = c.n_large;
  out->steps = (int64_t)c.steps;
  out->hits = (int64_t)c.hits;
  out->guard_stops = (int64_t)c.guard;
  return TSDF_OK;
}
