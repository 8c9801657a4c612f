// integrate.cu -- visible list (Section 4.2, third stage) and per-voxel
// integration (Section 4.3, computeUpdatedVoxelDepthInfo).
//
// visible_kernel  : (a) initialises the voxels of the blocks the commit handed
//                   out this frame (sdf 1, w 0); (b) scans the allocated
//                   blocks [0, high-water) (dense: pool indices are handed out
//                   in order and never freed) in even per-CTA ranges. For
//                   every block a conservative test decides whether any voxel
//                   can be written by rule U this frame; the blocks that pass
//                   are compacted (CTA prefix sum, one atomic per CTA and
//                   pass) into 32 B records carrying the block origin's
//                   camera point as a double-float.
// integrate_kernel: persistent; a visible block is four work units (its
//                   8x8x2-voxel slabs), four consecutive voxels (a quad) per
//                   lane, two units in flight per warp. A quad's projections
//                   are tested once against the image border (x is monotonic
//                   along a quad), all depth gathers are issued before voxel
//                   data is touched, and voxel data (16 B of f32 sdf + 4 B of
//                   weights per quad) is read and written only when the rule
//                   updates one of the quad's voxels. Its first thread counts
//                   the frame and zeroes the allocation counters (and the
//                   coarse depth pyramid) for the next frame; each CTA adds
//                   its update count with one atomic.
//
// Arithmetic: FP32 throughout, no FP64. The block origin is carried as an
// unevaluated sum of two floats built with exact product / sum transforms, so
// eta = d - z keeps ~1e-8 m accuracy at several metres; the per-voxel offset
// A l is a plain float (|A l| < 0.1 m).
#include <cstdlib>

#include "tsdf_internal.cuh"

namespace tsdf {

namespace {

// error-free transforms (Knuth two-sum; FMA two-product)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// camera point of voxel o (integer coordinates, |o| < 2^19), c = A o + t, as
// hi + lo with |error| ~ 2^-44 |c|
__device__ __forceinline__ void origin_df(const FrameConst& fc, const float o[3], float chi[3],
                                          float clo[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float s = fc.t_hi[r], err = fc.t_lo[r];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float p = fc.A_hi[3 * r + j] * o[j];
      const float pe = fmaf(fc.A_hi[3 * r + j], o[j], -p);  // exact product error
      float s2, e2;
      two_sum(s, p, s2, e2);
      s = s2;
      err += pe + e2 + fc.A_lo[3 * r + j] * o[j];
    }
    chi[r] = s + err;
    clo[r] = err - (chi[r] - s);
  }
}

// ----------------------------------------------------------------------------
// visible list

constexpr int kVisThreads = 256;

// Can rule U write any voxel l in [0,7] x [0,7] x [lz0, lz1] of the block whose
// origin voxel has the (float) camera point c0? Conservative: the voxels lie
// in the box spanned by those lattice offsets; its 8 corners bound every
// voxel's camera z and, when all are in front of the camera, the voxels'
// image points (perspective maps the box onto the hull of the corners'
// images).
__device__ __forceinline__ bool box_visible(const FrameConst& fc, const unsigned* tile_max,
                                            const float c0[3], float lz0, float lz1, float zfar) {
  const float kSlackZ = 1e-3f, kSlackPx = 1.0f;
  float zmin = INFINITY, zmax = -INFINITY, xmin = INFINITY, xmax = -INFINITY,
        ymin = INFINITY, ymax = -INFINITY;
  bool front = true;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float lx = (c & 1) ? 7.0f : 0.0f, ly = (c & 2) ? 7.0f : 0.0f, lz = (c & 4) ? lz1 : lz0;
    const float X = fmaf(fc.A_hi[0], lx, fmaf(fc.A_hi[1], ly, fmaf(fc.A_hi[2], lz, c0[0])));
    const float Y = fmaf(fc.A_hi[3], lx, fmaf(fc.A_hi[4], ly, fmaf(fc.A_hi[5], lz, c0[1])));
    const float Z = fmaf(fc.A_hi[6], lx, fmaf(fc.A_hi[7], ly, fmaf(fc.A_hi[8], lz, c0[2])));
    zmin = fminf(zmin, Z);
    zmax = fmaxf(zmax, Z);
    if (Z < kSlackZ) {
      front = false;
    } else {
      const float rz = 1.0f / Z;
      const float x = fmaf(fc.fx * X, rz, fc.cx), y = fmaf(fc.fy * Y, rz, fc.cy);
      xmin = fminf(xmin, x);
      xmax = fmaxf(xmax, x);
      ymin = fminf(ymin, y);
      ymax = fmaxf(ymax, y);
    }
  }
  if (zmax < -kSlackZ) return false;           // every voxel behind the camera
  if (zmin > zfar + kSlackZ) return false;     // every voxel > mu behind any depth
  if (!front) return true;                     // straddles the camera plane
  if (xmax < 1.0f - kSlackPx || xmin > fc.xmax + kSlackPx) return false;
  if (ymax < 1.0f - kSlackPx || ymin > fc.ymax + kSlackPx) return false;
  if (fc.use_tiles) {
    // Every voxel reads the depth of a pixel inside [xmin, xmax] x [ymin,
    // ymax] (rounded, plus slack); if the box's nearest point is more than mu
    // behind the largest depth over that rectangle, rule U rejects every
    // voxel (eta < -mu). The largest depth comes from the coarsest-enough
    // level of the depth-max pyramid: at most 2 x 2 cells (blocks larger on
    // screen than 2 x 2 cells of the coarsest level are kept).
    const int px0 = max(0, (int)floorf(xmin - kSlackPx));
    const int px1 = min(fc.width - 1, (int)ceilf(xmax + kSlackPx));
    const int py0 = max(0, (int)floorf(ymin - kSlackPx));
    const int py1 = min(fc.height - 1, (int)ceilf(ymax + kSlackPx));
    int l = 0;
    while (l < kPyramidLevels && (((px1 >> (4 + l)) - (px0 >> (4 + l))) > 1 ||
                                  ((py1 >> (4 + l)) - (py0 >> (4 + l))) > 1))
      ++l;
    if (l == kPyramidLevels) return true;  // too large on screen: no depth cull
    int wl, hl;
    const int off = pyramid_level(fc.tiles_x, fc.tiles_y, l, wl, hl);
    const int cx0 = px0 >> (4 + l), cx1 = px1 >> (4 + l);
    const int cy0 = py0 >> (4 + l), cy1 = py1 >> (4 + l);
    const unsigned m =
        max(max(__ldcg(&tile_max[off + cy0 * wl + cx0]), __ldcg(&tile_max[off + cy0 * wl + cx1])),
            max(__ldcg(&tile_max[off + cy1 * wl + cx0]), __ldcg(&tile_max[off + cy1 * wl + cx1])));
    if (zmin > __uint_as_float(m) + fc.mu + kSlackZ) return false;
  }
  return true;
}

template <int S>
__global__ void __launch_bounds__(kVisThreads) visible_kernel(FrameConst fc, SceneView sv) {
  using T = typename Storage<S>::T;
  __shared__ int s_warp[kVisThreads / 32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // (a) initialise this frame's new blocks: warp per block
  {
    const int n_new = __ldcg(&sv.fc->n_new);
    const int base = __ldcg(&sv.fc->assign_base);
    const int gw = blockIdx.x * (kVisThreads / 32) + warp;
    const int nw = gridDim.x * (kVisThreads / 32);
    const T init = Storage<S>::initial();
    for (int i = gw; i < n_new && base - 1 - i >= 0; i += nw) {
      const int ptr = __ldcg(&sv.free_stack[base - 1 - i]);
      if (ptr < 0 || ptr >= sv.pool) {
        if (lane == 0) set_status(sv.sc, kStInternal);
        continue;
      }
      T* sdf = reinterpret_cast<T*>(sv.sdf) + (size_t)ptr * kBlockVoxels;
#pragma unroll
      for (int j = 0; j < kBlockVoxels / 32; ++j) sdf[32 * j + lane] = init;
      reinterpret_cast<uint4*>(sv.w + (size_t)ptr * kBlockVoxels)[lane] = make_uint4(0, 0, 0, 0);
    }
  }

  // (b) this CTA's even share of the allocated blocks, one block per thread
  // and pass; each visible block gets one record
  const int high_water = sv.pool - __ldcg(&sv.sc->free_top);
  const unsigned dmax_bits = __ldcg(&sv.fc->depth_max_bits);
  const float zfar = __uint_as_float(dmax_bits) + fc.mu;
  const int b0 = (int)((long long)high_water * blockIdx.x / gridDim.x);
  const int b1 = (int)((long long)high_water * (blockIdx.x + 1) / gridDim.x);
  for (int i0 = b0; i0 < b1; i0 += kVisThreads) {
    const int ptr = i0 + threadIdx.x;
    bool vis = false;
    float o[3] = {0.0f, 0.0f, 0.0f};
    if (ptr < b1 && dmax_bits != 0u) {
      int bx, by, bz;
      unpack_key(__ldg(&sv.key_of_ptr[ptr]), bx, by, bz);
      o[0] = 8.0f * bx;
      o[1] = 8.0f * by;
      o[2] = 8.0f * bz;
      float c0[3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        c0[r] = fmaf(fc.A_hi[3 * r], o[0],
                     fmaf(fc.A_hi[3 * r + 1], o[1], fmaf(fc.A_hi[3 * r + 2], o[2], fc.t_hi[r])));
      vis = box_visible(fc, sv.tile_max, c0, 0.0f, 7.0f, zfar);
    }
    // CTA-wide compaction: warp ballots, warp offsets in shared memory, one
    // global atomic per CTA and pass
    const unsigned bal = __ballot_sync(0xffffffffu, vis);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int total = 0;
      for (int w = 0; w < kVisThreads / 32; ++w) {
        const int c = s_warp[w];
        s_warp[w] = total;
        total += c;
      }
      s_base = total ? atomicAdd(&sv.fc->n_visible, total) : 0;
    }
    __syncthreads();
    if (vis) {
      VisRec r;
      r.ptr = ptr;
      origin_df(fc, o, r.chi, r.clo);
      r.pad = 0;
      sv.visible[s_base + s_warp[warp] + __popc(bal & ((1u << lane) - 1u))] = r;
    }
    __syncthreads();  // s_warp / s_base are reused by the next pass
  }
}

// ----------------------------------------------------------------------------
// integration

constexpr int kIntThreads = 256;
constexpr int kIntWarps = kIntThreads / 32;

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One work unit = one 8x8x2-voxel slab of a visible block: lane l owns the
// quad of voxels 4l + 128k .. 4l + 128k + 3 of slab k. Each warp carries U
// units at once (units i, i + W, ... for W warps) so that their loads
// overlap; U trades registers (occupancy) for loads in flight per warp.

template <int S>
struct UnitState {
  int ptr, k;
  float chi2, lz[4];
  float fv[4];
  unsigned mask;
};

template <int S, int kUnitsInFlight>
__global__ void __launch_bounds__(kIntThreads) integrate_kernel(FrameConst fc, SceneView sv) {
  using St = Storage<S>;
  using T = typename St::T;
  __shared__ float s_rcp[256];  // s_rcp[w] = 1 / (w + 1), rounded once
  __shared__ unsigned long long s_upd[kIntWarps];
  s_rcp[threadIdx.x] = 1.0f / (float)(threadIdx.x + 1);

  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * kIntWarps + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * kIntWarps;
  const int n_units = 4 * __ldcg(&sv.fc->n_visible);

  // The allocation-group counters and the coarse pyramid levels were last
  // read by the visible kernel: count the frame and zero them for the next.
  {
    FrameCounters* fr = sv.fc;
    const int gtid = blockIdx.x * kIntThreads + threadIdx.x;
    if (gtid == 0) {
      sv.sc->frames += 1;
      sv.sc->last_new = (unsigned long long)fr->n_new;
      fr->n_new = 0;
      fr->n_overflow = 0;
      fr->assign_base = 0;
      fr->depth_max_bits = 0u;
      fr->alloc_done = 0;
      fr->frame_pending = 1;
    }
    if (gtid < kArriveGroups) fr->arrive[gtid] = 0;
    if (fc.use_tiles) {
      int wl, hl;
      const int lo = fc.tiles_x * fc.tiles_y;
      const int hi = pyramid_level(fc.tiles_x, fc.tiles_y, kPyramidLevels, wl, hl);
      for (int i = lo + gtid; i < hi; i += gridDim.x * kIntThreads) sv.tile_max[i] = 0u;
    }
  }
  __syncthreads();
  const float* __restrict__ depth = sv.depth_san;  // pitch = width, -inf = none
  const int dpitch = fc.width;

  // lane -> voxels 4*lane + 128*k + j of slab k (j = 0..3):
  // lx = 4 (lane & 1) + j, ly = (lane >> 1) & 7, lz = (lane >> 4) + 2 k
  const float lx0 = (float)(4 * (lane & 1));
  const float ly = (float)((lane >> 1) & 7);
  const float lz0 = (float)(lane >> 4);
  float lbase[3], dk[3];  // A l of the lane's first voxel in slab 0; slab step
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    lbase[r] = fmaf(fc.A_hi[3 * r], lx0, fmaf(fc.A_hi[3 * r + 1], ly, fc.A_hi[3 * r + 2] * lz0));
    dk[r] = 2.0f * fc.A_hi[3 * r + 2];
  }
  // one voxel step along x: camera z, and fx X, fy Y of the projection
  const float dz = fc.A_hi[6], pdx = fc.fx * fc.A_hi[0], pdy = fc.fy * fc.A_hi[3];
  const unsigned maxw = (unsigned)fc.max_weight;
  unsigned long long updated = 0;

  for (int base = gwarp; base < n_units; base += nwarps * kUnitsInFlight) {
    UnitState<S> us[kUnitsInFlight];
    // projections and depth gathers of every unit in flight
#pragma unroll
    for (int q = 0; q < kUnitsInFlight; ++q) {
      const int u = base + q * nwarps;
      us[q].mask = 0;
      us[q].ptr = -1;
      if (u >= n_units) continue;
      const VisRec vr = sv.visible[u >> 2];
      const int k = u & 3;
      if (vr.ptr < 0 || vr.ptr >= sv.pool) {
        if (lane == 0) set_status(sv.sc, kStInternal);  // inconsistent record: skip it
        continue;
      }
      us[q].ptr = vr.ptr;
      us[q].k = k;
      us[q].chi2 = vr.chi[2];
      const float kk = (float)k;
      // the quad's first voxel: z keeps its low part (for eta), x and y are
      // only needed to float accuracy
      const float lz_0 = vr.clo[2] + fmaf(kk, dk[2], lbase[2]);
      const float px_0 = fc.fx * (vr.chi[0] + (vr.clo[0] + fmaf(kk, dk[0], lbase[0])));
      const float py_0 = fc.fy * (vr.chi[1] + (vr.clo[1] + fmaf(kk, dk[1], lbase[1])));
      float Z[4], x[4], y[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        us[q].lz[j] = fmaf((float)j, dz, lz_0);
        Z[j] = vr.chi[2] + us[q].lz[j];
        const float rz = rcp_approx(Z[j]);
        x[j] = fmaf(fmaf((float)j, pdx, px_0), rz, fc.cx);
        y[j] = fmaf(fmaf((float)j, pdy, py_0), rz, fc.cy);
      }
      // x, y are monotonic along the quad when z > 0 on it (a ratio of
      // affine functions), so the ends bound the four voxels
      const bool quad_in = fminf(Z[0], Z[3]) > 0.0f && fminf(x[0], x[3]) >= 1.0f &&
                           fmaxf(x[0], x[3]) <= fc.xmax && fminf(y[0], y[3]) >= 1.0f &&
                           fmaxf(y[0], y[3]) <= fc.ymax;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool inb = quad_in || (Z[j] > 0.0f && x[j] >= 1.0f && x[j] <= fc.xmax &&
                                     y[j] >= 1.0f && y[j] <= fc.ymax);
        // nearest pixel, (int)(x + 0.5) for x >= 1
        const int off =
            inb ? __float2int_rd(y[j] + 0.5f) * dpitch + __float2int_rd(x[j] + 0.5f) : 0;
        us[q].fv[j] = __ldg(depth + off);  // depth for now; f after the loads
        us[q].mask |= inb ? (1u << j) : 0u;
      }
    }
    // rule U decisions, then the voxel loads of every unit that updates
    T old[kUnitsInFlight][4];
    unsigned wq[kUnitsInFlight];
#pragma unroll
    for (int q = 0; q < kUnitsInFlight; ++q) {
      unsigned m = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float eta = (us[q].fv[j] - us[q].chi2) - us[q].lz[j];
        us[q].fv[j] = fminf(1.0f, eta * fc.inv_mu);
        m |= ((us[q].mask >> j) & 1u) && eta >= -fc.mu ? (1u << j) : 0u;
      }
      us[q].mask = m;
      if (m) {
        const int v0 = 4 * lane + 128 * us[q].k;
        const T* sdf_q = reinterpret_cast<const T*>(sv.sdf) + (size_t)us[q].ptr * kBlockVoxels + v0;
        if constexpr (S == TSDF_STORAGE_F32) {
          const float4 t = *reinterpret_cast<const float4*>(sdf_q);
          old[q][0] = t.x; old[q][1] = t.y; old[q][2] = t.z; old[q][3] = t.w;
        } else {
          const uint2 t = *reinterpret_cast<const uint2*>(sdf_q);
          memcpy(old[q], &t, sizeof(t));
        }
        wq[q] = *reinterpret_cast<const unsigned*>(sv.w + (size_t)us[q].ptr * kBlockVoxels + v0);
      }
    }
    // running averages and write-back
#pragma unroll
    for (int q = 0; q < kUnitsInFlight; ++q) {
      const unsigned m = us[q].mask;
      if (!m) continue;
      unsigned w = wq[q];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // computed for all four voxels, committed by select where updated
        const unsigned w0 = (w >> (8 * j)) & 0xffu;
        const float w0f = __uint_as_float(w0 | 0x4B000000u) - 8388608.0f;  // exact
        const float Fn = fmaf(w0f, St::load(old[q][j]), us[q].fv[j]) * s_rcp[w0];
        const unsigned wn = min(w0 + 1u, maxw);
        const bool b = (m >> j) & 1u;
        old[q][j] = b ? St::store(Fn) : old[q][j];
        w = b ? ((w & ~(0xffu << (8 * j))) | (wn << (8 * j))) : w;
      }
      const int v0 = 4 * lane + 128 * us[q].k;
      T* sdf_q = reinterpret_cast<T*>(sv.sdf) + (size_t)us[q].ptr * kBlockVoxels + v0;
      if constexpr (S == TSDF_STORAGE_F32) {
        *reinterpret_cast<float4*>(sdf_q) = make_float4(old[q][0], old[q][1], old[q][2], old[q][3]);
      } else {
        uint2 t;
        memcpy(&t, old[q], sizeof(t));
        *reinterpret_cast<uint2*>(sdf_q) = t;
      }
      *reinterpret_cast<unsigned*>(sv.w + (size_t)us[q].ptr * kBlockVoxels + v0) = w;
      updated += __popc(m);
    }
  }

  // one reduction per CTA, one (non-returning) atomic per CTA
#pragma unroll
  for (int off = 16; off; off >>= 1) updated += __shfl_xor_sync(0xffffffffu, updated, off);
  if (lane == 0) s_upd[threadIdx.x >> 5] = updated;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kIntWarps; ++w) t += s_upd[w];
    if (t) atomicAdd(&sv.fc->n_updated, t);
  }
}

// Zeroes the allocation-group counters after work that ran the allocation
// stages without the integration kernel (the resume path).
__global__ void finish_frame_kernel(SceneView sv) {
  FrameCounters* fr = sv.fc;
  fr->n_new = 0;
  fr->n_overflow = 0;
  fr->assign_base = 0;
  fr->depth_max_bits = 0u;
  fr->alloc_done = 0;
  for (int g = 0; g < kArriveGroups; ++g) fr->arrive[g] = 0;
}

template <int S, int U>
cudaError_t launch_integrate_su(const FrameConst& fc, const SceneView& sv, int sm_count,
                                cudaStream_t st) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrate_kernel<S, U>, kIntThreads, 0);
    if (per_sm < 1) per_sm = 1;
  }
  integrate_kernel<S, U><<<sm_count * per_sm, kIntThreads, 0, st>>>(fc, sv);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_integrate_s(const FrameConst& fc, const SceneView& sv, int sm_count, int units,
                               cudaStream_t st) {
  switch (units) {
    case 1: return launch_integrate_su<S, 1>(fc, sv, sm_count, st);
    case 4: return launch_integrate_su<S, 4>(fc, sv, sm_count, st);
    default: return launch_integrate_su<S, 2>(fc, sv, sm_count, st);
  }
}

}  // namespace

cudaError_t launch_visible(const FrameConst& fc, const SceneView& sv, int sm_count,
                           cudaStream_t st) {
  const int grid = sm_count * 2;
  switch (sv.storage) {
    case TSDF_STORAGE_F32: visible_kernel<TSDF_STORAGE_F32><<<grid, kVisThreads, 0, st>>>(fc, sv); break;
    case TSDF_STORAGE_I16: visible_kernel<TSDF_STORAGE_I16><<<grid, kVisThreads, 0, st>>>(fc, sv); break;
    default: visible_kernel<TSDF_STORAGE_F16><<<grid, kVisThreads, 0, st>>>(fc, sv); break;
  }
  return cudaGetLastError();
}

// Work units each warp of the integration kernel keeps in flight: 1, 2 or 4
// (TSDF_INTEGRATE_UNITS), default 2.
int integrate_units() {
  static int u = 0;
  if (!u) {
    const char* e = getenv("TSDF_INTEGRATE_UNITS");
    u = e ? atoi(e) : 2;
    if (u != 1 && u != 2 && u != 4) u = 2;
  }
  return u;
}

cudaError_t launch_integrate(const FrameConst& fc, const SceneView& sv, int sm_count,
                             cudaStream_t st) {
  const int u = integrate_units();
  switch (sv.storage) {
    case TSDF_STORAGE_F32: return launch_integrate_s<TSDF_STORAGE_F32>(fc, sv, sm_count, u, st);
    case TSDF_STORAGE_I16: return launch_integrate_s<TSDF_STORAGE_I16>(fc, sv, sm_count, u, st);
    default: return launch_integrate_s<TSDF_STORAGE_F16>(fc, sv, sm_count, u, st);
  }
}

cudaError_t launch_finish_frame(const SceneView& sv, cudaStream_t st) {
  finish_frame_kernel<<<1, 1, 0, st>>>(sv);
  return cudaGetLastError();
}

}  // namespace tsdf
