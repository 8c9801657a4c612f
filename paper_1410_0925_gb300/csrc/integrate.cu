// integrate.cu -- visible-block list (Section 4.2, third stage) and per-voxel
// integration (Section 4.3, computeUpdatedVoxelDepthInfo).
//
// visible_kernel  : (a) initialises the voxels of the blocks the commit kernel
//                   handed out this frame (sdf 1, w 0); (b) scans the
//                   allocated blocks [0, high-water) (dense, as pool indices
//                   are handed out in order and never freed), keeps every
//                   block that can hold a voxel the integration rule would
//                   write, and compacts them with a CTA-level prefix sum (one
//                   atomic per CTA per pass). Each kept block's record carries
//                   the camera point of its origin voxel as a double-float.
// integrate_kernel: persistent; a visible block is split into 4/KQ work units
//                   of KQ quads (4 consecutive voxels) per lane, one warp per
//                   unit. All depth gathers of a unit are issued before any
//                   voxel data is touched; voxel data (16 B of f32 sdf + 4 B
//                   of weights per quad) is read and written only for quads
//                   the rule updates. The last warp to finish folds the
//                   frame's counters into the scene's and zeroes them for the
//                   next frame.
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

__device__ __forceinline__ bool block_visible(const FrameConst& fc, const unsigned* tile_max,
                                              const float c0[3], float zfar) {
  // Voxels of the block lie in the box spanned by lattice offsets 0..7; the
  // box's 8 corners bound every voxel's camera z and, when all are in front
  // of the camera, the voxels' image points (perspective keeps convexity).
  const float kSlackZ = 1e-3f, kSlackPx = 1.0f;
  float zmin = INFINITY, zmax = -INFINITY, xmin = INFINITY, xmax = -INFINITY,
        ymin = INFINITY, ymax = -INFINITY;
  bool front = true;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float lx = (c & 1) ? 7.0f : 0.0f, ly = (c & 2) ? 7.0f : 0.0f, lz = (c & 4) ? 7.0f : 0.0f;
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
    // ymax] (rounded, plus slack); if the block's nearest point is more than
    // mu behind the largest depth over that rectangle, rule U rejects every
    // voxel (eta < -mu). The largest depth comes from the coarsest-enough
    // level of the depth-max pyramid: at most 2 x 2 cells.
    const int px0 = max(0, (int)floorf(xmin - kSlackPx));
    const int px1 = min(fc.width - 1, (int)ceilf(xmax + kSlackPx));
    const int py0 = max(0, (int)floorf(ymin - kSlackPx));
    const int py1 = min(fc.height - 1, (int)ceilf(ymax + kSlackPx));
    int l = 0;
    while (l < kPyramidLevels - 1 && (((px1 >> (4 + l)) - (px0 >> (4 + l))) > 1 ||
                                      ((py1 >> (4 + l)) - (py0 >> (4 + l))) > 1))
      ++l;
    int wl, hl;
    const int off = pyramid_level(fc.tiles_x, fc.tiles_y, l, wl, hl);
    const int cx0 = px0 >> (4 + l), cx1 = px1 >> (4 + l);
    const int cy0 = py0 >> (4 + l), cy1 = py1 >> (4 + l);
    const unsigned m = max(max(__ldcg(&tile_max[off + cy0 * wl + cx0]), __ldcg(&tile_max[off + cy0 * wl + cx1])),
                           max(__ldcg(&tile_max[off + cy1 * wl + cx0]), __ldcg(&tile_max[off + cy1 * wl + cx1])));
    if (zmin > __uint_as_float(m) + fc.mu + kSlackZ) return false;
  }
  return true;
}

constexpr int kVisPerThread = 4;  // allocated blocks tested per thread and pass

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
    for (int i = gw; i < n_new; i += nw) {
      const int ptr = __ldcg(&sv.free_stack[base - 1 - i]);
      T* sdf = reinterpret_cast<T*>(sv.sdf) + (size_t)ptr * kBlockVoxels;
#pragma unroll
      for (int j = 0; j < kBlockVoxels / 32; ++j) sdf[32 * j + lane] = init;
      reinterpret_cast<uint4*>(sv.w + (size_t)ptr * kBlockVoxels)[lane] = make_uint4(0, 0, 0, 0);
    }
  }

  // (b) scan and compact: kVisPerThread blocks per thread and pass, one
  // global atomic per CTA and pass
  const int high_water = sv.pool - __ldcg(&sv.sc->free_top);
  const unsigned dmax_bits = __ldcg(&sv.fc->depth_max_bits);
  const float zfar = __uint_as_float(dmax_bits) + fc.mu;
  constexpr int kPass = kVisThreads * kVisPerThread;
  for (int i0 = blockIdx.x * kPass; i0 < high_water; i0 += gridDim.x * kPass) {
    unsigned long long keys[kVisPerThread];
#pragma unroll
    for (int q = 0; q < kVisPerThread; ++q) {
      const int ptr = i0 + q * kVisThreads + threadIdx.x;
      keys[q] = ptr < high_water ? __ldg(&sv.key_of_ptr[ptr]) : kKeyEmpty;
    }
    unsigned vis = 0;
#pragma unroll
    for (int q = 0; q < kVisPerThread; ++q) {
      if (keys[q] == kKeyEmpty || dmax_bits == 0u) continue;
      int bx, by, bz;
      unpack_key(keys[q], bx, by, bz);
      const float o[3] = {8.0f * bx, 8.0f * by, 8.0f * bz};
      float c0[3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        c0[r] = fmaf(fc.A_hi[3 * r], o[0],
                     fmaf(fc.A_hi[3 * r + 1], o[1], fmaf(fc.A_hi[3 * r + 2], o[2], fc.t_hi[r])));
      if (block_visible(fc, sv.tile_max, c0, zfar)) vis |= 1u << q;
    }
    // exclusive prefix of the per-thread counts over the CTA
    const int cnt = __popc(vis);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
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
    int pos = s_base + s_warp[warp] + incl - cnt;
#pragma unroll
    for (int q = 0; q < kVisPerThread; ++q) {
      if (!(vis & (1u << q))) continue;
      int bx, by, bz;
      unpack_key(keys[q], bx, by, bz);
      const float o[3] = {8.0f * bx, 8.0f * by, 8.0f * bz};
      VisRec r;
      r.ptr = i0 + q * kVisThreads + threadIdx.x;
      origin_df(fc, o, r.chi, r.clo);
      r.pad = 0;
      sv.visible[pos++] = r;
    }
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

// KQ: quads (of 4 voxels) per lane per work unit; a block is 4 / KQ units,
// each taken by one warp. Larger KQ keeps more loads in flight per warp,
// smaller KQ needs fewer registers (more warps per SM).
template <int S, int KQ>
__global__ void __launch_bounds__(kIntThreads) integrate_kernel(FrameConst fc, SceneView sv) {
  static_assert(KQ == 1 || KQ == 2 || KQ == 4, "KQ must divide 4");
  constexpr int kUnits = 4 / KQ;
  using St = Storage<S>;
  using T = typename St::T;
  __shared__ float s_rcp[256];  // s_rcp[w] = 1 / (w + 1), rounded once
  s_rcp[threadIdx.x] = 1.0f / (float)(threadIdx.x + 1);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * kIntWarps + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * kIntWarps;
  const int n_units = __ldcg(&sv.fc->n_visible) * kUnits;

  // lane -> voxels 4*lane + 128*k + j (k, j = 0..3):
  // lx = 4 (lane & 1) + j, ly = (lane >> 1) & 7, lz = (lane >> 4) + 2 k
  const float lx0 = (float)(4 * (lane & 1));
  const float ly = (float)((lane >> 1) & 7);
  const float lz0 = (float)(lane >> 4);
  float lbase[3], dk[3], dj[3];  // A l of the lane's first voxel; steps in z (2) and x (1)
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    lbase[r] = fmaf(fc.A_hi[3 * r], lx0, fmaf(fc.A_hi[3 * r + 1], ly, fc.A_hi[3 * r + 2] * lz0));
    dk[r] = 2.0f * fc.A_hi[3 * r + 2];
    dj[r] = fc.A_hi[3 * r];
  }
  const unsigned maxw = (unsigned)fc.max_weight;
  unsigned long long updated = 0;

  // image-plane steps of one voxel along x: fx * A[0][0], fy * A[1][0]
  const float pdx = fc.fx * dj[0], pdy = fc.fy * dj[1];

  for (int u = gwarp; u < n_units; u += nwarps) {
    const int kq0 = (u % kUnits) * KQ;  // first quad of this unit
    const VisRec vr = sv.visible[u / kUnits];
    float fv[4 * KQ];
    unsigned mask = 0;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const float kk = (float)(kq0 + q);
      // camera point of the quad's first voxel: hi + lo per coordinate; x
      // and y are only needed to float accuracy, z keeps its low part for eta
      float lz = vr.clo[2] + fmaf(kk, dk[2], lbase[2]);
      float px = fc.fx * (vr.chi[0] + (vr.clo[0] + fmaf(kk, dk[0], lbase[0])));
      float py = fc.fy * (vr.chi[1] + (vr.clo[1] + fmaf(kk, dk[1], lbase[1])));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j) {
          px += pdx;
          py += pdy;
          lz += dj[2];
        }
        const float Z = vr.chi[2] + lz;
        const float rz = rcp_approx(Z);
        const float x = fmaf(px, rz, fc.cx);
        const float y = fmaf(py, rz, fc.cy);
        const bool inb = Z > 0.0f && x >= 1.0f && x <= fc.xmax && y >= 1.0f && y <= fc.ymax;
        // nearest pixel, (int)(x + 0.5) for x >= 1
        const int off = inb ? __float2int_rd(y + 0.5f) * fc.pitch + __float2int_rd(x + 0.5f) : 0;
        const float d = __ldg(fc.depth + off);
        const float eta = (d - vr.chi[2]) - lz;
        const bool ok = inb && d > 0.0f && d < INFINITY && eta >= -fc.mu;
        fv[4 * q + j] = fminf(1.0f, eta * fc.inv_mu);
        mask |= (ok ? 1u : 0u) << (4 * q + j);
      }
    }
    if (!mask) continue;
    T* sdf_blk = reinterpret_cast<T*>(sv.sdf) + (size_t)vr.ptr * kBlockVoxels;
    unsigned* w_blk = reinterpret_cast<unsigned*>(sv.w + (size_t)vr.ptr * kBlockVoxels);
    // issue every needed quad load before using any of them
    T old[KQ][4];
    unsigned wq[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      if ((mask >> (4 * q)) & 0xfu) {
        const int v0 = 4 * lane + 128 * (kq0 + q);
        if constexpr (S == TSDF_STORAGE_F32) {
          const float4 t = *reinterpret_cast<const float4*>(sdf_blk + v0);
          old[q][0] = t.x; old[q][1] = t.y; old[q][2] = t.z; old[q][3] = t.w;
        } else {
          const uint2 t = *reinterpret_cast<const uint2*>(sdf_blk + v0);
          memcpy(old[q], &t, sizeof(t));
        }
        wq[q] = w_blk[v0 >> 2];
      }
    }
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const unsigned m = (mask >> (4 * q)) & 0xfu;
      if (!m) continue;
      unsigned wqk = wq[q];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // computed for all four voxels, committed by select where updated
        const unsigned w0 = (wqk >> (8 * j)) & 0xffu;
        const float w0f = __uint_as_float(w0 | 0x4B000000u) - 8388608.0f;  // exact
        const float Fn = fmaf(w0f, St::load(old[q][j]), fv[4 * q + j]) * s_rcp[w0];
        const unsigned wn = min(w0 + 1u, maxw);
        const bool b = (m >> j) & 1u;
        old[q][j] = b ? St::store(Fn) : old[q][j];
        wqk = b ? ((wqk & ~(0xffu << (8 * j))) | (wn << (8 * j))) : wqk;
      }
      const int v0 = 4 * lane + 128 * (kq0 + q);
      if constexpr (S == TSDF_STORAGE_F32) {
        *reinterpret_cast<float4*>(sdf_blk + v0) =
            make_float4(old[q][0], old[q][1], old[q][2], old[q][3]);
      } else {
        uint2 t;
        memcpy(&t, old[q], sizeof(t));
        *reinterpret_cast<uint2*>(sdf_blk + v0) = t;
      }
      w_blk[v0 >> 2] = wqk;
    }
    updated += __popc(mask);
  }

  // per-frame bookkeeping: the last warp to finish folds the counters into
  // the scene's and zeroes them for the next frame
#pragma unroll
  for (int off = 16; off; off >>= 1) updated += __shfl_xor_sync(0xffffffffu, updated, off);
  int last = 0;
  if (lane == 0) {
    if (updated) atomicAdd(&sv.fc->n_updated, updated);
    __threadfence();
    last = atomicAdd(&sv.fc->warps_done, 1) == nwarps - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence();
    if (fc.use_tiles) {
      // coarser pyramid levels accumulate by atomicMax: zero them
      int wl, hl;
      const int lo = fc.tiles_x * fc.tiles_y;
      const int hi = pyramid_level(fc.tiles_x, fc.tiles_y, kPyramidLevels, wl, hl);
      for (int i = lo + lane; i < hi; i += 32) sv.tile_max[i] = 0u;
    }
    if (lane == 0) {
      FrameCounters* fr = sv.fc;
      SceneCounters* sc = sv.sc;
      const unsigned long long upd = atomicAdd(&fr->n_updated, 0ull);
      const int nv = atomicAdd(&fr->n_visible, 0);
      const int nn = atomicAdd(&fr->n_new, 0);
      sc->frames += 1;
      sc->last_new = (unsigned long long)nn;
      sc->last_visible = (unsigned long long)nv;
      sc->last_updated = upd;
      sc->total_updated += upd;
      sc->total_visible += (unsigned long long)nv;
      FrameCounters z{};
      *fr = z;
    }
  }
}

// Zeroes the frame counters after work that ran the allocation stages
// without the integration kernel (the resume path).
__global__ void finish_frame_kernel(SceneView sv) {
  FrameCounters z{};
  *sv.fc = z;
}

template <int S, int KQ>
int integrate_blocks_per_sm() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, integrate_kernel<S, KQ>, kIntThreads, 0);
  return b > 0 ? b : 1;
}

template <int S, int KQ>
cudaError_t launch_integrate_kq(const FrameConst& fc, const SceneView& sv, int sm_count,
                                cudaStream_t st) {
  static int per_sm = 0;
  if (!per_sm) per_sm = integrate_blocks_per_sm<S, KQ>();
  integrate_kernel<S, KQ><<<sm_count * per_sm, kIntThreads, 0, st>>>(fc, sv);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_integrate_s(const FrameConst& fc, const SceneView& sv, int sm_count, int kq,
                               cudaStream_t st) {
  switch (kq) {
    case 1: return launch_integrate_kq<S, 1>(fc, sv, sm_count, st);
    case 4: return launch_integrate_kq<S, 4>(fc, sv, sm_count, st);
    default: return launch_integrate_kq<S, 2>(fc, sv, sm_count, st);
  }
}

}  // namespace

cudaError_t launch_visible(const FrameConst& fc, const SceneView& sv, int sm_count,
                           cudaStream_t st) {
  int grid = (sv.pool + kVisThreads * kVisPerThread - 1) / (kVisThreads * kVisPerThread);
  if (grid > sm_count * 2) grid = sm_count * 2;
  switch (sv.storage) {
    case TSDF_STORAGE_F32: visible_kernel<TSDF_STORAGE_F32><<<grid, kVisThreads, 0, st>>>(fc, sv); break;
    case TSDF_STORAGE_I16: visible_kernel<TSDF_STORAGE_I16><<<grid, kVisThreads, 0, st>>>(fc, sv); break;
    default: visible_kernel<TSDF_STORAGE_F16><<<grid, kVisThreads, 0, st>>>(fc, sv); break;
  }
  return cudaGetLastError();
}

// Quads per lane of the integration kernel: TSDF_INTEGRATE_KQ (1, 2 or 4) if
// set, else 1 (fastest measured on GB300 for 640x480 / 5 mm frames).
int integrate_kq() {
  static int kq = 0;
  if (!kq) {
    const char* e = getenv("TSDF_INTEGRATE_KQ");
    kq = e ? atoi(e) : 1;
    if (kq != 1 && kq != 2 && kq != 4) kq = 1;
  }
  return kq;
}

cudaError_t launch_integrate(const FrameConst& fc, const SceneView& sv, int sm_count,
                             cudaStream_t st) {
  const int kq = integrate_kq();
  switch (sv.storage) {
    case TSDF_STORAGE_F32: return launch_integrate_s<TSDF_STORAGE_F32>(fc, sv, sm_count, kq, st);
    case TSDF_STORAGE_I16: return launch_integrate_s<TSDF_STORAGE_I16>(fc, sv, sm_count, kq, st);
    default: return launch_integrate_s<TSDF_STORAGE_F16>(fc, sv, sm_count, kq, st);
  }
}

cudaError_t launch_finish_frame(const SceneView& sv, cudaStream_t st) {
  finish_frame_kernel<<<1, 1, 0, st>>>(sv);
  return cudaGetLastError();
}

}  // namespace tsdf
