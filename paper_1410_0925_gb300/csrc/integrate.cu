// integrate.cu -- visible-block list (Section 4.2, third stage) and per-voxel
// integration (Section 4.3, computeUpdatedVoxelDepthInfo).
//
// visible_kernel  : scans the allocated blocks [0, high-water) (dense, as pool
//                   indices are handed out in order and never freed), keeps
//                   every block that can hold a voxel the integration rule
//                   would write, and compacts them with a CTA-level prefix sum
//                   (one atomic per CTA per pass).
// integrate_kernel: persistent; one warp per visible block, four consecutive
//                   voxels per lane and step (16 B of f32 sdf + 4 B of weights
//                   per lane, 512 B + 128 B per warp-step, fully coalesced).
//
// Arithmetic: FP32 throughout, no FP64. The camera-space block origin is
// carried as an unevaluated sum of two floats (hi + lo) built with exact
// product / sum transforms, so eta = d - z keeps ~1e-8 m accuracy at several
// metres of depth; the per-voxel offset A l is a plain float (|A l| < 0.1 m).
#include "tsdf_internal.cuh"

namespace tsdf {

namespace {

// ----------------------------------------------------------------------------
// visible list

constexpr int kVisThreads = 256;

__device__ __forceinline__ bool block_visible(const FrameConst& fc, unsigned long long key,
                                              float zfar) {
  int bx, by, bz;
  unpack_key(key, bx, by, bz);
  const float o[3] = {8.0f * bx, 8.0f * by, 8.0f * bz};
  float c0[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    c0[r] = fmaf(fc.A_hi[3 * r], o[0],
                 fmaf(fc.A_hi[3 * r + 1], o[1], fmaf(fc.A_hi[3 * r + 2], o[2], fc.t_hi[r])));
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
      const float x = fc.fx * X / Z + fc.cx, y = fc.fy * Y / Z + fc.cy;
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
  return true;
}

__global__ void __launch_bounds__(kVisThreads) visible_kernel(FrameConst fc, SceneView sv) {
  __shared__ int s_warp[kVisThreads / 32];
  __shared__ int s_base;
  const int high_water = sv.pool - __ldcg(&sv.sc->free_top);
  const float zfar = __uint_as_float(__ldcg(&sv.fc->depth_max_bits)) + fc.mu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool any_depth = __ldcg(&sv.fc->depth_max_bits) != 0u;
  for (int i0 = blockIdx.x * kVisThreads; i0 < high_water; i0 += gridDim.x * kVisThreads) {
    const int ptr = i0 + threadIdx.x;
    bool vis = false;
    if (ptr < high_water && any_depth) vis = block_visible(fc, sv.key_of_ptr[ptr], zfar);
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
    if (vis) sv.visible[s_base + s_warp[warp] + __popc(bal & ((1u << lane) - 1u))] = ptr;
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// integration

// error-free transforms (Knuth two-sum, FMA two-product)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

constexpr int kIntWarps = 4;

template <int S>
__global__ void __launch_bounds__(32 * kIntWarps) integrate_kernel(FrameConst fc, SceneView sv) {
  using St = Storage<S>;
  using T = typename St::T;
  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * kIntWarps + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * kIntWarps;
  const int n = __ldcg(&sv.fc->n_visible);

  // lane -> voxels 4*lane + 128*k + j (k = 0..3, j = 0..3)
  const float lx0 = (float)(4 * (lane & 1));
  const float ly = (float)((lane >> 1) & 7);
  const float lz0 = (float)(lane >> 4);
  const float maxw = (float)fc.max_weight;
  unsigned long long updated = 0;

  for (int i = gwarp; i < n; i += nwarps) {
    const int ptr = __ldcg(&sv.visible[i]);
    int bx, by, bz;
    unpack_key(__ldcg(&sv.key_of_ptr[ptr]), bx, by, bz);
    const float o[3] = {8.0f * bx, 8.0f * by, 8.0f * bz};  // exact (|o| < 2^19)
    // camera point of the block origin, c = A o + t, as hi + lo
    float chi[3], clo[3];
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

    T* sdf_blk = reinterpret_cast<T*>(sv.sdf) + (size_t)ptr * kBlockVoxels;
    unsigned* w_blk = reinterpret_cast<unsigned*>(sv.w + (size_t)ptr * kBlockVoxels);

#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const float lz = lz0 + 2.0f * k;
      // low part of the camera point of voxel (lx0, ly, lz)
      float lo[3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        lo[r] = fmaf(fc.A_hi[3 * r], lx0, fmaf(fc.A_hi[3 * r + 1], ly, fmaf(fc.A_hi[3 * r + 2], lz, clo[r])));
      float f[4];
      unsigned upd = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j) {
          lo[0] += fc.A_hi[0];
          lo[1] += fc.A_hi[3];
          lo[2] += fc.A_hi[6];
        }
        const float z = chi[2] + lo[2];
        f[j] = 0.0f;
        if (z > 0.0f) {
          const float rz = __frcp_rn(z);
          const float x = fmaf(fc.fx * (chi[0] + lo[0]), rz, fc.cx);
          const float y = fmaf(fc.fy * (chi[1] + lo[1]), rz, fc.cy);
          if (x >= 1.0f && x <= fc.xmax && y >= 1.0f && y <= fc.ymax) {
            const int ix = __float2int_rd(x + 0.5f), iy = __float2int_rd(y + 0.5f);
            const float d = __ldg(fc.depth + (long long)iy * fc.pitch + ix);
            if (d > 0.0f && d < INFINITY) {
              const float eta = (d - chi[2]) - lo[2];
              if (eta >= -fc.mu) {
                f[j] = fminf(1.0f, eta * fc.inv_mu);
                upd |= 1u << j;
              }
            }
          }
        }
      }
      if (upd) {
        const int v0 = 4 * lane + 128 * k;
        T old[4];
        if constexpr (S == TSDF_STORAGE_F32) {
          const float4 q = *reinterpret_cast<const float4*>(sdf_blk + v0);
          old[0] = q.x; old[1] = q.y; old[2] = q.z; old[3] = q.w;
        } else {
          const uint2 q = *reinterpret_cast<const uint2*>(sdf_blk + v0);
          memcpy(old, &q, sizeof(q));
        }
        unsigned wq = w_blk[v0 >> 2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (upd & (1u << j)) {
            const float w0 = (float)((wq >> (8 * j)) & 0xffu);
            const float F = St::load(old[j]);
            const float Fn = __fdiv_rn(fmaf(w0, F, f[j]), w0 + 1.0f);
            const unsigned wn = (unsigned)fminf(w0 + 1.0f, maxw);
            old[j] = St::store(Fn);
            wq = (wq & ~(0xffu << (8 * j))) | (wn << (8 * j));
          }
        }
        if constexpr (S == TSDF_STORAGE_F32) {
          *reinterpret_cast<float4*>(sdf_blk + v0) = make_float4(old[0], old[1], old[2], old[3]);
        } else {
          uint2 q;
          memcpy(&q, old, sizeof(q));
          *reinterpret_cast<uint2*>(sdf_blk + v0) = q;
        }
        w_blk[v0 >> 2] = wq;
        updated += __popc(upd);
      }
    }
  }

  // per-frame bookkeeping: the last warp to finish folds the counters
  for (int off = 16; off; off >>= 1) updated += __shfl_xor_sync(0xffffffffu, updated, off);
  if (lane == 0) {
    if (updated) atomicAdd(&sv.fc->n_updated, updated);
  }
}

__global__ void finish_frame_kernel(SceneView sv) {
  SceneCounters* sc = sv.sc;
  const FrameCounters* fr = sv.fc;
  sc->frames += 1;
  sc->last_new = (unsigned long long)fr->n_new;
  sc->last_visible = (unsigned long long)fr->n_visible;
  sc->last_updated = fr->n_updated;
  sc->total_updated += fr->n_updated;
  sc->total_visible += (unsigned long long)fr->n_visible;
}

}  // namespace

cudaError_t launch_visible(const FrameConst& fc, const SceneView& sv, int sm_count,
                           cudaStream_t st) {
  int grid = (sv.pool + kVisThreads - 1) / kVisThreads;
  if (grid > sm_count * 8) grid = sm_count * 8;
  visible_kernel<<<grid, kVisThreads, 0, st>>>(fc, sv);
  return cudaGetLastError();
}

cudaError_t launch_integrate(const FrameConst& fc, const SceneView& sv, int sm_count,
                             cudaStream_t st) {
  const int grid = sm_count * 16;
  switch (sv.storage) {
    case TSDF_STORAGE_F32:
      integrate_kernel<TSDF_STORAGE_F32><<<grid, 32 * kIntWarps, 0, st>>>(fc, sv);
      break;
    case TSDF_STORAGE_I16:
      integrate_kernel<TSDF_STORAGE_I16><<<grid, 32 * kIntWarps, 0, st>>>(fc, sv);
      break;
    default:
      integrate_kernel<TSDF_STORAGE_F16><<<grid, 32 * kIntWarps, 0, st>>>(fc, sv);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_finish_frame(const SceneView& sv, cudaStream_t st) {
  finish_frame_kernel<<<1, 1, 0, st>>>(sv);
  return cudaGetLastError();
}

}  // namespace tsdf
