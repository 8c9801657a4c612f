// readback.cu -- canonical readback, retrieval and resume.
//
// The result of fusion is the set of (block key, 512 sdf, 512 w); where a
// block sits in the pool or in the hash table depends on the order in which
// threads won atomics and is not part of the result. Readback therefore sorts
// the allocated blocks by their signed (x, y, z) block coordinate (bitonic
// sort over a power-of-two padded key array) and gathers them in that order.
#include "tsdf_internal.cuh"

namespace tsdf {

namespace {

__global__ void fill_sort_kernel(const unsigned long long* key_of_ptr, int n, int n2,
                                 unsigned long long* sk, int* sp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    if (i < n) {
      sk[i] = canonical_key(key_of_ptr[i]);
      sp[i] = i;
    } else {
      sk[i] = ~0ull;
      sp[i] = -1;
    }
  }
}

// one compare-exchange pass (j, k) of the bitonic network
__global__ void bitonic_pass_kernel(unsigned long long* sk, int* sp, int n2, int j, int k) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    const int l = i ^ j;
    if (l > i) {
      const unsigned long long a = sk[i], b = sk[l];
      const bool up = (i & k) == 0;
      if ((a > b) == up) {
        sk[i] = b;
        sk[l] = a;
        const int t = sp[i];
        sp[i] = sp[l];
        sp[l] = t;
      }
    }
  }
}

// Passes with j < 1024 of one k run inside a 2048-element shared-memory tile.
constexpr int kTile = 2048;
__global__ void __launch_bounds__(1024) bitonic_local_kernel(unsigned long long* sk, int* sp, int n2,
                                                             int k, int j_start) {
  __shared__ unsigned long long s_k[kTile];
  __shared__ int s_p[kTile];
  const int base = blockIdx.x * kTile;
  for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
    s_k[t] = sk[base + t];
    s_p[t] = sp[base + t];
  }
  __syncthreads();
  for (int j = j_start; j > 0; j >>= 1) {
    for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
      const int l = t ^ j;
      if (l > t) {
        const int gi = base + t;
        const bool up = (gi & k) == 0;
        const unsigned long long a = s_k[t], b = s_k[l];
        if ((a > b) == up) {
          s_k[t] = b;
          s_k[l] = a;
          const int x = s_p[t];
          s_p[t] = s_p[l];
          s_p[l] = x;
        }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
    sk[base + t] = s_k[t];
    sp[base + t] = s_p[t];
  }
}

template <typename T>
__global__ void gather_kernel(SceneView sv, const int* ptrs, int n, short* keys_out, T* sdf_out,
                              unsigned char* w_out) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = gwarp; b < n; b += nw) {
    const int ptr = ptrs[b];
    if (lane == 0 && keys_out) {
      int x, y, z;
      unpack_key(sv.key_of_ptr[ptr], x, y, z);
      keys_out[3 * b] = (short)x;
      keys_out[3 * b + 1] = (short)y;
      keys_out[3 * b + 2] = (short)z;
    }
    const T* src = reinterpret_cast<const T*>(sv.sdf) + (size_t)ptr * kBlockVoxels;
    // canonical voxel v lives at storage_voxel(v)
    if (sdf_out)
      for (int v = lane; v < kBlockVoxels; v += 32)
        sdf_out[(size_t)b * kBlockVoxels + v] = src[storage_voxel(v)];
    if (w_out) {
      const unsigned char* ws = sv.w + (size_t)ptr * kBlockVoxels;
      for (int v = lane; v < kBlockVoxels; v += 32)
        w_out[(size_t)b * kBlockVoxels + v] = ws[storage_voxel(v)];
    }
  }
}

__global__ void lookup_kernel(const unsigned long long* keys, int n, int* ptr_out, SceneView sv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = find_entry(sv, keys[i]);
    int p = e >= 0 ? sv.entries[e].ptr : -1;
    ptr_out[i] = p >= 0 ? p : -1;
  }
}

template <typename T>
__global__ void scatter_kernel(SceneView sv, const unsigned long long* keys, int n, const T* sdf_in,
                               const unsigned char* w_in) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = gwarp; b < n; b += nw) {
    const int e = find_entry(sv, keys[b]);
    const int ptr = e >= 0 ? sv.entries[e].ptr : -1;
    if (ptr < 0) continue;  // not allocated (capacity error already recorded)
    T* dst = reinterpret_cast<T*>(sv.sdf) + (size_t)ptr * kBlockVoxels;
    unsigned char* wd = sv.w + (size_t)ptr * kBlockVoxels;
    for (int v = lane; v < kBlockVoxels; v += 32) {
      dst[storage_voxel(v)] = sdf_in[(size_t)b * kBlockVoxels + v];
      wd[storage_voxel(v)] = w_in[(size_t)b * kBlockVoxels + v];
    }
  }
}

int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 65535) g = 65535;
  return (int)g;
}

}  // namespace

cudaError_t launch_sort_allocated(const SceneView& sv, int n, unsigned long long* sk, int* sp,
                                  int n2, cudaStream_t st) {
  fill_sort_kernel<<<grid_for(n2, 256), 256, 0, st>>>(sv.key_of_ptr, n, n2, sk, sp);
  for (int k = 2; k <= n2; k <<= 1) {
    int j = k >> 1;
    if (n2 >= kTile) {
      // partners i ^ j with j >= kTile live in different tiles: global passes
      for (; j >= kTile; j >>= 1)
        bitonic_pass_kernel<<<grid_for(n2, 256), 256, 0, st>>>(sk, sp, n2, j, k);
      bitonic_local_kernel<<<n2 / kTile, 1024, 0, st>>>(sk, sp, n2, k, j);
    } else {
      for (; j > 0; j >>= 1) bitonic_pass_kernel<<<grid_for(n2, 256), 256, 0, st>>>(sk, sp, n2, j, k);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_blocks(const SceneView& sv, const int* ptrs, int n, short* keys_out,
                                 void* sdf_out, unsigned char* w_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = grid_for((long long)n * 32, 256);
  if (sv.storage == TSDF_STORAGE_F32)
    gather_kernel<float><<<grid, 256, 0, st>>>(sv, ptrs, n, keys_out, (float*)sdf_out, w_out);
  else
    gather_kernel<unsigned short><<<grid, 256, 0, st>>>(sv, ptrs, n, keys_out,
                                                        (unsigned short*)sdf_out, w_out);
  return cudaGetLastError();
}

namespace {
// voxel colour words of blocks ptrs[0..n) in canonical voxel order
__global__ void gather_colour_kernel(SceneView sv, const int* ptrs, int n, unsigned* out) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = gwarp; b < n; b += nw) {
    const unsigned* src = sv.rgbw + (size_t)ptrs[b] * kBlockVoxels;
    for (int v = lane; v < kBlockVoxels; v += 32)
      out[(size_t)b * kBlockVoxels + v] = src[storage_voxel(v)];
  }
}
}  // namespace

cudaError_t launch_gather_colour(const SceneView& sv, const int* ptrs, int n, unsigned* out,
                                 cudaStream_t st) {
  if (n <= 0 || !sv.rgbw) return cudaSuccess;
  gather_colour_kernel<<<grid_for((long long)n * 32, 256), 256, 0, st>>>(sv, ptrs, n, out);
  return cudaGetLastError();
}

cudaError_t launch_lookup(const unsigned long long* keys, int n, int* ptr_out, const SceneView& sv,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  lookup_kernel<<<grid_for(n, 256), 256, 0, st>>>(keys, n, ptr_out, sv);
  return cudaGetLastError();
}

cudaError_t launch_scatter_blocks(const SceneView& sv, const unsigned long long* keys, int n,
                                  const void* sdf_in, const unsigned char* w_in, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = grid_for((long long)n * 32, 256);
  if (sv.storage == TSDF_STORAGE_F32)
    scatter_kernel<float><<<grid, 256, 0, st>>>(sv, keys, n, (const float*)sdf_in, w_in);
  else
    scatter_kernel<unsigned short><<<grid, 256, 0, st>>>(sv, keys, n, (const unsigned short*)sdf_in,
                                                         w_in);
  return cudaGetLastError();
}

}  // namespace tsdf
