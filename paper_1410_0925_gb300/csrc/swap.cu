// swap.cu -- swapping (Section 5): only the part of the map in or near the
// view stays in device memory; the rest lives in a host voxel block array
// with one slot per hash entry, so a hash entry index is all it takes to
// find a block's host copy.
//
// GB300 form: the host array is pinned, mapped host memory that the kernels
// read and write directly over the chip-to-chip link, so no transfer buffer
// is staged and no host code runs per block; a call still moves at most
// `transfer_blocks` blocks (the fixed bound of the report's transfer
// buffers). Every call is a fixed sequence of stream-ordered launches with
// no host synchronisation, so it can be captured in a CUDA graph.
//
//   tsdf_swap_out: device blocks that are not visible and have no pending
//     host copy are copied to the host array; their hash entries keep the key
//     but lose the pool block (kPtrUnallocated), so a later band meeting one
//     allocates a fresh block through the ordinary allocation stage. The
//     freed pool blocks are filled by moving the last used blocks into them,
//     which keeps the pool's used part dense and its bump allocation valid.
//   tsdf_swap_in: host blocks that the allocation stage gave a fresh device
//     block are merged into it (secondary integration); host blocks that are
//     visible are copied into new pool blocks if the pool has room for a
//     full call.
//   Both calls select the candidates with the smallest (x, y, z) keys when
//   there are more than transfer_blocks (radix selection of the threshold
//   key, six 8-bit digit passes).
//
// Visibility (the rule of the oracle, evaluated in FP64): a block is visible
// when some corner of its box is in front of the camera and either some
// corner is not, or the bounding box of its projected corners meets the
// image rectangle grown by the margin (and its nearest corner is within the
// depth limit). Each test is a linear function of the corner, so its extreme
// over the eight corners is the value at the block origin plus a per-call
// constant: five dot products per block, no division.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "scene_impl.h"

namespace tsdf {

namespace {

constexpr int kSwapThreads = 256;
constexpr int kSwapWarps = kSwapThreads / 32;

struct __align__(16) SwapCand {
  unsigned long long ckey;  // canonical key (selection order)
  int ptr;                  // pool block, or kPtrUnallocated (swap-in only)
  int entry;                // hash entry
};

// Per call; zeroed by the call's first operation.
struct SwapCounters {
  int n_cand;
  int hw0;      // used pool blocks when the call started
  int free0;    // free pool blocks when the call started
  int n_moved;  // blocks swapped out / in
  int n_pairs;  // pool compaction moves
  int n_alloc;  // swap-in: new pool blocks
  int n_merged;
  int need;     // radix selection: rank still sought among the prefix's keys
  int ticket;
  int compact_failed;
  int pad[2];
  unsigned long long prefix;  // radix selection: the threshold's digits so far
  unsigned hist[256];
};

// Persistent per scene.
struct SwapTotals {
  long long host_blocks;
  long long total_out, total_in, total_merged;
  long long last_out_candidates, last_out, last_in_candidates, last_in, last_merged;
};

// Per-call constants: for each of five linear functions f(p) = g . p + h of
// a world point (camera z, and the four image-edge tests), its extremes over
// a block's corners are f(origin) + ext_max / ext_min.
struct SwapConst {
  double g[5][3];
  double h[5];
  double ext_max[5], ext_min[5];
  double voxel_size;
  double max_depth;  // <= 0: no depth limit
  int capacity;
  int max_weight;
};

struct SwapDev {
  unsigned char* state;      // per hash entry: 1 = a host copy exists
  SwapCand* cand;
  int cand_cap;
  unsigned char* freed;      // per pool block (swap-out)
  int* freed_list;           // capacity
  int2* pairs;               // capacity: (hole, mover)
  SwapCounters* ctr;
  SwapTotals* totals;
  unsigned char* host;       // device view of the host voxel block array
  long long block_bytes;
  int n_entries;
  int sdf_bytes;             // 512 x element size
};

// (also compiled for the host: tsdf_swap_visibility runs the same code)
__host__ __device__ bool swap_visible(const SwapConst& k, unsigned long long key) {
  int b[3];
  unpack_key(key, b[0], b[1], b[2]);
  double p[3];
  for (int a = 0; a < 3; ++a) p[a] = (8.0 * (double)b[a]) * k.voxel_size;
  double f[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) f[i] = k.g[i][0] * p[0] + k.g[i][1] * p[1] + k.g[i][2] * p[2] + k.h[i];
  const double zmax = f[0] + k.ext_max[0], zmin = f[0] + k.ext_min[0];
  if (zmax <= 0.0) return false;  // every corner behind the camera
  if (zmin <= 0.0) return true;   // the block straddles the camera plane
  return f[1] + k.ext_max[1] >= 0.0 && f[2] + k.ext_min[2] <= 0.0 &&
         f[3] + k.ext_max[3] >= 0.0 && f[4] + k.ext_min[4] <= 0.0 &&
         (k.max_depth <= 0.0 || zmin <= k.max_depth);
}

__device__ __forceinline__ void append_cand(const SwapDev& d, unsigned long long key, int ptr,
                                            int entry) {
  const int i = atomicAdd(&d.ctr->n_cand, 1);
  if (i < d.cand_cap) {
    SwapCand c;
    c.ckey = canonical_key(key);
    c.ptr = ptr;
    c.entry = entry;
    d.cand[i] = c;
  }
}

// Swap-out candidates: used pool blocks that are not visible and have no
// pending host copy.
__global__ void __launch_bounds__(kSwapThreads) swap_out_select_kernel(SwapConst k, SceneView sv,
                                                                       SwapDev d) {
  const int free_top = __ldcg(&sv.sc->free_top);
  const int hw = sv.pool - free_top;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctr->hw0 = hw;
    d.ctr->free0 = free_top;
  }
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < hw; p += gridDim.x * blockDim.x) {
    const unsigned long long key = __ldcg(&sv.key_of_ptr[p]);
    if (swap_visible(k, key)) continue;
    const int e = find_entry(sv, key);
    if (e < 0 || __ldcg(&sv.entries[e].ptr) != p) {
      set_status(sv.sc, kStInternal);
      continue;
    }
    if (d.state[e]) continue;  // merged by a swap-in first
    append_cand(d, key, p, e);
  }
}

// Swap-in candidates: hash entries with a host copy that either have a
// fresh pool block (given by the allocation stage) or are visible while the
// pool has room for a full call.
__global__ void __launch_bounds__(kSwapThreads) swap_in_select_kernel(SwapConst k, SceneView sv,
                                                                      SwapDev d) {
  const int free_top = __ldcg(&sv.sc->free_top);
  const bool prefetch = free_top >= k.capacity;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctr->hw0 = sv.pool - free_top;
    d.ctr->free0 = free_top;
  }
  const int used = min(d.n_entries, sv.n_bucket_entries + min(__ldcg(&sv.sc->excess_top), sv.excess_cap));
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < used; e += gridDim.x * blockDim.x) {
    if (!d.state[e]) continue;
    const unsigned long long key = __ldcg(&sv.entries[e].key);
    const int ptr = __ldcg(&sv.entries[e].ptr);
    if (ptr >= 0 || (ptr == kPtrUnallocated && prefetch && swap_visible(k, key)))
      append_cand(d, key, ptr, e);
  }
}

// One pass of the radix selection of the capacity-th smallest candidate key
// (pass 0 = bits 40..47, ..., pass 5 = bits 0..7). Each CTA builds a digit
// histogram of the candidates that match the digits found so far; the last
// CTA to finish picks the digit holding the sought rank. Nothing to do when
// every candidate fits.
__global__ void __launch_bounds__(kSwapThreads) swap_radix_kernel(SwapDev d, int capacity, int pass) {
  const int n = min(__ldcg(&d.ctr->n_cand), d.cand_cap);
  if (n <= capacity) return;
  __shared__ unsigned h[256];
  __shared__ bool last;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int shift = 40 - 8 * pass;
  const unsigned long long prefix = __ldcg(&d.ctr->prefix);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long c = d.cand[i].ckey;
    if (pass == 0 || (c >> (shift + 8)) == (prefix >> (shift + 8)))
      atomicAdd(&h[(c >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&d.ctr->hist[i], h[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&d.ctr->ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    const unsigned need = pass == 0 ? (unsigned)capacity : (unsigned)__ldcg(&d.ctr->need);
    unsigned cum = 0;
    int g = 255;
    for (int b = 0; b < 256; ++b) {
      const unsigned c = __ldcg(&d.ctr->hist[b]);
      if (cum + c >= need) {
        g = b;
        break;
      }
      cum += c;
    }
    d.ctr->prefix = prefix | ((unsigned long long)g << shift);
    d.ctr->need = (int)(need - cum);
    d.ctr->ticket = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) d.ctr->hist[i] = 0;
}

__device__ __forceinline__ bool selected(const SwapDev& d, const SwapCand& c, int n, int capacity) {
  return n <= capacity || c.ckey <= __ldcg(&d.ctr->prefix);
}

// 16-byte copies of `bytes` (a multiple of 16) by the lanes of one warp.
__device__ __forceinline__ void warp_copy(void* dst, const void* src, int bytes, int lane) {
  uint4* o = reinterpret_cast<uint4*>(dst);
  const uint4* in = reinterpret_cast<const uint4*>(src);
  for (int i = lane; i < bytes / 16; i += 32) o[i] = in[i];
}

__device__ __forceinline__ unsigned char* dev_sdf(const SceneView& sv, const SwapDev& d, int ptr) {
  return reinterpret_cast<unsigned char*>(sv.sdf) + (size_t)ptr * d.sdf_bytes;
}

// Copy the selected blocks to the host array, one warp per block, and
// release their pool blocks.
__global__ void __launch_bounds__(kSwapThreads) swap_out_copy_kernel(SceneView sv, SwapDev d,
                                                                     int capacity) {
  const int n = min(__ldcg(&d.ctr->n_cand), d.cand_cap);
  const int lane = threadIdx.x & 31;
  const int n_warps = gridDim.x * kSwapWarps;
  for (int i = blockIdx.x * kSwapWarps + (threadIdx.x >> 5); i < n; i += n_warps) {
    const SwapCand c = d.cand[i];
    if (!selected(d, c, n, capacity)) continue;
    if (c.ptr < 0 || c.ptr >= sv.pool || c.entry < 0 || c.entry >= d.n_entries) {
      if (lane == 0) set_status(sv.sc, kStInternal);
      continue;
    }
    unsigned char* host = d.host + (size_t)c.entry * d.block_bytes;
    warp_copy(host, dev_sdf(sv, d, c.ptr), d.sdf_bytes, lane);
    warp_copy(host + d.sdf_bytes, sv.w + (size_t)c.ptr * kBlockVoxels, kBlockVoxels, lane);
    if (sv.rgbw)
      warp_copy(host + d.sdf_bytes + kBlockVoxels, sv.rgbw + (size_t)c.ptr * kBlockVoxels,
                kBlockVoxels * 4, lane);
    __syncwarp();
    if (lane == 0) {
      d.state[c.entry] = 1;
      sv.entries[c.entry].ptr = kPtrUnallocated;
      d.freed[c.ptr] = 1;
      const int j = atomicAdd(&d.ctr->n_moved, 1);
      if (j < capacity) d.freed_list[j] = c.ptr;
      else set_status(sv.sc, kStInternal);
    }
  }
}

// Pool compaction (one CTA): the k freed blocks leave holes; the used blocks
// among the last k positions move into the holes below them, so that the
// used part becomes [0, hw - k) again.
__global__ void __launch_bounds__(1024) swap_compact_kernel(SwapDev d, int capacity) {
  __shared__ int n_holes, n_movers;
  if (threadIdx.x == 0) n_holes = n_movers = 0;
  __syncthreads();
  const int hw = d.ctr->hw0;
  const int k = min(d.ctr->n_moved, capacity);
  const int lo = hw - k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const int q = lo + j;  // the tail position j
    if (q >= 0 && !d.freed[q]) d.pairs[atomicAdd(&n_movers, 1)].y = q;
    const int p = d.freed_list[j];
    if (p < lo) d.pairs[atomicAdd(&n_holes, 1)].x = p;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) d.freed[d.freed_list[j]] = 0;
  if (threadIdx.x == 0) {
    // equal by construction (every freed block lies below hw)
    const bool ok = n_holes == n_movers;
    d.ctr->n_pairs = ok ? n_holes : 0;
    d.ctr->compact_failed = !ok;
  }
}

// Move each (hole, mover) pair's block, one warp per pair, and repoint its
// hash entry.
__global__ void __launch_bounds__(kSwapThreads) swap_move_kernel(SceneView sv, SwapDev d) {
  const int n = __ldcg(&d.ctr->n_pairs);
  const int lane = threadIdx.x & 31;
  const int n_warps = gridDim.x * kSwapWarps;
  for (int j = blockIdx.x * kSwapWarps + (threadIdx.x >> 5); j < n; j += n_warps) {
    const int2 pr = d.pairs[j];
    const int hole = pr.x, mover = pr.y;
    if (hole < 0 || hole >= sv.pool || mover < 0 || mover >= sv.pool || hole >= mover) {
      if (lane == 0) set_status(sv.sc, kStInternal);
      continue;
    }
    warp_copy(dev_sdf(sv, d, hole), dev_sdf(sv, d, mover), d.sdf_bytes, lane);
    warp_copy(sv.w + (size_t)hole * kBlockVoxels, sv.w + (size_t)mover * kBlockVoxels,
              kBlockVoxels, lane);
    if (sv.rgbw)
      warp_copy(sv.rgbw + (size_t)hole * kBlockVoxels, sv.rgbw + (size_t)mover * kBlockVoxels,
                kBlockVoxels * 4, lane);
    if (lane == 0) {
      const unsigned long long key = sv.key_of_ptr[mover];
      sv.key_of_ptr[hole] = key;
      const int e = find_entry(sv, key);
      if (e >= 0) sv.entries[e].ptr = hole;
      else set_status(sv.sc, kStInternal);
    }
  }
}

// Secondary integration of one voxel (host h into device d), on its stored
// form: an empty side (weight 0) yields the other; else the weighted mean of
// the two averages and the capped sum of the weights. int16 averages the
// stored integers exactly (C division truncates toward zero); FP16 takes
// the FP32 mean rounded to nearest even. Host and device run this code
// (tsdf_swap_merge_voxels is the host entry).
__host__ __device__ __forceinline__ int merged_weight(int wh, int wd, int maxw) {
  return wh + wd < maxw ? wh + wd : maxw;
}
__host__ __device__ __forceinline__ float merge_value(float fh, int wh, float fd, int wd) {
  return fmaf((float)wh, fh, (float)wd * fd) / (float)(wh + wd);
}
__host__ __device__ __forceinline__ void merge_f32(float fh, int wh, float& fd, int& wd, int maxw) {
  if (wh == 0) return;
  if (wd == 0) {
    fd = fh;
    wd = wh;
    return;
  }
  fd = merge_value(fh, wh, fd, wd);
  wd = merged_weight(wh, wd, maxw);
}
__host__ __device__ __forceinline__ void merge_i16(unsigned short qh, int wh, unsigned short& qd,
                                                   int& wd, int maxw) {
  if (wh == 0) return;
  if (wd == 0) {
    qd = qh;
    wd = wh;
    return;
  }
  const int num = wh * (int)(short)qh + wd * (int)(short)qd;
  qd = (unsigned short)(short)(num / (wh + wd));
  wd = merged_weight(wh, wd, maxw);
}
__host__ __device__ __forceinline__ void merge_f16(unsigned short hh, int wh, unsigned short& hd,
                                                   int& wd, int maxw) {
  if (wh == 0) return;
  if (wd == 0) {
    hd = hh;
    wd = wh;
    return;
  }
  const float fh = __half2float(__ushort_as_half(hh));
  const float fd = __half2float(__ushort_as_half(hd));
  hd = __half_as_ushort(__float2half_rn(merge_value(fh, wh, fd, wd)));
  wd = merged_weight(wh, wd, maxw);
}
// colour words: bytes r, g, b, colour weight
__host__ __device__ __forceinline__ unsigned merge_colour(unsigned h, unsigned dv, int maxw) {
  const int wh = h >> 24, wd = dv >> 24;
  if (wh == 0) return dv;
  if (wd == 0) return h;
  const int w = wh + wd;
  unsigned out = (unsigned)merged_weight(wh, wd, maxw) << 24;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int num = wh * (int)((h >> (8 * c)) & 255u) + wd * (int)((dv >> (8 * c)) & 255u);
    out |= (unsigned)((2 * num + w) / (2 * w)) << (8 * c);
  }
  return out;
}

template <int S>
__device__ void merge_block(const SwapConst& k, const SceneView& sv, const SwapDev& d,
                            const unsigned char* host, int ptr, int lane) {
  // a lane takes quads of four consecutive voxels (one weight word)
  const unsigned* hw_ = reinterpret_cast<const unsigned*>(host + d.sdf_bytes);
  unsigned* dw = reinterpret_cast<unsigned*>(sv.w + (size_t)ptr * kBlockVoxels);
  for (int q = lane; q < kBlockVoxels / 4; q += 32) {
    const unsigned wh4 = hw_[q], wd4 = dw[q];
    unsigned wo4 = 0;
    if (S == 0) {
      const float4 fh = reinterpret_cast<const float4*>(host)[q];
      float4* dp = reinterpret_cast<float4*>(dev_sdf(sv, d, ptr)) + q;
      float4 fd = *dp;
      float* a = &fd.x;
      const float* b = &fh.x;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int w = (wd4 >> (8 * v)) & 255;
        merge_f32(b[v], (wh4 >> (8 * v)) & 255, a[v], w, k.max_weight);
        wo4 |= (unsigned)w << (8 * v);
      }
      *dp = fd;
    } else {
      const uint2 hh = reinterpret_cast<const uint2*>(host)[q];
      uint2* dp = reinterpret_cast<uint2*>(dev_sdf(sv, d, ptr)) + q;
      uint2 dd = *dp;
      const unsigned short hs[4] = {(unsigned short)(hh.x & 0xffffu), (unsigned short)(hh.x >> 16),
                                    (unsigned short)(hh.y & 0xffffu), (unsigned short)(hh.y >> 16)};
      unsigned short ds[4] = {(unsigned short)(dd.x & 0xffffu), (unsigned short)(dd.x >> 16),
                              (unsigned short)(dd.y & 0xffffu), (unsigned short)(dd.y >> 16)};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int w = (wd4 >> (8 * v)) & 255;
        const int wh = (wh4 >> (8 * v)) & 255;
        if (S == 1) merge_i16(hs[v], wh, ds[v], w, k.max_weight);
        else merge_f16(hs[v], wh, ds[v], w, k.max_weight);
        wo4 |= (unsigned)w << (8 * v);
      }
      dd.x = (unsigned)ds[0] | ((unsigned)ds[1] << 16);
      dd.y = (unsigned)ds[2] | ((unsigned)ds[3] << 16);
      *dp = dd;
    }
    dw[q] = wo4;
  }
  if (sv.rgbw) {
    const unsigned* hc = reinterpret_cast<const unsigned*>(host + d.sdf_bytes + kBlockVoxels);
    unsigned* dc = sv.rgbw + (size_t)ptr * kBlockVoxels;
    for (int v = lane; v < kBlockVoxels; v += 32) dc[v] = merge_colour(hc[v], dc[v], k.max_weight);
  }
}

// Bring the selected host blocks back, one warp per block: merge into the
// fresh pool block the allocation stage gave it, or copy into a new one.
template <int S>
__global__ void __launch_bounds__(kSwapThreads) swap_in_kernel(SwapConst k, SceneView sv, SwapDev d) {
  const int n = min(__ldcg(&d.ctr->n_cand), d.cand_cap);
  const int capacity = k.capacity;
  const int lane = threadIdx.x & 31;
  const int n_warps = gridDim.x * kSwapWarps;
  const int hw0 = __ldcg(&d.ctr->hw0);
  for (int i = blockIdx.x * kSwapWarps + (threadIdx.x >> 5); i < n; i += n_warps) {
    const SwapCand c = d.cand[i];
    if (!selected(d, c, n, capacity)) continue;
    if (c.entry < 0 || c.entry >= d.n_entries || c.ptr >= sv.pool) {
      if (lane == 0) set_status(sv.sc, kStInternal);
      continue;
    }
    const unsigned char* host = d.host + (size_t)c.entry * d.block_bytes;
    int ptr = c.ptr;
    if (ptr >= 0) {
      merge_block<S>(k, sv, d, host, ptr, lane);
      if (lane == 0) atomicAdd(&d.ctr->n_merged, 1);
    } else {
      int slot = 0;
      if (lane == 0) slot = atomicAdd(&d.ctr->n_alloc, 1);
      slot = __shfl_sync(0xffffffffu, slot, 0);
      ptr = hw0 + slot;
      if (ptr >= sv.pool) {  // cannot happen while prefetching needs a full call of room
        if (lane == 0) set_status(sv.sc, kStInternal);
        continue;
      }
      warp_copy(dev_sdf(sv, d, ptr), host, d.sdf_bytes, lane);
      warp_copy(sv.w + (size_t)ptr * kBlockVoxels, host + d.sdf_bytes, kBlockVoxels, lane);
      if (sv.rgbw)
        warp_copy(sv.rgbw + (size_t)ptr * kBlockVoxels, host + d.sdf_bytes + kBlockVoxels,
                  kBlockVoxels * 4, lane);
      if (lane == 0) {
        sv.key_of_ptr[ptr] = __ldcg(&sv.entries[c.entry].key);
        sv.entries[c.entry].ptr = ptr;
      }
    }
    __syncwarp();
    if (lane == 0) {
      d.state[c.entry] = 0;
      atomicAdd(&d.ctr->n_moved, 1);
    }
  }
}

// Fold the call's counts into the scene: free pool blocks and the totals.
__global__ void swap_finish_kernel(SceneView sv, SwapDev d, int out) {
  SwapCounters* c = d.ctr;
  SwapTotals* t = d.totals;
  const long long moved = c->n_moved;
  if (out) {
    if (c->compact_failed) set_status(sv.sc, kStInternal);  // the pool keeps its holes
    else sv.sc->free_top += (int)moved;
    t->host_blocks += moved;
    t->total_out += moved;
    t->last_out = moved;
    t->last_out_candidates = c->n_cand;
  } else {
    sv.sc->free_top -= c->n_alloc;
    t->host_blocks -= moved;
    t->total_in += moved;
    t->total_merged += c->n_merged;
    t->last_in = moved;
    t->last_merged = c->n_merged;
    t->last_in_candidates = c->n_cand;
  }
}

}  // namespace

struct SwapWork {
  SwapDev d;
  unsigned char* host;  // host pointer of the host voxel block array
  int capacity;
};

void free_swap_work(tsdf_scene* s) {
  SwapWork* w = s->swap;
  if (!w) return;
  cudaFree(w->d.state);
  cudaFree(w->d.cand);
  cudaFree(w->d.freed);
  cudaFree(w->d.freed_list);
  cudaFree(w->d.pairs);
  cudaFree(w->d.ctr);
  cudaFree(w->d.totals);
  if (w->host) cudaFreeHost(w->host);
  free(w);
  s->swap = nullptr;
}

int swap_reset(tsdf_scene* s) {
  if (!s->swap) return TSDF_OK;
  SwapWork* w = s->swap;
  TSDF_CUDA(cudaMemsetAsync(w->d.state, 0, (size_t)w->d.n_entries, s->stream));
  TSDF_CUDA(cudaMemsetAsync(w->d.totals, 0, sizeof(SwapTotals), s->stream));
  return TSDF_OK;
}

int swap_host_blocks(tsdf_scene* s, long long* n) {
  *n = 0;
  if (!s->swap) return TSDF_OK;
  SwapTotals t;
  TSDF_CUDA(cudaMemcpyAsync(&t, s->swap->d.totals, sizeof(t), cudaMemcpyDeviceToHost, s->stream));
  TSDF_CUDA(cudaStreamSynchronize(s->stream));
  *n = t.host_blocks;
  return TSDF_OK;
}

namespace {

int elem_bytes(int storage) { return storage == TSDF_STORAGE_F32 ? 4 : 2; }

// The view's constants (capacity and max_weight are the caller's).
int make_view_const(double voxel_size, const tsdf_intrinsics* in, const double* M,
                    double margin, double max_depth, SwapConst* k) {
  if (!in || !M || validate_intr(in)) return TSDF_ERR_INVALID_ARG;
  if (!(voxel_size > 0.0) || !std::isfinite(voxel_size)) return TSDF_ERR_INVALID_ARG;
  if (!std::isfinite(margin) || margin < 0.0 || !std::isfinite(max_depth))
    return TSDF_ERR_INVALID_ARG;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(M[i])) return TSDF_ERR_INVALID_ARG;
  if (M[12] != 0.0 || M[13] != 0.0 || M[14] != 0.0 || M[15] != 1.0) return TSDF_ERR_INVALID_ARG;
  const double fx = in->fx, fy = in->fy, cx = in->cx, cy = in->cy;
  const double lo_u = -0.5 - margin, hi_u = in->width - 0.5 + margin;
  const double lo_v = -0.5 - margin, hi_v = in->height - 0.5 + margin;
  // camera-space coefficient rows: z, and the four edge tests (see swap_visible)
  const double alpha[5][3] = {{0.0, 0.0, 1.0},
                              {fx, 0.0, cx - lo_u},
                              {fx, 0.0, cx - hi_u},
                              {0.0, fy, cy - lo_v},
                              {0.0, fy, cy - hi_v}};
  const double bs = 8.0 * voxel_size;
  for (int f = 0; f < 5; ++f) {
    double emax = 0.0, emin = 0.0, h = 0.0;
    for (int j = 0; j < 3; ++j) {
      double g = 0.0;
      for (int i = 0; i < 3; ++i) g += alpha[f][i] * M[4 * i + j];
      k->g[f][j] = g;
      emax += std::max(0.0, g);
      emin += std::min(0.0, g);
    }
    for (int i = 0; i < 3; ++i) h += alpha[f][i] * M[4 * i + 3];
    k->h[f] = h;
    k->ext_max[f] = bs * emax;
    k->ext_min[f] = bs * emin;
  }
  k->voxel_size = voxel_size;
  k->max_depth = max_depth;
  k->capacity = 0;
  k->max_weight = 0;
  return TSDF_OK;
}

int make_swap_const(const tsdf_scene* s, const tsdf_intrinsics* in, const double* M,
                    double margin, double max_depth, SwapConst* k) {
  const int rc = make_view_const((double)s->desc.voxel_size, in, M, margin, max_depth, k);
  if (rc) return rc;
  k->capacity = s->swap->capacity;
  k->max_weight = s->desc.max_weight;
  return TSDF_OK;
}

int grid_for(const tsdf_scene* s) { return s->sm_count * 4; }

int enqueue_radix(tsdf_scene* s, const SwapDev& d, int capacity) {
  for (int pass = 0; pass < 6; ++pass) {
    swap_radix_kernel<<<grid_for(s), kSwapThreads, 0, s->stream>>>(d, capacity, pass);
    TSDF_CUDA(cudaGetLastError());
  }
  s->launches += 6;
  return TSDF_OK;
}

}  // namespace

}  // namespace tsdf

using namespace tsdf;

int tsdf_scene_enable_swapping(tsdf_scene* s, int32_t transfer_blocks) {
  if (!s || s->swap || transfer_blocks < 1 || transfer_blocks > s->sv.pool)
    return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  SwapWork* w = (SwapWork*)calloc(1, sizeof(SwapWork));
  if (!w) return TSDF_ERR_OUT_OF_MEMORY;
  s->swap = w;
  w->capacity = transfer_blocks;
  SwapDev& d = w->d;
  d.n_entries = (int)s->n_entries;
  d.cand_cap = std::max(s->sv.pool, d.n_entries);
  d.sdf_bytes = kBlockVoxels * elem_bytes(s->desc.storage);
  d.block_bytes = (long long)d.sdf_bytes + kBlockVoxels + (s->sv.rgbw ? 4 * kBlockVoxels : 0);
  cudaError_t e = cudaMalloc((void**)&d.state, (size_t)d.n_entries);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.cand, (size_t)d.cand_cap * sizeof(SwapCand));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.freed, (size_t)s->sv.pool);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.freed_list, (size_t)transfer_blocks * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.pairs, (size_t)transfer_blocks * sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.ctr, sizeof(SwapCounters));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.totals, sizeof(SwapTotals));
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&w->host, (size_t)d.n_entries * (size_t)d.block_bytes,
                      cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&d.host, w->host, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.state, 0, (size_t)d.n_entries, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.freed, 0, (size_t)s->sv.pool, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.ctr, 0, sizeof(SwapCounters), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.totals, 0, sizeof(SwapTotals), s->stream);
  if (e != cudaSuccess) {
    free_swap_work(s);
    return e == cudaErrorMemoryAllocation ? TSDF_ERR_OUT_OF_MEMORY : cuda_fail(e);
  }
  return TSDF_OK;
}

int tsdf_swap_out(tsdf_scene* s, const tsdf_intrinsics* intr, const double world_to_cam[16],
                  double margin_px, double max_depth) {
  if (!s || !s->swap) return TSDF_ERR_INVALID_ARG;
  SwapConst k;
  int rc = make_swap_const(s, intr, world_to_cam, margin_px, max_depth, &k);
  if (rc) return rc;
  TSDF_CUDA(cudaSetDevice(s->device));
  const SwapDev& d = s->swap->d;
  TSDF_CUDA(cudaMemsetAsync(d.ctr, 0, sizeof(SwapCounters), s->stream));
  swap_out_select_kernel<<<grid_for(s), kSwapThreads, 0, s->stream>>>(k, s->sv, d);
  TSDF_CUDA(cudaGetLastError());
  s->launches += 1;
  if ((rc = enqueue_radix(s, d, k.capacity))) return rc;
  swap_out_copy_kernel<<<grid_for(s), kSwapThreads, 0, s->stream>>>(s->sv, d, k.capacity);
  TSDF_CUDA(cudaGetLastError());
  swap_compact_kernel<<<1, 1024, 0, s->stream>>>(d, k.capacity);
  TSDF_CUDA(cudaGetLastError());
  swap_move_kernel<<<grid_for(s), kSwapThreads, 0, s->stream>>>(s->sv, d);
  TSDF_CUDA(cudaGetLastError());
  swap_finish_kernel<<<1, 1, 0, s->stream>>>(s->sv, d, 1);
  TSDF_CUDA(cudaGetLastError());
  s->launches += 4;
  return TSDF_OK;
}

int tsdf_swap_in(tsdf_scene* s, const tsdf_intrinsics* intr, const double world_to_cam[16],
                 double margin_px, double max_depth) {
  if (!s || !s->swap) return TSDF_ERR_INVALID_ARG;
  SwapConst k;
  int rc = make_swap_const(s, intr, world_to_cam, margin_px, max_depth, &k);
  if (rc) return rc;
  TSDF_CUDA(cudaSetDevice(s->device));
  const SwapDev& d = s->swap->d;
  TSDF_CUDA(cudaMemsetAsync(d.ctr, 0, sizeof(SwapCounters), s->stream));
  swap_in_select_kernel<<<grid_for(s), kSwapThreads, 0, s->stream>>>(k, s->sv, d);
  TSDF_CUDA(cudaGetLastError());
  s->launches += 1;
  if ((rc = enqueue_radix(s, d, k.capacity))) return rc;
  switch (s->desc.storage) {
    case TSDF_STORAGE_I16:
      swap_in_kernel<1><<<grid_for(s), kSwapThreads, 0, s->stream>>>(k, s->sv, d);
      break;
    case TSDF_STORAGE_F16:
      swap_in_kernel<2><<<grid_for(s), kSwapThreads, 0, s->stream>>>(k, s->sv, d);
      break;
    default:
      swap_in_kernel<0><<<grid_for(s), kSwapThreads, 0, s->stream>>>(k, s->sv, d);
  }
  TSDF_CUDA(cudaGetLastError());
  swap_finish_kernel<<<1, 1, 0, s->stream>>>(s->sv, d, 0);
  TSDF_CUDA(cudaGetLastError());
  s->launches += 2;
  return TSDF_OK;
}

int tsdf_swap_visibility(float voxel_size, const tsdf_intrinsics* intr,
                         const double world_to_cam[16], double margin_px, double max_depth,
                         const int16_t* keys, int64_t n, uint8_t* visible) {
  if (n < 0 || (n > 0 && (!keys || !visible))) return TSDF_ERR_INVALID_ARG;
  SwapConst k;
  const int rc = make_view_const((double)voxel_size, intr, world_to_cam, margin_px, max_depth, &k);
  if (rc) return rc;
  for (int64_t i = 0; i < n; ++i)
    visible[i] = swap_visible(k, pack_key(keys[3 * i], keys[3 * i + 1], keys[3 * i + 2])) ? 1 : 0;
  return TSDF_OK;
}

int tsdf_swap_merge_voxels(int32_t storage, int32_t max_weight, int64_t n, const void* host_sdf,
                           const uint8_t* host_w, const uint32_t* host_rgbw, void* sdf,
                           uint8_t* w, uint32_t* rgbw) {
  if (storage < TSDF_STORAGE_F32 || storage > TSDF_STORAGE_F16 || max_weight < 1 ||
      max_weight > 255 || n < 0 || (n > 0 && (!host_sdf || !host_w || !sdf || !w)) ||
      (!host_rgbw != !rgbw))
    return TSDF_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) {
    int wd = w[i];
    const int wh = host_w[i];
    if (storage == TSDF_STORAGE_F32) {
      merge_f32(static_cast<const float*>(host_sdf)[i], wh, static_cast<float*>(sdf)[i], wd,
                max_weight);
    } else if (storage == TSDF_STORAGE_I16) {
      merge_i16(static_cast<const unsigned short*>(host_sdf)[i], wh,
                static_cast<unsigned short*>(sdf)[i], wd, max_weight);
    } else {
      merge_f16(static_cast<const unsigned short*>(host_sdf)[i], wh,
                static_cast<unsigned short*>(sdf)[i], wd, max_weight);
    }
    w[i] = (uint8_t)wd;
    if (rgbw) rgbw[i] = merge_colour(host_rgbw[i], rgbw[i], max_weight);
  }
  return TSDF_OK;
}

int tsdf_get_swap_stats(tsdf_scene* s, tsdf_swap_stats* out) {
  if (!s || !out || !s->swap) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  SwapTotals t;
  TSDF_CUDA(cudaMemcpyAsync(&t, s->swap->d.totals, sizeof(t), cudaMemcpyDeviceToHost, s->stream));
  TSDF_CUDA(cudaStreamSynchronize(s->stream));
  out->host_blocks = t.host_blocks;
  out->transfer_blocks = s->swap->capacity;
  out->last_out_candidates = t.last_out_candidates;
  out->last_out = t.last_out;
  out->last_in_candidates = t.last_in_candidates;
  out->last_in = t.last_in;
  out->last_merged = t.last_merged;
  out->total_out = t.total_out;
  out->total_in = t.total_in;
  out->total_merged = t.total_merged;
  return TSDF_OK;
}

int tsdf_read_host_blocks(tsdf_scene* s, int16_t* keys, void* sdf, uint8_t* w, uint8_t* rgbw,
                          int64_t capacity, int64_t* n_written) {
  if (!s || !n_written || !s->swap || (rgbw && !s->sv.rgbw)) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  const SwapDev& d = s->swap->d;
  std::vector<unsigned char> state((size_t)d.n_entries);
  std::vector<HashEntry> entries((size_t)d.n_entries);
  TSDF_CUDA(cudaMemcpyAsync(state.data(), d.state, state.size(), cudaMemcpyDeviceToHost, s->stream));
  TSDF_CUDA(cudaMemcpyAsync(entries.data(), s->sv.entries, entries.size() * sizeof(HashEntry),
                            cudaMemcpyDeviceToHost, s->stream));
  TSDF_CUDA(cudaStreamSynchronize(s->stream));
  std::vector<std::pair<unsigned long long, int>> found;
  for (int e = 0; e < d.n_entries; ++e)
    if (state[e] && entries[e].key != kKeyEmpty) found.emplace_back(canonical_key(entries[e].key), e);
  std::sort(found.begin(), found.end());
  const int64_t n = (int64_t)found.size();
  *n_written = n;
  if (capacity < n) return TSDF_ERR_CAPACITY;
  const int eb = elem_bytes(s->desc.storage);
  for (int64_t i = 0; i < n; ++i) {
    const int e = found[i].second;
    const unsigned char* blk = s->swap->host + (size_t)e * d.block_bytes;
    int x, y, z;
    unpack_key(entries[e].key, x, y, z);
    if (keys) {
      keys[3 * i] = (int16_t)x;
      keys[3 * i + 1] = (int16_t)y;
      keys[3 * i + 2] = (int16_t)z;
    }
    for (int l = 0; l < kBlockVoxels; ++l) {  // canonical voxel l from storage order
      const int v = storage_voxel(l);
      if (sdf)
        memcpy((unsigned char*)sdf + ((size_t)i * kBlockVoxels + l) * eb, blk + (size_t)v * eb, eb);
      if (w) w[(size_t)i * kBlockVoxels + l] = blk[d.sdf_bytes + v];
      if (rgbw)
        memcpy(rgbw + ((size_t)i * kBlockVoxels + l) * 4, blk + d.sdf_bytes + kBlockVoxels + 4 * v, 4);
    }
  }
  return TSDF_OK;
}
