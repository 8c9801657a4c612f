// alloc.cu -- allocation stage of the fusion step (Section 4.2, first and
// second stages).
//
//   alloc_kernel : one CTA per pixel tile (16x16 by default; 16x8 or 32x8).
//     1. every valid pixel walks its ray segment between camera depths d - mu
//        and d + mu block by block (3-D DDA over the unit block grid) and
//        drops each block key into a shared-memory set (duplicates within the
//        tile collapse there);
//     2. the distinct keys are probed in parallel, one thread per key: found
//        in the hash table, or inserted into a free bucket entry (lock-free
//        CAS on the key word); keys whose bucket is full go to a per-frame
//        overflow set;
//     3. the tile's depth maximum goes into the depth-max pyramid for the
//        integration kernel's block selection;
//     4. the last CTA to finish commits the frame: overflow keys get an
//        excess-list entry linked at the tail of their bucket's chain (CAS on
//        the link); if the frame needs more pool blocks than are free, the new
//        keys are sorted and the smallest ones win; the free stack is popped
//        and every new block's pool index is written into its hash entry and
//        into key_of_ptr (its voxels are initialised by the integration
//        kernel). The frame's counters and depth maxima go to its set of
//        per-frame state (FrameConst::set, see FrameCounters).
//
// Departure from the report: its first stage uses plain non-atomic writes and
// accepts that two new blocks with the same hash index in one frame drop one
// of them. Here no block is dropped: bucket entries are claimed by CAS, the
// overflow set deduplicates excess candidates, and excess entries are linked
// by CAS, so every block met by a band segment is allocated in the frame that
// meets it (as long as the pool and the excess list have room).
//
// All loops are bounded; none waits on another thread.
#include "tsdf_internal.cuh"

namespace tsdf {

namespace {

// Record a key that needs a pool block. `free0` is the number of free pool
// blocks when the frame began: while the frame's new keys fit, the i-th one
// takes pool block pool - free0 + i at once (the free stack's pop, done
// eagerly; the commit then only updates the counters). If more keys arrive
// than fit, the commit reassigns every new key by the smallest-keys rule.
__device__ __forceinline__ void append_new(const SceneView& sv, AllocCounters* A,
                                           unsigned long long key, int entry, int free0) {
  const int i = atomicAdd(&A->n_new, 1);
  if (i < sv.new_cap) {
    sv.new_list[i].key = key;
    sv.new_list[i].entry = entry;
    if (i < free0) {
      const int ptr = sv.pool - free0 + i;
      sv.entries[entry].ptr = ptr;
      sv.key_of_ptr[ptr] = key;
    }
    // the committing CTA reads the record after the frame's last arrival
    __threadfence();
  } else {
    // cannot record it this frame: leave it unallocated (retried next frame)
    atomicExch(&sv.entries[entry].ptr, kPtrUnallocated);
    set_status(sv.sc, kStPool);
  }
}

__device__ void overflow_insert(const SceneView& sv, AllocCounters* A, unsigned long long key,
                                unsigned bucket) {
  const unsigned mask = (unsigned)sv.ov_set_mask;
  unsigned h = set_hash(key) & mask;
  for (unsigned i = 0; i <= mask; ++i) {
    unsigned long long k = __ldcg(&sv.ov_set[h]);
    if (k == kKeyEmpty) {
      k = atomicCAS(&sv.ov_set[h], kKeyEmpty, key);
      if (k == kKeyEmpty) {
        // one list slot per set slot, so j < set size always
        const int j = atomicAdd(&A->n_overflow, 1);
        sv.ov_list[j].key = key;
        sv.ov_list[j].bucket = (int)bucket;
        sv.ov_list[j].set_slot = (int)h;
        __threadfence();  // read by the committing CTA
        return;
      }
    }
    if (k == key) return;
    h = (h + 1) & mask;
  }
  set_status(sv.sc, kStExcess);  // frame overflow set full
}

__device__ __forceinline__ ulonglong2 load_entry(const SceneView& sv, int e) {
  return __ldcg(reinterpret_cast<const ulonglong2*>(&sv.entries[e]));
}
__device__ __forceinline__ int entry_ptr(ulonglong2 q) { return (int)(unsigned)(q.y & 0xffffffffull); }
__device__ __forceinline__ int entry_next(ulonglong2 q) { return (int)(unsigned)(q.y >> 32); }

// Find `key` or claim a bucket entry for it; mark it for allocation if it has
// no pool block yet. Chains are not modified while this runs (excess entries
// are only added by the commit), so a chain walk sees a fixed list.
__device__ void find_or_insert(const SceneView& sv, AllocCounters* A, unsigned long long key,
                               int free0) {
  const unsigned b = bucket_of(key, (unsigned)sv.bucket_mask);
  const int base = (int)b * sv.entries_per_bucket;
  const int E = sv.entries_per_bucket;
  // the first two entries (key, ptr, next) are read in one round trip
  const ulonglong2 q0 = load_entry(sv, base);
  ulonglong2 q1 = E > 1 ? load_entry(sv, base + 1) : make_ulonglong2(kKeyEmpty, 0);
  int slot = -1, ptr = kPtrUnallocated;
  for (int s = 0; s < E; ++s) {
    const ulonglong2 q = s == 0 ? q0 : (s == 1 ? q1 : load_entry(sv, base + s));
    unsigned long long k = q.x;
    if (k == key) {
      slot = base + s;
      ptr = entry_ptr(q);
      break;
    }
    if (k != kKeyEmpty) continue;
    // occupied entries form a prefix: the key is absent; claim this entry
    k = atomicCAS(&sv.entries[base + s].key, kKeyEmpty, key);
    if (k == kKeyEmpty) {
      slot = base + s;
      ptr = kPtrUnallocated;
      break;
    }
    if (k == key) {
      slot = base + s;
      ptr = __ldcg(&sv.entries[base + s].ptr);
      break;
    }
    // another key took this entry: the next one may have changed since it
    // was read, so read it again
    if (s == 0 && E > 1) q1 = load_entry(sv, base + 1);
  }
  if (slot < 0) {
    int idx = entry_next(q0);
    for (int guard = 0; idx >= 0; ++guard) {
      if (guard > sv.excess_cap) {
        set_status(sv.sc, kStTimeout);
        return;
      }
      const int ei = sv.n_bucket_entries + idx;
      const ulonglong2 q = load_entry(sv, ei);
      if (q.x == key) {
        slot = ei;
        ptr = entry_ptr(q);
        break;
      }
      idx = entry_next(q);
    }
  }
  if (slot < 0) {
    overflow_insert(sv, A, key, b);
    return;
  }
  if (ptr == kPtrUnallocated &&
      atomicCAS(&sv.entries[slot].ptr, kPtrUnallocated, kPtrPending) == kPtrUnallocated)
    append_new(sv, A, key, slot, free0);
}

// Bitonic sort of new_list[0, n2) by canonical key (n2 a power of two) within
// one CTA; entries at [n, n2) were padded with the largest key.
__device__ void sort_new_list(NewRec* a, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          NewRec x = a[i], y = a[l];
          const unsigned long long cx = x.key == kKeyEmpty ? ~0ull : canonical_key(x.key);
          const unsigned long long cy = y.key == kKeyEmpty ? ~0ull : canonical_key(y.key);
          const bool up = (i & k) == 0;
          if ((cx > cy) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// The frame's commit, run by one whole CTA after every find-or-insert of the
// frame has finished (see the file comment, step 4).
__device__ void commit_frame(const SceneView& sv, AllocCounters* A) {
  // 1. excess entries for the overflow keys
  const int n_ov = min(__ldcg(&A->n_overflow), sv.ov_set_mask + 1);
  const int free0 = __ldcg(&sv.sc->free_top);  // unchanged since the frame began
  for (int i = threadIdx.x; i < n_ov; i += blockDim.x) {
    const OverflowRec rec = sv.ov_list[i];
    if (rec.bucket < 0 || rec.bucket > sv.bucket_mask || rec.set_slot < 0 ||
        rec.set_slot > sv.ov_set_mask) {
      set_status(sv.sc, kStInternal);  // inconsistent record: skip it
      continue;
    }
    const int idx = atomicAdd(&sv.sc->excess_top, 1);
    if (idx >= sv.excess_cap) {
      set_status(sv.sc, kStExcess);
      sv.ov_set[rec.set_slot] = kKeyEmpty;
      continue;
    }
    const int e = sv.n_bucket_entries + idx;
    sv.entries[e].key = rec.key;
    sv.entries[e].ptr = kPtrPending;
    sv.entries[e].next = kLinkNone;
    __threadfence();
    int* link = &sv.entries[rec.bucket * sv.entries_per_bucket].next;
    bool linked = false;
    for (int guard = 0; guard <= sv.excess_cap; ++guard) {
      const int old = atomicCAS(link, kLinkNone, idx);
      if (old == kLinkNone) {
        linked = true;
        break;
      }
      link = &sv.entries[sv.n_bucket_entries + old].next;
    }
    if (!linked) {
      set_status(sv.sc, kStTimeout);
    } else {
      append_new(sv, A, rec.key, e, free0);
    }
    sv.ov_set[rec.set_slot] = kKeyEmpty;
  }
  __syncthreads();

  // 2. pool blocks: if too few are free, the smallest keys are allocated
  __shared__ int s_n, s_free;
  if (threadIdx.x == 0) {
    s_n = min(__ldcg(&A->n_new), sv.new_cap);
    s_free = __ldcg(&sv.sc->free_top);
  }
  __syncthreads();
  int n = s_n;
  const int free_blocks = s_free;
  if (n > free_blocks) {
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int i = n + threadIdx.x; i < n2; i += blockDim.x) {
      sv.new_list[i].key = kKeyEmpty;
      sv.new_list[i].entry = -1;
    }
    __syncthreads();
    sort_new_list(sv.new_list, n2);
    for (int i = free_blocks + threadIdx.x; i < n; i += blockDim.x) {
      const int e = sv.new_list[i].entry;
      if (e >= 0 && e < sv.n_bucket_entries + sv.excess_cap)
        sv.entries[e].ptr = kPtrUnallocated;
      else
        set_status(sv.sc, kStInternal);
    }
    n = free_blocks;
    if (threadIdx.x == 0) set_status(sv.sc, kStPool);
  }
  __syncthreads();
  // 3. pop the free stack: new block i gets pool index pool - free + i
  // (already done by append_new unless the pool ran short and the keys were
  // sorted above)
  for (int i = threadIdx.x; i < n && s_n > free_blocks; i += blockDim.x) {
    const NewRec rec = sv.new_list[i];
    const int ptr = sv.pool - free_blocks + i;
    if (rec.entry < 0 || rec.entry >= sv.n_bucket_entries + sv.excess_cap || ptr < 0 ||
        ptr >= sv.pool) {
      set_status(sv.sc, kStInternal);  // inconsistent record: skip it
      continue;
    }
    sv.entries[rec.entry].ptr = ptr;
    sv.key_of_ptr[ptr] = rec.key;
  }
  if (threadIdx.x == 0) {
    A->n_new = n;
    A->assign_base = free_blocks;
    sv.sc->free_top = free_blocks - n;
  }
}

// shared-memory key set per CTA: two slots per pixel of the tile
__host__ __device__ constexpr int set_slots(int threads) { return 2 * threads; }
constexpr int kSetProbe = 32;            // probe limit before the global fallback
constexpr int kMaxDdaSteps = 64;
constexpr float kKeyLimit = 32767.0f;

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Add `key` to the CTA's shared set; if the set is crowded, probe the global
// table directly instead (same result, more global traffic).
template <int kSetSlots>
__device__ __forceinline__ void tile_set_add(unsigned long long* set, const SceneView& sv,
                                             AllocCounters* A, unsigned long long key,
                                             int free0) {
  unsigned h = set_hash(key) & (kSetSlots - 1);
  for (int i = 0; i < kSetProbe; ++i) {
    const unsigned long long k = atomicCAS(&set[h], kKeyEmpty, key);
    if (k == kKeyEmpty || k == key) return;
    h = (h + 1) & (kSetSlots - 1);
  }
  find_or_insert(sv, A, key, free0);
}

// One CTA's share of a scene's allocation stage: pixel tile (tx, ty) of
// kTileW x kTileH pixels, the cta-th of the scene's n_cta tiles.
template <int kTileW, int kTileH>
__device__ void alloc_tile(const FrameConst& fc, const SceneView& sv, int tx, int ty, int cta,
                           int n_cta) {
  constexpr int kAllocThreads = kTileW * kTileH;
  constexpr int kSetSlots = set_slots(kAllocThreads);
  __shared__ unsigned long long s_set[kSetSlots];
  __shared__ unsigned s_max[kAllocThreads / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSetSlots; i += kAllocThreads) s_set[i] = kKeyEmpty;
  // everything below reads or writes what the previous kernel of the scene
  // may still be using (counters, sanitised depth, the hash table)
  wait_prior_grid();
  // this frame's set of per-frame state (clear: see FrameCounters)
  const int par = fc.set;
  AllocCounters* A = &sv.fc->a[par];
  const int free0 = __ldcg(&sv.sc->free_top);  // free pool blocks as the frame begins

  const int u = tx * kTileW + (threadIdx.x % kTileW);
  const int v = ty * kTileH + (threadIdx.x / kTileW);
  const bool in_img = u < fc.width && v < fc.height;
  const float d = in_img ? __ldg(fc.depth + v * fc.pitch + u) : 0.0f;
  const bool active = in_img && isfinite(d) && d > 0.0f;
  // sanitised copy for the integration kernel: no measurement -> -1e30 (a
  // finite stand-in far below any camera depth), so its eta = d - z test
  // rejects such pixels by itself and its arithmetic stays finite
  if (in_img) sv.depth_san[par * sv.depth_san_stride + v * fc.width + u] = active ? d : -1e30f;

  // tile maximum of the measured depth (visible-list pruning)
  const unsigned bits = active ? __float_as_uint(d) : 0u;
  const unsigned wm = __reduce_max_sync(0xffffffffu, bits);
  if (lane == 0) s_max[warp] = wm;
  __syncthreads();  // also publishes the cleared key set

  // band segment in block units: P(sigma) = g + sigma * G r, walked by a 3-D
  // DDA (Amanatides & Woo) over the unit block grid; scalar state so nothing
  // is indexed dynamically
  if (active) {
    const float rx = ((float)u - fc.cx) * fc.inv_fx;
    const float ry = ((float)v - fc.cy) * fc.inv_fy;
    const float s0 = d - fc.mu, s1 = d + fc.mu;
    const float dirx = fmaf(fc.G[0], rx, fmaf(fc.G[1], ry, fc.G[2]));
    const float diry = fmaf(fc.G[3], rx, fmaf(fc.G[4], ry, fc.G[5]));
    const float dirz = fmaf(fc.G[6], rx, fmaf(fc.G[7], ry, fc.G[8]));
    const float p0x = fmaf(s0, dirx, fc.g[0]), p1x = fmaf(s1, dirx, fc.g[0]);
    const float p0y = fmaf(s0, diry, fc.g[1]), p1y = fmaf(s1, diry, fc.g[1]);
    const float p0z = fmaf(s0, dirz, fc.g[2]), p1z = fmaf(s1, dirz, fc.g[2]);
    const bool in_range = fabsf(p0x) < kKeyLimit && fabsf(p1x) < kKeyLimit &&
                          fabsf(p0y) < kKeyLimit && fabsf(p1y) < kKeyLimit &&
                          fabsf(p0z) < kKeyLimit && fabsf(p1z) < kKeyLimit;
    if (!in_range) {
      set_status(sv.sc, kStKeyRange);
    } else {
      int bx, by, bz, ex, ey, ez, sx, sy, sz;
      float tx, ty, tz, dx, dy, dz;
      auto axis = [](float p0, float p1, int& b, int& e, int& st, float& tm, float& td) {
        b = (int)floorf(p0);
        e = (int)floorf(p1);
        const float D = p1 - p0;
        const float r = rcp_approx(D);
        if (D > 0.0f) {
          st = 1;
          td = r;
          tm = ((float)(b + 1) - p0) * r;
        } else if (D < 0.0f) {
          st = -1;
          td = -r;
          tm = ((float)b - p0) * r;
        } else {
          st = 0;
          td = INFINITY;
          tm = INFINITY;
        }
      };
      axis(p0x, p1x, bx, ex, sx, tx, dx);
      axis(p0y, p1y, by, ey, sy, ty, dy);
      axis(p0z, p1z, bz, ez, sz, tz, dz);
      int it = 0;
      for (; it < kMaxDdaSteps; ++it) {
        {
          // lanes of the warp at the same block in this step insert it once
          const unsigned long long key = pack_key(bx, by, bz);
          const unsigned peers = __match_any_sync(__activemask(), key);
          if ((peers & ((1u << lane) - 1u)) == 0) tile_set_add<kSetSlots>(s_set, sv, A, key, free0);
        }
        if (bx == ex && by == ey && bz == ez) break;
        const float tmin = fminf(tx, fminf(ty, tz));
        if (tmin > 1.0f) break;  // rounding overshot the end block: segment done
        if (tx == tmin) {
          bx += sx;
          tx += dx;
        } else if (ty == tmin) {
          by += sy;
          ty += dy;
        } else {
          bz += sz;
          tz += dz;
        }
      }
      if (it == kMaxDdaSteps) set_status(sv.sc, kStTimeout);
    }
  }
  __syncthreads();

  // the tile's distinct keys, probed in parallel
  for (int i = threadIdx.x; i < kSetSlots; i += kAllocThreads) {
    const unsigned long long k = s_set[i];
    if (k != kKeyEmpty) find_or_insert(sv, A, k, free0);
  }

  if (threadIdx.x == 32) {
    // The tile's depth maximum for the integration kernel (read after this
    // kernel): reductions without a return value, so no round trip, issued
    // by a thread other than the one that signals the arrival below (whose
    // fence would otherwise wait for them).
    unsigned mm = 0;
    for (int i = 0; i < kAllocThreads / 32; ++i) mm = max(mm, s_max[i]);
    if (mm) atomicMax(&A->depth_max_bits, mm);
    // depth-max pyramid for the block selection: level 0 = 16x16-pixel
    // cells, written directly when the tile is one whole cell, else by
    // atomicMax into every cell the tile overlaps (the tile maximum bounds
    // each part); levels 1 and 2 by atomicMax. The integration kernel of the
    // frame that used this set before clears every level.
    if (fc.use_tiles) {
      unsigned* pyr = pyramid_set(sv, par);
      constexpr bool kWholeCell = kTileW == 16 && kTileH == 16;
      const int cx0 = (tx * kTileW) >> 4, cy0 = (ty * kTileH) >> 4;
      const int cx1 = min((tx * kTileW + kTileW - 1) >> 4, fc.tiles_x - 1);
      const int cy1 = min((ty * kTileH + kTileH - 1) >> 4, fc.tiles_y - 1);
      if (kWholeCell) pyr[cy0 * fc.tiles_x + cx0] = mm;
      if (mm) {
        for (int l = kWholeCell ? 1 : 0; l < kPyramidLevels; ++l) {
          int wl, hl;
          const int off = pyramid_level(fc.tiles_x, fc.tiles_y, l, wl, hl);
          for (int cy = cy0 >> l; cy <= (cy1 >> l); ++cy)
            for (int cx = cx0 >> l; cx <= (cx1 >> l); ++cx) atomicMax(&pyr[off + cy * wl + cx], mm);
        }
      }
    }
  }

  // The last CTA to finish commits the frame. Every thread that wrote a
  // new-list / overflow-list record fenced it; after the CTA barrier thread 0
  // fences and signals the arrival (one counter: one round trip), so the
  // committing CTA reads only completed records.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&A->alloc_done, 1) == n_cta - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    commit_frame(sv, A);
  }
}

// 2048 threads per SM (32 registers, a few spilled to L1): a 640x480
// image's 16x16 tiles then run in one wave.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH, 2048 / (TW * TH)) alloc_kernel(FrameConst fc,
                                                                         SceneView sv) {
  allow_dependents();
  alloc_tile<TW, TH>(fc, sv, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x,
                     gridDim.x * gridDim.y);
}

// Batched: CTA b belongs to the slot whose tile range holds b (binary search
// over the slot table); the slot's view and constants go to shared memory.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH, 2048 / (TW * TH)) alloc_batch_kernel(
    const SlotDesc* slots, int n) {
  __shared__ SlotDesc s_slot;
  __shared__ int s_idx;
  allow_dependents();
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (slots[mid].tile_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_idx = lo;
  }
  __syncthreads();
  {
    const unsigned* src = reinterpret_cast<const unsigned*>(&slots[s_idx]);
    unsigned* dst = reinterpret_cast<unsigned*>(&s_slot);
    for (int i = threadIdx.x; i < (int)(sizeof(SlotDesc) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int local = (int)blockIdx.x - s_slot.tile_begin;
  const int tiles_x = s_slot.fc.ctiles_x;
  alloc_tile<TW, TH>(s_slot.fc, s_slot.sv, local % tiles_x, local / tiles_x, local,
                     tiles_x * s_slot.fc.ctiles_y);
}

constexpr int kCommitThreads = 1024;

__global__ void __launch_bounds__(kCommitThreads) commit_kernel(SceneView sv, int set) {
  commit_frame(sv, &sv.fc->a[set]);
}

// Initialise the voxels of the blocks the commit handed out (sdf 1, w 0).
// The fusion step does this inside the integration kernel; this launch serves
// the resume path.
template <int S>
__global__ void __launch_bounds__(128) assign_kernel(SceneView sv, int set) {
  using T = typename Storage<S>::T;
  const AllocCounters* A = &sv.fc->a[set];
  const int n = A->n_new;
  const int base = A->assign_base;
  const int t = threadIdx.x;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int ptr = sv.pool - base + i;
    T* sdf = reinterpret_cast<T*>(sv.sdf) + (size_t)ptr * kBlockVoxels + 4 * t;
    const T init = Storage<S>::initial();
#pragma unroll
    for (int j = 0; j < 4; ++j) sdf[j] = init;
    reinterpret_cast<unsigned*>(sv.w + (size_t)ptr * kBlockVoxels)[t] = 0u;
  }
}

__global__ void insert_keys_kernel(const unsigned long long* keys, int n, SceneView sv, int set) {
  AllocCounters* A = &sv.fc->a[set];
  const int free0 = __ldcg(&sv.sc->free_top);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    find_or_insert(sv, A, keys[i], free0);
}

}  // namespace

cudaError_t launch_alloc(const FrameConst& fc, const SceneView& sv, cudaStream_t st) {
  const dim3 g(fc.ctiles_x, fc.ctiles_y);
  switch (fc.alloc_tile) {
    case kAllocTile16x8: return launch_pdl(alloc_kernel<16, 8>, g, dim3(128), st, fc, sv);
    case kAllocTile32x8: return launch_pdl(alloc_kernel<32, 8>, g, dim3(256), st, fc, sv);
    default: return launch_pdl(alloc_kernel<16, 16>, g, dim3(256), st, fc, sv);
  }
}

// (every slot of a batch uses the same tile shape)
cudaError_t launch_alloc_batch(const SlotDesc* d_slots, const SlotDesc* h_slots, int n,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const SlotDesc& last = h_slots[n - 1];
  const dim3 g(last.tile_begin + last.fc.ctiles_x * last.fc.ctiles_y);
  switch (last.fc.alloc_tile) {
    case kAllocTile16x8: return launch_pdl(alloc_batch_kernel<16, 8>, g, dim3(128), st, d_slots, n);
    case kAllocTile32x8: return launch_pdl(alloc_batch_kernel<32, 8>, g, dim3(256), st, d_slots, n);
    default: return launch_pdl(alloc_batch_kernel<16, 16>, g, dim3(256), st, d_slots, n);
  }
}

cudaError_t launch_commit(const SceneView& sv, int set, cudaStream_t st) {
  commit_kernel<<<1, kCommitThreads, 0, st>>>(sv, set);
  return cudaGetLastError();
}

cudaError_t launch_assign(const SceneView& sv, int set, int sm_count, cudaStream_t st) {
  const int grid = sm_count * 8;
  switch (sv.storage) {
    case TSDF_STORAGE_F32: assign_kernel<TSDF_STORAGE_F32><<<grid, 128, 0, st>>>(sv, set); break;
    case TSDF_STORAGE_I16: assign_kernel<TSDF_STORAGE_I16><<<grid, 128, 0, st>>>(sv, set); break;
    default: assign_kernel<TSDF_STORAGE_F16><<<grid, 128, 0, st>>>(sv, set); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_insert_keys(const unsigned long long* keys, int n, const SceneView& sv,
                               int set, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + 255) / 256;
  insert_keys_kernel<<<grid < 4096 ? grid : 4096, 256, 0, st>>>(keys, n, sv, set);
  return cudaGetLastError();
}

}  // namespace tsdf
