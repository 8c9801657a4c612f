// tsdf_internal.cuh -- device data layout and helpers of libtsdf (sm_103a).
//
// Layout in HBM (one scene):
//   entries   : (2^k * E + excess) x HashEntry (16 B). The first 2^k * E are
//               the ordered buckets of E entries (Section 3.3); the rest is
//               the unordered excess list. A bucket's chain of excess
//               entries hangs off the `next` field of the bucket's entry 0.
//   key_of_ptr: pool x u64, the packed block key stored in each pool block
//               (dense over [0, high-water): fusion never frees a block, and
//               a swap-out refills the blocks it frees from the pool's tail).
//   free pool blocks: the stack of Section 4.2 (second stage) is popped from
//               the top and never pushed back (the pool's used part stays
//               [0, pool - free_top)), so it needs no array: new block i of
//               a frame gets pool - free_top + i.
//   sdf, w    : structure of arrays, block-major: sdf[ptr*512 + l] (f32, or
//               i16 / f16) and w[ptr*512 + l] (u8), l in the storage voxel
//               order (storage_voxel). One block is 2 KB of f32 sdf (1 KB for
//               i16/f16) plus 512 B of weights, so a thread that owns four
//               consecutive voxels does one 16 B (8 B) and one 4 B access.
//   frame work: new-block list, overflow (excess-candidate) set and list,
//               sanitised depth, two depth-max pyramids over 16x16 tiles,
//               per-frame counters.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tsdf.h"

namespace tsdf {

constexpr int kBlockSide = 8;
constexpr int kBlockVoxels = 512;

// Voxel order inside a block in device memory: x fastest, then z, then y
// (index x + 8 z + 64 y), so that the voxels one warp instruction touches in
// the integration (x and z vary across lanes, y per slab) project near one
// image row for a camera held level. The canonical order of readback and
// load is x + 8 y + 64 z; the map between the two swaps the y and z fields
// and is its own inverse.
__host__ __device__ __forceinline__ int storage_voxel(int v) {
  return (v & 7) | (((v >> 6) & 7) << 3) | (((v >> 3) & 7) << 6);
}
constexpr unsigned long long kKeyEmpty = ~0ull;
constexpr int kPtrUnallocated = -2;  // entry holds a key but no pool block
constexpr int kPtrPending = -3;      // entry is in this frame's new list
constexpr int kLinkNone = -1;

// device status bits (SceneCounters::status)
enum : unsigned {
  kStPool = 1u,
  kStExcess = 2u,
  kStKeyRange = 4u,
  kStTimeout = 8u,
  kStInternal = 16u,  // a device index failed a consistency check; the access was skipped
};

struct __align__(16) HashEntry {
  unsigned long long key;  // packed block key or kKeyEmpty
  int ptr;                 // >= 0 pool index, kPtrUnallocated, kPtrPending
  int next;                // excess chain link (index into the excess list)
};

struct __align__(16) NewRec {
  unsigned long long key;
  int entry;  // index into entries[]
  int pad;
};

struct __align__(16) OverflowRec {
  unsigned long long key;
  int bucket;
  int set_slot;
};

// Per-frame state comes in two sets; frame t uses set t mod 2 (chosen by the
// host and passed in FrameConst::set): its counters here, its depth-max
// pyramid and its sanitised depth. The allocation kernel of the frame writes
// the set, the integration kernel reads it, and the integration kernel's last
// CTA folds the frame's counts into the scene counters and clears the set
// (counters and the pyramid levels built by atomics). So a frame always finds
// its set clear whatever ran before it (also when one captured frame is
// replayed), and frame t + 1's allocation can run while frame t is still
// being integrated (different sets).
constexpr int kArriveGroups = 32;
struct AllocCounters {
  // written by the allocation kernel
  int n_new;
  int n_overflow;
  int assign_base;           // free_top before this frame's pops
  unsigned depth_max_bits;   // max valid depth as float bits (non-negative)
  int alloc_done;            // arrival groups complete (last-CTA commit)
  int arrive[kArriveGroups]; // allocation CTAs finished, per arrival group
  // written by the integration kernel
  int n_visible;
  int integ_arrive;          // integration CTAs finished (last-CTA close)
  int pad;
  unsigned long long n_updated;
  // staged integration kernel: arrivals, visible blocks and updated voxels
  // of its CTAs in one word (see kPackArriveShift)
  unsigned long long integ_packed;
};
struct FrameCounters {
  AllocCounters a[2];
};

// A block selected for integration: its pool index, whether this frame's
// allocation handed it out (its voxels are initialised by the integration),
// and the camera-space point of its origin voxel as an unevaluated sum
// hi + lo per coordinate (32 B).
struct __align__(16) VisRec {
  int ptr;
  float chi[3];
  float clo[3];
  int fresh;
};

// persistent per scene
struct SceneCounters {
  int free_top;
  int excess_top;
  unsigned status;
  int pad;
  unsigned long long total_updated;
  unsigned long long total_visible;
  unsigned long long frames;
  unsigned long long last_new;
  unsigned long long last_visible;
  unsigned long long last_updated;
};

// Both counter structs live in one allocation so the host reads them with
// one copy.
struct Counters {
  SceneCounters sc;
  FrameCounters fc;
};

struct SceneView {
  HashEntry* entries;
  int bucket_mask;     // 2^k - 1
  int entries_per_bucket;
  int n_bucket_entries;  // 2^k * E
  int excess_cap;
  unsigned long long* key_of_ptr;
  int pool;
  void* sdf;
  unsigned char* w;
  int storage;
  NewRec* new_list;
  int new_cap;           // power of two >= pool
  OverflowRec* ov_list;
  unsigned long long* ov_set;
  int ov_set_mask;       // set size - 1 (power of two)
  float* depth_san;      // two buffers of depth_san_stride floats (frame set):
                         // the frame's depth, dense pitch = width, with every
                         // pixel without a measurement set to -1e30
  long long depth_san_stride;
  unsigned* tile_max;    // two depth-max pyramids (float bits), 2 tile_cap each:
                         // level 0 = 16x16 tiles
  int tile_cap;          // level-0 tiles a pyramid can describe
  FrameCounters* fc;
  SceneCounters* sc;
  unsigned* rgbw;        // voxel colours (tsdf_scene_enable_colour) or null:
                         // bytes r, g, b, colour weight, storage voxel order
};

// Per-frame constants, computed on the host in FP64 and rounded (hi/lo pairs
// for the world->camera transform of voxel coordinates).
struct FrameConst {
  // camera point of voxel v (integer coordinates): c = A v + t, A = s R.
  float A_hi[9], A_lo[9];
  float t_hi[3], t_lo[3];
  // world point of camera point q, in block units: G q + g
  // (G = R^-1 / (8 s), g = -R^-1 t / (8 s)).
  float G[9];
  float g[3];
  float fx, fy, cx, cy, inv_fx, inv_fy;
  float mu, inv_mu;
  float xmax, ymax;       // width - 2, height - 2
  int width, height;
  int pitch;              // depth row pitch in elements (pitch * height < 2^31)
  int tiles_x, tiles_y;   // 16x16 depth tiles of this image (pyramid level 0)
  int ctiles_x, ctiles_y; // allocation CTA tiles (of the shape alloc_tile names)
  int alloc_tile;         // allocation tile shape: kAllocTile16x16 / 16x8 / 32x8
  int use_tiles;          // the tile maxima fit in tile_max
  int max_weight;
  float voxel_size;
  const float* depth;
  int set;                // the frame's set of per-frame state (0 or 1)
  const uchar4* rgb;      // colour image registered to the depth (pitch =
                          // width) or null
};

// One scene of a batched step: its view, this step's frame constants, and the
// scene's first CTA in the batch's allocation grid.
struct SlotDesc {
  SceneView sv;
  FrameConst fc;
  int tile_begin;   // allocation grid: CTAs [tile_begin, tile_begin + tiles)
  int pad[3];
};
constexpr int kMaxBatch = 1024;  // scenes per batched step

// Pixels of one allocation CTA (one thread per pixel): 16x16 (one level-0
// cell of the depth-max pyramid, the default), 16x8 or 32x8 (batches pick
// the shape their autotuner finds fastest).
enum { kAllocTile16x16 = 0, kAllocTile16x8 = 1, kAllocTile32x8 = 2 };
__host__ __device__ constexpr int alloc_tile_w(int shape) { return shape == kAllocTile32x8 ? 32 : 16; }
__host__ __device__ constexpr int alloc_tile_h(int shape) { return shape == kAllocTile16x16 ? 16 : 8; }

// Programmatic dependent launch: a kernel launched with the programmatic
// serialization attribute may start while its predecessor finishes; it
// waits here before touching anything the predecessor writes (a no-op
// without the attribute), and lets its own dependents launch once all of
// its CTAs have started.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// ---------------------------------------------------------------------------
// keys

__host__ __device__ __forceinline__ unsigned long long pack_key(int x, int y, int z) {
  return (unsigned long long)(unsigned short)x |
         ((unsigned long long)(unsigned short)y << 16) |
         ((unsigned long long)(unsigned short)z << 32);
}

__host__ __device__ __forceinline__ void unpack_key(unsigned long long k, int& x, int& y, int& z) {
  x = (short)(k & 0xffffu);
  y = (short)((k >> 16) & 0xffffu);
  z = (short)((k >> 32) & 0xffffu);
}

// Sort key whose unsigned order is the lexicographic (x, y, z) order of the
// signed block coordinates.
__host__ __device__ __forceinline__ unsigned long long canonical_key(unsigned long long k) {
  int x, y, z;
  unpack_key(k, x, y, z);
  return ((unsigned long long)(x + 32768) << 32) | ((unsigned long long)(y + 32768) << 16) |
         (unsigned long long)(z + 32768);
}

// Bucket of a block: the spatial hash of Section 3.3 (three large primes
// multiplied into the coordinates and xor-ed, masked to the table size).
__device__ __forceinline__ unsigned bucket_of(unsigned long long k, unsigned mask) {
  int x, y, z;
  unpack_key(k, x, y, z);
  return (((unsigned)x * 73856093u) ^ ((unsigned)y * 19349669u) ^ ((unsigned)z * 83492791u)) & mask;
}

// Depth-max pyramid: level 0 holds one value per 16x16 pixel tile, level l
// halves the previous level's width and height (rounding up), levels are
// stored one after another (three levels: 16, 32 and 64 pixel cells).
// Returns the offset of level l and its width and height.
constexpr int kPyramidLevels = 3;
__host__ __device__ __forceinline__ int pyramid_level(int tiles_x, int tiles_y, int l, int& wl,
                                                      int& hl) {
  int off = 0;
  wl = tiles_x;
  hl = tiles_y;
  for (int i = 0; i < l; ++i) {
    off += wl * hl;
    wl = (wl + 1) >> 1;
    hl = (hl + 1) >> 1;
  }
  return off;
}

// Depth-max pyramid of allocation set p.
__host__ __device__ __forceinline__ unsigned* pyramid_set(const SceneView& sv, int p) {
  return sv.tile_max + (size_t)p * 2 * sv.tile_cap;
}

// Slot hash of the per-frame overflow set (64-bit finaliser mix).
__device__ __forceinline__ unsigned set_hash(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return (unsigned)k;
}

__device__ __forceinline__ void set_status(SceneCounters* sc, unsigned bits) {
  atomicOr(&sc->status, bits);
}

// Find a block's entry: bucket first, then the bucket's excess chain
// (Section 3.3 retrieval). Returns the entry index or -1. The chain walk is
// bounded by the excess-list length.
__device__ __forceinline__ int find_entry(const SceneView& sv, unsigned long long key) {
  const unsigned b = bucket_of(key, (unsigned)sv.bucket_mask);
  const int base = (int)b * sv.entries_per_bucket;
  for (int s = 0; s < sv.entries_per_bucket; ++s) {
    unsigned long long k = __ldcg(&sv.entries[base + s].key);
    if (k == key) return base + s;
    if (k == kKeyEmpty) return -1;  // occupied slots form a prefix
  }
  int idx = __ldcg(&sv.entries[base].next);
  for (int guard = 0; idx >= 0 && guard <= sv.excess_cap; ++guard) {
    const int e = sv.n_bucket_entries + idx;
    if (__ldcg(&sv.entries[e].key) == key) return e;
    idx = __ldcg(&sv.entries[e].next);
  }
  return -1;
}

// ---------------------------------------------------------------------------
// storage forms

template <int S> struct Storage;

template <> struct Storage<TSDF_STORAGE_F32> {
  using T = float;
  __device__ __forceinline__ static float load(T v) { return v; }
  __device__ __forceinline__ static T store(float x) { return x; }
  __device__ __forceinline__ static T initial() { return 1.0f; }
};

// Section 3.1: value = q / 32767, q = (short)(x * 32767) (truncation).
// The load multiplies by 1/32767 rounded up (0x38000101, within 1.5e-7 of
// q / 32767 for every q): with it, store(load(q)) == q for every code (with
// round-to-nearest, 1536 codes come back one lower), so an unchanged value
// stores back unchanged. (float)q is formed exactly from the bits of
// 1.5 * 2^23 + q (|q| < 2^22) minus 1.5 * 2^23, without a conversion
// instruction.
template <> struct Storage<TSDF_STORAGE_I16> {
  using T = short;
  __device__ __forceinline__ static float load(T v) {
    const float q = __int_as_float(0x4B400000 + (int)v) - 12582912.0f;
    return q * __int_as_float(0x38000101);
  }
  __device__ __forceinline__ static T store(float x) { return (short)__float2int_rz(x * 32767.0f); }
  __device__ __forceinline__ static T initial() { return 32767; }
};

template <> struct Storage<TSDF_STORAGE_F16> {
  using T = __half;
  __device__ __forceinline__ static float load(T v) { return __half2float(v); }
  __device__ __forceinline__ static T store(float x) { return __float2half_rn(x); }
  __device__ __forceinline__ static T initial() { return __float2half_rn(1.0f); }
};

inline size_t storage_bytes(int storage) { return storage == TSDF_STORAGE_F32 ? 4 : 2; }

// ---------------------------------------------------------------------------
// kernel launchers (one translation unit each)

// Launch with programmatic stream serialization (see wait_prior_grid): the
// kernel's CTAs may be scheduled while the previous kernel on the stream
// finishes; stream order still holds for everything after its wait.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// raycast (Section 4.4)

// Per-raycast constants, computed on the host in FP64 and rounded.
struct RayConst {
  float A_hi[9], A_lo[9];  // voxel v (integer) -> camera: c = A v + t, A = s R
  float t_hi[3], t_lo[3];
  float L[9];              // camera point q (metres) -> world voxel units: L q + o (L = R^-1 / s)
  float o_hi[3], o_lo[3];  // o: the camera centre in voxel units
  float fx, fy, cx, cy, inv_fx, inv_fy;
  float z_near;            // near plane of the search range (metres)
  float mu_v;              // truncation band in voxels (mu / s)
  float voxel_size;
  int width, height;
  int tiles_x, tiles_y;    // kRayTile x kRayTile pixel tiles
};

// One block's footprint in the search range: the pixels [u0, u1] x [v0, v1]
// (centres inside the bounding box of its projected corners) get the camera
// depths [z_lo, z_hi] of its corners.
struct __align__(16) RayRec {
  float z_lo, z_hi;
  unsigned short u0, u1, v0, v1;
};

constexpr int kRayTile = 16;           // pixel tile side; one CTA of kRayTile^2 threads
constexpr int kRayMaxTilesPerRec = 16; // wider footprints go to the list every tile reads
constexpr int kRayMaxSteps = 1 << 16;  // march guard (a ray reaching it reports no surface)

struct RayCounters {
  int n_rec;     // footprints this raycast
  int n_large;   // footprints spanning more than kRayMaxTilesPerRec tiles
  int pad[2];
  unsigned long long steps;  // samples taken by all rays
  unsigned long long hits;   // rays that found a surface
  unsigned long long guard;  // rays stopped by kRayMaxSteps
};

// Raycast work buffers of a scene (allocated on its first raycast, grown
// with the pool and the image's tile count).
struct RayWork {
  RayRec* rec;         // pool footprints
  int* frag;           // kRayMaxTilesPerRec * pool footprint indices, grouped by tile
  int* large;          // pool footprint indices
  RayCounters* ctr;    // the counters, then tile_count[tile_cap] (zeroed together)
  int* tile_count;
  int* tile_off;       // tile_cap + 1 (exclusive prefix of the counts)
  int* tile_cursor;    // tile_cap
  int tile_cap;
  int pool;
};

// The raycast of one view in two parts: the search range's inputs (zero the
// counters, footprints, tile offsets, fragment scatter), then one CTA per
// tile (each pixel's search range + march). points: width * height float4
// (world metres, w = 1 on a surface, else all 0); range (optional): width *
// height float2 (z_lo, z_hi).
cudaError_t launch_raycast_range(const RayConst& rc, const SceneView& sv, const RayWork& w,
                                 int sm_count, cudaStream_t st);
cudaError_t launch_raycast_march(const RayConst& rc, const SceneView& sv, const RayWork& w,
                                 int storage, float4* points, float2* range, cudaStream_t st);

cudaError_t launch_alloc(const FrameConst& fc, const SceneView& sv, cudaStream_t st);
cudaError_t launch_commit(const SceneView& sv, int set, cudaStream_t st);
cudaError_t launch_assign(const SceneView& sv, int set, int sm_count, cudaStream_t st);
// ctas_per_sm: integration CTAs per SM (0 = as many as fit)
cudaError_t launch_integrate(const FrameConst& fc, const SceneView& sv, int sm_count, cudaStream_t st,
                             int ctas_per_sm = 0);
cudaError_t launch_finish_frame(const SceneView& sv, int set, cudaStream_t st);

// batched step over n slots (device array), one launch per stage (the
// integration: one per storage form present); the allocation tile shape is
// the slots' fc.alloc_tile
enum { kBatchKernelStaged = 0, kBatchKernelGeneral = 1 };
struct BatchIntegLaunch {
  int kernel;       // kBatchKernelStaged / kBatchKernelGeneral
  int threads;      // staged: 256 or 512
  int ctas_per_sm;  // general: CTAs per SM
};
cudaError_t launch_alloc_batch(const SlotDesc* d_slots, const SlotDesc* h_slots, int n,
                               cudaStream_t st);
cudaError_t launch_integrate_batch(const SlotDesc* d_slots, const SlotDesc* h_slots, int n,
                                   int sm_count, const BatchIntegLaunch& how, cudaStream_t st);


// keys-in insertion used by load_blocks: find or insert each key (same
// rules as the band allocation), leaving new ones in the new list.
cudaError_t launch_insert_keys(const unsigned long long* keys, int n, const SceneView& sv,
                               int set, cudaStream_t st);
cudaError_t launch_lookup(const unsigned long long* keys, int n, int* ptr_out, const SceneView& sv,
                          cudaStream_t st);
// canonical order of the allocated blocks: sorted (canonical key, ptr)
cudaError_t launch_sort_allocated(const SceneView& sv, int n, unsigned long long* sort_keys,
                                  int* sort_ptrs, int n_pow2, cudaStream_t st);
cudaError_t launch_gather_blocks(const SceneView& sv, const int* ptrs, int n, short* keys_out,
                                 void* sdf_out, unsigned char* w_out, cudaStream_t st);
cudaError_t launch_scatter_blocks(const SceneView& sv, const unsigned long long* keys, int n,
                                  const void* sdf_in, const unsigned char* w_in, cudaStream_t st);
// voxel colour words (r, g, b, weight bytes) of blocks ptrs[0..n), canonical
// voxel order, into out[n][512]
cudaError_t launch_gather_colour(const SceneView& sv, const int* ptrs, int n, unsigned* out,
                                 cudaStream_t st);

}  // namespace tsdf
