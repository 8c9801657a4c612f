// integrate.cu -- visible-block selection (Section 4.2, third stage) fused
// with the per-voxel integration (Section 4.3, computeUpdatedVoxelDepthInfo),
// for one scene per launch and for a batch of scenes per launch.
//
// One kernel per frame after the allocation kernel. Each CTA takes a strided
// share of the allocated blocks [0, high-water) (dense: pool indices are
// handed out in order, and a swap-out refills what it frees), one block per
// thread and pass:
//   1. a conservative test decides whether any voxel of the block can be
//      written by rule U this frame (frustum, the frame's maximum depth, and
//      the allocation's depth-max pyramid); blocks handed out by this frame's
//      allocation always pass (they are initialised here);
//   2. the passing blocks are compacted into shared memory as 32 B records
//      (pool index and the block origin's camera point as a double-float);
//   3. the CTA's warps take the records one by one (a shared counter) and
//      integrate a block each: every lane takes a quad (four voxels
//      consecutive in x and in memory) in each of the block's four 8x8x2
//      slabs; a quad's projections are tested once against the image border
//      (x is monotonic along a quad); the lane's sixteen depth gathers are
//      issued before any is used and its voxel loads before they return;
//      writes go to the quads rule U updates (every quad of a new block).
// Voxels are stored x + 8 z + 64 y in a block, so the voxels of one gather
// instruction project near one image row for a level camera.
//
// The allocation results of a frame (its counters, depth-max pyramid and
// sanitised depth) live in the frame's set of per-frame state; the last CTA
// of this kernel folds the frame's counts into the scene counters and clears
// the set, so the next frame that uses it finds it clear (see FrameCounters).
//
// Arithmetic: FP32 throughout, no FP64. The block origin is carried as an
// unevaluated sum of two floats built with exact product / sum transforms, so
// eta = d - z keeps ~1e-8 m accuracy at several metres; the per-voxel offset
// A l is a plain float (|A l| < 0.1 m).
#include <cstdlib>

#include "async_copy.cuh"
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

// Copy a struct of 4-byte words from global to shared memory with a CTA.
template <typename T>
__device__ __forceinline__ void cta_copy(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "word copy");
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

// ----------------------------------------------------------------------------
// integration

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Per-lane constants of one scene's frame for the integration of its blocks.
struct UnitConsts {
  const float* depth;  // sanitised depth, pitch = width, -1e30 = no measurement
  void* sdf;
  unsigned char* w;
  int pool;
  unsigned width, off_bias;  // pixel offset = vbits * width + ubits + off_bias
  float lbase[3], dk[3];     // A l of the lane's first voxel in slab 0; slab step
  float dz, pdx, pdy;        // one voxel step along x: camera z, fx X, fy Y
  float fx, fy, cxh, cyh;    // cxh = cx + 1/2, cyh = cy + 1/2
  float xlo, xhi, ylo, yhi;  // x + 1/2 in [1.5, W - 1.5], y + 1/2 in [1.5, H - 1.5]
  float mu, inv_mu;
  unsigned maxw4;  // maxW in every byte
  const uchar4* rgb;  // the frame's colour image (pitch = width) or null
  unsigned* rgbw;     // voxel colours (r, g, b, colour weight bytes) or null
};

// 2^23: for 0 <= v < 2^23, v + 2^23 rounded down is the float whose bit
// pattern is 0x4B000000 + floor(v), so a round-down add gives floor(v) as
// an integer without a conversion instruction.
constexpr float kFloorMagic = 8388608.0f;
constexpr unsigned kFloorBits = 0x4B000000u;

__device__ __forceinline__ void make_unit_consts(const FrameConst& fc, const SceneView& sv,
                                                 int lane, UnitConsts& K) {
  // lane -> stored voxels 4*lane + 128*i + j of slab i (i, j = 0..3), i.e.
  // lx = 4 (lane & 1) + j, lz = (lane >> 1) & 7, ly = (lane >> 4) + 2 i
  // (storage order x + 8 z + 64 y)
  const float lx0 = (float)(4 * (lane & 1));
  const float lz = (float)((lane >> 1) & 7);
  const float ly0 = (float)(lane >> 4);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    K.lbase[r] = fmaf(fc.A_hi[3 * r], lx0, fmaf(fc.A_hi[3 * r + 1], ly0, fc.A_hi[3 * r + 2] * lz));
    K.dk[r] = 2.0f * fc.A_hi[3 * r + 1];
  }
  K.dz = fc.A_hi[6];
  K.pdx = fc.fx * fc.A_hi[0];
  K.pdy = fc.fy * fc.A_hi[3];
  K.fx = fc.fx;
  K.fy = fc.fy;
  K.cxh = fc.cx + 0.5f;
  K.cyh = fc.cy + 0.5f;
  K.xlo = 1.5f;
  K.ylo = 1.5f;
  K.xhi = fc.xmax + 0.5f;
  K.yhi = fc.ymax + 0.5f;
  K.mu = fc.mu;
  K.inv_mu = fc.inv_mu;
  K.maxw4 = (unsigned)fc.max_weight * 0x01010101u;
  K.width = (unsigned)fc.width;
  K.off_bias = 0u - kFloorBits * ((unsigned)fc.width + 1u);  // modulo 2^32
  K.depth = sv.depth_san + fc.set * sv.depth_san_stride;
  K.sdf = sv.sdf;
  K.w = sv.w;
  K.pool = sv.pool;
  K.rgb = fc.rgb;
  K.rgbw = sv.rgbw;
}

// Colour of one voxel (bytes r, g, b, colour weight) after an observation o:
// per channel the listing's average (w c + o) / (w + 1), evaluated in float
// and rounded to the nearest integer, floor(fl(fl(N / D) + 1/2)) with
// N = w c + o, D = w + 1. N and D are small integers, so that is exactly the
// integer floor((2N + D) / (2D)): a fraction of N / D that is not 1/2 lies at
// least 1 / (2D) >= 1/512 from it, far beyond the two roundings (< 3e-5), and
// a tie is exact in float. The integer quotient is umulhi(2N + D, m) with
// m = ceil(2^32 / (2D)) (cinv[w]), exact for 2N + D < 2^17 because the
// reciprocal's excess stays below 2^-15 < 1/512. The colour weight becomes
// min(w + 1, maxW).
__device__ __forceinline__ unsigned colour_update(unsigned word, uchar4 o, unsigned maxw,
                                                  const unsigned* cinv) {
  const unsigned wc = word >> 24, D = wc + 1u, m = cinv[wc];
  const unsigned r = __umulhi(2u * (wc * (word & 0xffu) + o.x) + D, m);
  const unsigned g = __umulhi(2u * (wc * ((word >> 8) & 0xffu) + o.y) + D, m);
  const unsigned b = __umulhi(2u * (wc * ((word >> 16) & 0xffu) + o.z) + D, m);
  return r | (g << 8) | (b << 16) | (min(D, maxw) << 24);
}

// cinv[w] = ceil(2^32 / (2 (w + 1))) for the colour average
__device__ __forceinline__ void init_colour_table(unsigned* cinv) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) cinv[i] = 0xffffffffu / (2u * (i + 1)) + 1u;
}

// One lane's quad of voxel data: four sdf values (16 B f32 / 8 B) and their
// four weights (4 B).
template <int S>
__device__ __forceinline__ void load_quad(const typename Storage<S>::T* q, const unsigned* wq,
                                          typename Storage<S>::T* old, unsigned& w) {
  if constexpr (S == TSDF_STORAGE_F32) {
    const float4 t = *reinterpret_cast<const float4*>(q);
    old[0] = t.x; old[1] = t.y; old[2] = t.z; old[3] = t.w;
  } else {
    const uint2 t = *reinterpret_cast<const uint2*>(q);
    memcpy(old, &t, sizeof(t));
  }
  w = *wq;
}

// Slabs (8x8x2 voxels, a quad per lane) whose depth gathers and voxel loads
// are in flight together; a block is 4 slabs.
constexpr int kSlabsInFlight = 4;
// Load a slab group's voxel data before its depth gathers return: the two
// latencies overlap, at the cost of reading quads the rule then leaves alone
// (writes stay limited to updated quads).
constexpr bool kSpeculativeData = true;

// Integrate visible block b with one warp: 4 slabs x (a quad of 4 voxels
// along x) per lane, kSlabsInFlight slabs at a time. All depth gathers of a
// group of slabs are issued before any is used, and all their quads' voxel
// loads before any update; returns the number of voxels this lane updated.
// C: the scene keeps voxel colours (a new block's colours start at 0; when
// the frame has a colour image, every voxel rule U updates also averages the
// colour of its pixel).
template <int S, bool C = false>
__device__ __forceinline__ unsigned process_block(const UnitConsts& K, const VisRec& vr, int lane,
                                                  const float* s_rcp, SceneCounters* sc,
                                                  const unsigned* s_cinv = nullptr) {
  // a block handed out by this frame's allocation holds no data yet: its
  // voxels start from (initial sdf, weight 0) and every quad is written
  const bool fresh = vr.fresh != 0;
  using St = Storage<S>;
  using T = typename St::T;
  constexpr int G = kSlabsInFlight;
  constexpr int NV = 4 * G;  // voxels per lane per group
  if (vr.ptr < 0 || vr.ptr >= K.pool) {
    if (lane == 0) set_status(sc, kStInternal);  // inconsistent record: skip it
    return 0;
  }
  T* sdf_b = reinterpret_cast<T*>(K.sdf) + (size_t)vr.ptr * kBlockVoxels + 4 * lane;
  unsigned* w_b = reinterpret_cast<unsigned*>(K.w + (size_t)vr.ptr * kBlockVoxels + 4 * lane);
  unsigned updated = 0;
#pragma unroll 1
  for (int g = 0; g < 4; g += G) {
    // --- projections and depth gathers ----------------------------------
    unsigned off[NV];
    unsigned inb = 0;  // bit 4 i + j: voxel j of quad i projects inside
    float lz0[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const float fi = (float)(g + i);
      // the quad's first voxel: z keeps its low part (for eta), x and y are
      // only needed to float accuracy
      lz0[i] = vr.clo[2] + fmaf(fi, K.dk[2], K.lbase[2]);
      const float px = K.fx * (vr.chi[0] + (vr.clo[0] + fmaf(fi, K.dk[0], K.lbase[0])));
      const float py = K.fy * (vr.chi[1] + (vr.clo[1] + fmaf(fi, K.dk[1], K.lbase[1])));
      float x[4], y[4], Z[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        Z[j] = vr.chi[2] + fmaf((float)j, K.dz, lz0[i]);
        const float rz = rcp_approx(Z[j]);
        x[j] = fmaf(fmaf((float)j, K.pdx, px), rz, K.cxh);  // x + 1/2
        y[j] = fmaf(fmaf((float)j, K.pdy, py), rz, K.cyh);
      }
      // x and y are monotonic along the quad when z > 0 on it (a ratio of
      // affine functions), so the ends bound the four voxels
      const bool quad_in = fminf(Z[0], Z[3]) > 0.0f && fminf(x[0], x[3]) >= K.xlo &&
                           fmaxf(x[0], x[3]) <= K.xhi && fminf(y[0], y[3]) >= K.ylo &&
                           fmaxf(y[0], y[3]) <= K.yhi;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // nearest pixel: floor(x + 1/2), floor(y + 1/2) (x, y >= 1 inside)
        const unsigned ub = __float_as_uint(__fadd_rd(x[j], kFloorMagic));
        const unsigned vb = __float_as_uint(__fadd_rd(y[j], kFloorMagic));
        off[4 * i + j] = vb * K.width + ub + K.off_bias;
      }
      unsigned qin = 0xfu;
      if (!quad_in) {
        // border quads: test every voxel, read pixel 0 for those outside
        qin = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = Z[j] > 0.0f && x[j] >= K.xlo && x[j] <= K.xhi && y[j] >= K.ylo &&
                          y[j] <= K.yhi;
          qin |= in ? (1u << j) : 0u;
          off[4 * i + j] = in ? off[4 * i + j] : 0u;
        }
      }
      inb |= qin << (4 * i);
    }
    float d[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) d[k] = __ldg(K.depth + off[k]);
    uchar4 col[C ? NV : 1];
    if constexpr (C) {
      if (K.rgb) {
#pragma unroll
        for (int k = 0; k < NV; ++k) col[k] = __ldg(K.rgb + off[k]);
      }
    }
    T old[NV];
    unsigned w[G];
    if (fresh) {
#pragma unroll
      for (int k = 0; k < NV; ++k) old[k] = St::initial();
#pragma unroll
      for (int i = 0; i < G; ++i) w[i] = 0u;
    } else if constexpr (kSpeculativeData) {
#pragma unroll
      for (int i = 0; i < G; ++i)
        load_quad<S>(sdf_b + 128 * (g + i), w_b + 32 * (g + i), &old[4 * i], w[i]);
    }
    // --- rule U decisions -------------------------------------------------
    unsigned mask = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float eta = (d[4 * i + j] - vr.chi[2]) - fmaf((float)j, K.dz, lz0[i]);
        d[4 * i + j] = fminf(1.0f, eta * K.inv_mu);  // about -1e30 / mu where no measurement
        mask |= eta >= -K.mu ? (1u << (4 * i + j)) : 0u;
      }
    }
    mask &= inb;
    if (!mask && !fresh) continue;
    updated += (unsigned)__popc(mask);
    // --- voxel data: read every touched quad, then update and write ------
    if constexpr (!kSpeculativeData) {
      if (!fresh) {
#pragma unroll
        for (int i = 0; i < G; ++i)
          if ((mask >> (4 * i)) & 0xfu)
            load_quad<S>(sdf_b + 128 * (g + i), w_b + 32 * (g + i), &old[4 * i], w[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const unsigned qm = (mask >> (4 * i)) & 0xfu;
      if (!qm && !fresh) continue;
      const unsigned wq = w[i];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // F <- (w F + f) / (w + 1), evaluated as F + (f - F) / (w + 1);
        // computed for all four voxels, committed by select where updated
        const float F = St::load(old[4 * i + j]);
        const float Fn = fmaf(d[4 * i + j] - F, s_rcp[__byte_perm(wq, 0u, 0x4440u + j)], F);
        old[4 * i + j] = ((qm >> j) & 1u) ? St::store(Fn) : old[4 * i + j];
      }
      // w <- min(w + 1, maxW) for the updated voxels, four bytes at once:
      // stored weights never exceed maxW, so w < maxW iff the byte differs
      // from maxW (bytes of wq ^ maxW4 that are non-zero get a 1)
      const unsigned t = wq ^ K.maxw4;
      const unsigned nz = ((((t & 0x7f7f7f7fu) + 0x7f7f7f7fu) | t) >> 7) & 0x01010101u;
      const unsigned upd = (qm * 0x00204081u) & 0x01010101u;  // bit j -> byte j
      const unsigned wq_new = wq + (nz & upd);
      T* q = sdf_b + 128 * (g + i);
      if constexpr (S == TSDF_STORAGE_F32) {
        *reinterpret_cast<float4*>(q) =
            make_float4(old[4 * i], old[4 * i + 1], old[4 * i + 2], old[4 * i + 3]);
      } else {
        uint2 t;
        memcpy(&t, &old[4 * i], sizeof(t));
        *reinterpret_cast<uint2*>(q) = t;
      }
      w_b[32 * (g + i)] = wq_new;
      if constexpr (C) {
        if (fresh || K.rgb) {
          uint4* cq = reinterpret_cast<uint4*>(K.rgbw + (size_t)vr.ptr * kBlockVoxels + 4 * lane +
                                               128 * (g + i));
          uint4 cw = fresh ? make_uint4(0u, 0u, 0u, 0u) : *cq;
          if (K.rgb) {
            const unsigned maxw = K.maxw4 & 0xffu;
            if (qm & 1u) cw.x = colour_update(cw.x, col[4 * i], maxw, s_cinv);
            if (qm & 2u) cw.y = colour_update(cw.y, col[4 * i + 1], maxw, s_cinv);
            if (qm & 4u) cw.z = colour_update(cw.z, col[4 * i + 2], maxw, s_cinv);
            if (qm & 8u) cw.w = colour_update(cw.w, col[4 * i + 3], maxw, s_cinv);
          }
          *cq = cw;
        }
      }
    }
  }
  return updated;
}

__device__ __forceinline__ void init_rcp_table(float* s_rcp) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_rcp[i] = 1.0f / (float)(i + 1);
}



// The allocation results of the frame being integrated (its set).
struct FrameAlloc {
  int par;             // the frame's set
  int fresh_from;      // pool indices >= fresh_from were handed out this frame
  int high_water;      // allocated pool indices are [0, high_water)
  unsigned dmax_bits;  // largest measured depth of the frame (float bits)
  int n_new;           // blocks handed out this frame
};

// (The high-water mark comes from the frame's own commit, not from free_top,
// which the next frame's allocation may already be moving.)
__device__ __forceinline__ FrameAlloc frame_alloc(const SceneView& sv, int set) {
  FrameAlloc f;
  f.par = set;
  const AllocCounters* a = &sv.fc->a[set];
  f.fresh_from = sv.pool - __ldcg(&a->assign_base);
  f.n_new = __ldcg(&a->n_new);
  f.high_water = f.fresh_from + f.n_new;
  f.dmax_bits = __ldcg(&a->depth_max_bits);
  return f;
}

// Fold a frame's counts (blocks handed out, visible blocks, updated voxels)
// into its scene's counters and clear the frame's set (counters, and the
// pyramid levels built by atomics: level 0 is rewritten by every allocation
// tile). Run by one CTA after every CTA that integrated the frame has added
// its counts.
__device__ void close_frame_with(const FrameConst& fc, const SceneView& sv, int n_new, int vis,
                                 unsigned long long upd) {
  AllocCounters* a = &sv.fc->a[fc.set];
  if (threadIdx.x == 0) {
    SceneCounters* sc = sv.sc;
    sc->frames += 1;
    sc->last_new = (unsigned long long)n_new;
    sc->last_visible = (unsigned long long)vis;
    sc->last_updated = upd;
    sc->total_visible += (unsigned long long)vis;
    sc->total_updated += upd;
    a->n_new = 0;
    a->n_overflow = 0;
    a->assign_base = 0;
    a->depth_max_bits = 0u;
    a->alloc_done = 0;
    a->n_visible = 0;
    a->integ_arrive = 0;
    a->n_updated = 0ull;
    a->integ_packed = 0ull;
  }
  for (int i = threadIdx.x; i < kArriveGroups; i += blockDim.x) a->arrive[i] = 0;
  if (fc.use_tiles) {
    // every level (level 0 too: allocation tiles smaller than a cell build
    // it by atomicMax)
    unsigned* pyr = pyramid_set(sv, fc.set);
    int wl, hl;
    const int hi = pyramid_level(fc.tiles_x, fc.tiles_y, kPyramidLevels, wl, hl);
    for (int i = (int)threadIdx.x; i < hi; i += blockDim.x) pyr[i] = 0u;
  }
}

// The same with the counts read from the frame's set.
__device__ void close_frame(const FrameConst& fc, const SceneView& sv) {
  __shared__ int s_nn, s_vis;
  __shared__ unsigned long long s_u;
  const AllocCounters* a = &sv.fc->a[fc.set];
  if (threadIdx.x == 0) {
    s_nn = __ldcg(&a->n_new);
    s_vis = __ldcg(&a->n_visible);
    s_u = __ldcg(&a->n_updated);
  }
  __syncthreads();
  close_frame_with(fc, sv, s_nn, s_vis, s_u);
}

// Arrival of a CTA that has added its counts (thread 0 added them, or every
// thread that added some fenced them); returns true in the last one.
__device__ __forceinline__ bool last_to_arrive(int* counter, int n_ctas) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(counter, 1) == n_ctas - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Culling constants of a frame for the staged selection, built by every
// thread: the voxel box of a block is [0, 7]^3 lattice steps from its
// origin, so its camera-space corners are c0 + the sums of the columns of
// 7 A, and it lies inside the sphere around c0 + 3.5 A (1, 1, 1) of radius
// 3.5 sqrt(3) s. The four planes through the camera centre that bound the
// image rectangle grown by kSlackPx (unit normals, pointing inwards): a
// sphere entirely on the outer side of one holds no voxel that projects
// inside (nor any with z <= 0, which rule U skips).
struct StagedCull {
  float a7[9];     // 7 A, row-major (camera = rows)
  float half[3];   // 3.5 A (1, 1, 1)
  float radius;
  float pl[4][2];  // plane normals (n_x or n_y, n_z) of left, right, top, bottom
};

constexpr float kCullSlackZ = 1e-3f, kCullSlackPx = 1.0f;

__device__ __forceinline__ void make_staged_cull(const FrameConst& fc, StagedCull& C) {
#pragma unroll
  for (int i = 0; i < 9; ++i) C.a7[i] = 7.0f * fc.A_hi[i];
#pragma unroll
  for (int r = 0; r < 3; ++r) C.half[r] = 3.5f * (fc.A_hi[3 * r] + fc.A_hi[3 * r + 1] + fc.A_hi[3 * r + 2]);
  // |A column| = voxel size; a small relative margin covers the roundings
  C.radius = 3.5f * 1.7320508f * fc.voxel_size * 1.001f + 1e-5f;
  const float xl = 1.0f - kCullSlackPx, xr = fc.xmax + kCullSlackPx;
  const float yt = 1.0f - kCullSlackPx, yb = fc.ymax + kCullSlackPx;
  const float n[4][2] = {{fc.fx, fc.cx - xl}, {-fc.fx, xr - fc.cx},
                         {fc.fy, fc.cy - yt}, {-fc.fy, yb - fc.cy}};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float inv = rsqrtf(n[k][0] * n[k][0] + n[k][1] * n[k][1]);
    C.pl[k][0] = n[k][0] * inv;
    C.pl[k][1] = n[k][1] * inv;
  }
}

// Screen test of a block whose origin voxel has the (float) camera point c0:
// returns whether rule U can write any of its voxels (as block_visible) and
// sets `interior` when every voxel lies in front of the camera and projects
// at least kCullSlackPx inside the border [1, W-2] x [1, H-2]. With `test`
// false (a block new this frame, always integrated) only `interior` is
// computed.
__device__ __forceinline__ bool block_screen(const FrameConst& fc, const StagedCull& C,
                                             const unsigned* tile_max, bool pyr_shared,
                                             const float c0[3], float zfar, bool test,
                                             bool& interior) {
  interior = false;
  if (test) {
    // bounding sphere first: most allocated blocks leave the view here
    const float cx = c0[0] + C.half[0], cy = c0[1] + C.half[1], cz = c0[2] + C.half[2];
    if (cz + C.radius < -kCullSlackZ || cz - C.radius > zfar + kCullSlackZ) return false;
    if (fmaf(C.pl[0][0], cx, C.pl[0][1] * cz) < -C.radius ||
        fmaf(C.pl[1][0], cx, C.pl[1][1] * cz) < -C.radius ||
        fmaf(C.pl[2][0], cy, C.pl[2][1] * cz) < -C.radius ||
        fmaf(C.pl[3][0], cy, C.pl[3][1] * cz) < -C.radius)
      return false;
  }
  // the 8 corners: c0 plus the sums of the columns of 7 A
  float zmin = INFINITY, zmax = -INFINITY, xmin = INFINITY, xmax = -INFINITY,
        ymin = INFINITY, ymax = -INFINITY;
  bool front = true;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float X = c0[0], Y = c0[1], Z = c0[2];
    if (c & 1) { X += C.a7[0]; Y += C.a7[3]; Z += C.a7[6]; }
    if (c & 2) { X += C.a7[1]; Y += C.a7[4]; Z += C.a7[7]; }
    if (c & 4) { X += C.a7[2]; Y += C.a7[5]; Z += C.a7[8]; }
    zmin = fminf(zmin, Z);
    zmax = fmaxf(zmax, Z);
    if (Z < kCullSlackZ) {
      front = false;
    } else {
      const float rz = rcp_approx(Z);
      const float x = fmaf(fc.fx * X, rz, fc.cx), y = fmaf(fc.fy * Y, rz, fc.cy);
      xmin = fminf(xmin, x);
      xmax = fmaxf(xmax, x);
      ymin = fminf(ymin, y);
      ymax = fmaxf(ymax, y);
    }
  }
  interior = front && xmin >= 1.0f + kCullSlackPx && xmax <= fc.xmax - kCullSlackPx &&
             ymin >= 1.0f + kCullSlackPx && ymax <= fc.ymax - kCullSlackPx;
  if (!test) return true;
  if (zmax < -kCullSlackZ) return false;
  if (zmin > zfar + kCullSlackZ) return false;
  if (!front) return true;
  if (xmax < 1.0f - kCullSlackPx || xmin > fc.xmax + kCullSlackPx) return false;
  if (ymax < 1.0f - kCullSlackPx || ymin > fc.ymax + kCullSlackPx) return false;
  if (fc.use_tiles) {
    // the depth-max pyramid test of block_visible
    const int px0 = max(0, (int)floorf(xmin - kCullSlackPx));
    const int px1 = min(fc.width - 1, (int)ceilf(xmax + kCullSlackPx));
    const int py0 = max(0, (int)floorf(ymin - kCullSlackPx));
    const int py1 = min(fc.height - 1, (int)ceilf(ymax + kCullSlackPx));
    int l = 0;
    while (l < kPyramidLevels && (((px1 >> (4 + l)) - (px0 >> (4 + l))) > 1 ||
                                  ((py1 >> (4 + l)) - (py0 >> (4 + l))) > 1))
      ++l;
    if (l == kPyramidLevels) return true;
    int wl, hl;
    const int off = pyramid_level(fc.tiles_x, fc.tiles_y, l, wl, hl);
    const int cx0 = px0 >> (4 + l), cx1 = px1 >> (4 + l);
    const int cy0 = py0 >> (4 + l), cy1 = py1 >> (4 + l);
    auto cell = [&](int i) { return pyr_shared ? tile_max[i] : __ldcg(&tile_max[i]); };
    const unsigned m = max(max(cell(off + cy0 * wl + cx0), cell(off + cy0 * wl + cx1)),
                           max(cell(off + cy1 * wl + cx0), cell(off + cy1 * wl + cx1)));
    if (zmin > __uint_as_float(m) + fc.mu + kCullSlackZ) return false;
  }
  return true;
}

// Step 1 for allocated block `ptr`: does it need integrating, and its record
// (the same screen test as the staged kernels, so every kernel selects the
// same blocks).
__device__ __forceinline__ bool select_block(const FrameConst& fc, const SceneView& sv,
                                             const FrameAlloc& fa, int ptr, VisRec& r) {
  int bx, by, bz;
  unpack_key(__ldg(&sv.key_of_ptr[ptr]), bx, by, bz);
  const float o[3] = {8.0f * bx, 8.0f * by, 8.0f * bz};
  const bool fresh = ptr >= fa.fresh_from;
  bool vis = fresh;
  if (!vis && fa.dmax_bits != 0u) {
    float c0[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
      c0[q] = fmaf(fc.A_hi[3 * q], o[0],
                   fmaf(fc.A_hi[3 * q + 1], o[1], fmaf(fc.A_hi[3 * q + 2], o[2], fc.t_hi[q])));
    StagedCull C;
    make_staged_cull(fc, C);
    bool interior;
    vis = block_screen(fc, C, pyramid_set(sv, fa.par), false, c0,
                       __uint_as_float(fa.dmax_bits) + fc.mu, true, interior);
  }
  if (vis) {
    r.ptr = ptr;
    origin_df(fc, o, r.chi, r.clo);
    r.fresh = fresh ? 1 : 0;
  }
  return vis;
}

constexpr int kIntegThreads = 256;

// Steps 2-3 helpers: CTA-wide compaction of this pass's selected blocks into
// s_blk (returns their count); warps then take records by a shared counter.
__device__ __forceinline__ int compact_pass(bool sel, const VisRec& r, VisRec* s_blk,
                                            int* s_warp, int* s_total, int* s_next) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, sel);
  if (lane == 0) s_warp[warp] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const int c = s_warp[w];
      s_warp[w] = total;
      total += c;
    }
    *s_total = total;
    *s_next = 0;
  }
  __syncthreads();
  if (sel) s_blk[s_warp[warp] + __popc(bal & ((1u << lane) - 1u))] = r;
  __syncthreads();
  return *s_total;
}

__device__ __forceinline__ int grab_record(int* s_next, int lane) {
  int i = 0;
  if (lane == 0) i = atomicAdd(s_next, 1);
  return __shfl_sync(0xffffffffu, i, 0);
}

// (the colour path holds 16 more gathered values per lane: 2 CTAs per SM
// leave it the registers to do so without spilling)
template <int S, bool C>
__global__ void __launch_bounds__(kIntegThreads, C ? 2 : 3) integrate_kernel(FrameConst fc,
                                                                            SceneView sv) {
  __shared__ float s_rcp[256];  // s_rcp[w] = 1 / (w + 1), rounded once
  __shared__ unsigned s_cinv[C ? 256 : 1];
  __shared__ VisRec s_blk[kIntegThreads];
  __shared__ int s_warp[kIntegThreads / 32];
  __shared__ int s_total, s_next;
  __shared__ unsigned long long s_upd[kIntegThreads / 32];
  allow_dependents();
  init_rcp_table(s_rcp);
  if constexpr (C) init_colour_table(s_cinv);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  UnitConsts K;
  make_unit_consts(fc, sv, lane, K);
  wait_prior_grid();  // the allocation kernel's results
  const FrameAlloc fa = frame_alloc(sv, fc.set);
  unsigned long long updated = 0;
  int visible = 0;
  // block ptr is tested by CTA ptr % gridDim.x: neighbouring pool indices
  // (blocks of similar cost) spread over all CTAs
  const int per_pass = gridDim.x * blockDim.x;
  for (int base = blockIdx.x; base < fa.high_water; base += per_pass) {
    const int ptr = base + threadIdx.x * gridDim.x;
    VisRec r;
    const bool sel = ptr < fa.high_water && select_block(fc, sv, fa, ptr, r);
    const int nb = compact_pass(sel, r, s_blk, s_warp, &s_total, &s_next);
    visible += nb;
    for (int i = grab_record(&s_next, lane); i < nb; i = grab_record(&s_next, lane)) {
      const VisRec rec = s_blk[i];
      updated += process_block<S, C>(K, rec, lane, s_rcp, sv.sc, s_cinv);
    }
    __syncthreads();  // s_blk, s_warp and the counters are reused next pass
  }
  // one reduction per CTA, one (non-returning) atomic per counter and CTA
#pragma unroll
  for (int off = 16; off; off >>= 1) updated += __shfl_xor_sync(0xffffffffu, updated, off);
  if (lane == 0) s_upd[warp] = updated;
  __syncthreads();
  AllocCounters* a = &sv.fc->a[fc.set];
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_upd[w];
    if (t) atomicAdd(&a->n_updated, t);
    if (visible) atomicAdd(&a->n_visible, visible);
  }
  if (last_to_arrive(&a->integ_arrive, gridDim.x)) close_frame(fc, sv);
}

// ----------------------------------------------------------------------------
// Staged integration (one scene, depth only): the selection compacts the
// CTA's visible blocks into a shared-memory list; then every warp takes
// blocks from the list one at a time and keeps the voxel data of its next
// two blocks in flight: one lane issues bulk asynchronous copies of a
// block's sdf (2 KB f32, 1 KB 16-bit) and weights (512 B) into one of the
// warp's three shared-memory slots, completed on the slot's mbarrier. While
// those copies run, the warp projects its current block's voxels and
// gathers their depths, then waits for the block's slot and applies rule U,
// writing back only the quads it updates. Blocks whose screen box lies
// inside the image border skip the per-voxel border test; voxel pairs go
// through packed f32x2 arithmetic (two IEEE operations per instruction, the
// same roundings as the scalar form).

// CTA sizes: 512 threads (one CTA per SM) for a frame that has the GPU to
// itself, 256 when other kernels run beside it (a pipelined sequence runs
// the next frame's allocation at the same time).
constexpr int kStagedThreadsMax = 512;
constexpr int kStagedWarpsMax = kStagedThreadsMax / 32;
constexpr int kStagedSlots = 3;            // per warp: the current block + two in flight
constexpr int kStagedWaitPolls = 1 << 20;  // mbarrier polls before a wait gives up
constexpr int kStagedListCap = 1536;       // records of the CTA's visible-block list
constexpr int kStagedPyrWords = 6144;      // depth-max pyramid copy (images to ~1600 x 1200)
constexpr int kStagedKeyPrefetch = 3;      // candidate keys a thread loads up front (first round)

// the sanitised depth of a pixel without a measurement (finite, so that a
// voxel rule U leaves alone still computes finite values)
constexpr float kNoDepth = -1e30f;

// 1 when x >= 0 (+0 included), else 0, for |x| >= 2^-43 or x = 0: the
// product with 2^64 saturates to [0, 1] after the + 1
__device__ __forceinline__ float step01(float x) {
  float r;
  asm("fma.rn.sat.f32 %0, %1, 0f5F800000, 0f3F800000;" : "=f"(r) : "f"(x));
  return r;
}

// record flags
constexpr float kStagedMinMu = 1.0f / 1048576.0f;
constexpr int kRecFresh = 1;     // handed out by this frame's allocation
constexpr int kRecInterior = 2;  // every voxel projects inside [1, W-2] x [1, H-2]

// Arrivals, visible blocks and updated voxels of the staged kernel's CTAs in
// one 64-bit counter (pools below 2^22 blocks: visible < 2^22, updated <
// 2^31): one atomic per CTA tells the last one that it is last and the
// frame's totals.
constexpr int kPackArriveShift = 53, kPackVisShift = 31;
constexpr int kPackMaxPool = 1 << 22;

template <int S, int NT>
struct StagedGeom {
  static constexpr int kWarps = NT / 32;
  static constexpr int kSdfBytes = kBlockVoxels * (int)sizeof(typename Storage<S>::T);
  static constexpr int kSlotBytes = kSdfBytes + kBlockVoxels;  // sdf + weights
  // dynamic shared memory: rcp table | mbarriers | counters | pyramid barrier |
  // pyramid | list | slots
  static constexpr int kOffBar = 1024;
  static constexpr int kOffCtr = kOffBar + kWarps * kStagedSlots * 8;
  static constexpr int kOffPyrBar = 2040;
  static constexpr int kOffPyr = 2048;
  static constexpr int kOffList = kOffPyr + 4 * kStagedPyrWords;
  static constexpr int kOffSlots = kOffList + kStagedListCap * (int)sizeof(VisRec);
  static constexpr int kBytes = kOffSlots + kWarps * kStagedSlots * kSlotBytes;
};
static_assert(StagedGeom<TSDF_STORAGE_F32, kStagedThreadsMax>::kOffCtr + 32 +
                      8 * kStagedWarpsMax <= StagedGeom<TSDF_STORAGE_F32, kStagedThreadsMax>::kOffPyrBar,
              "shared layout");
static_assert(kStagedPyrWords % 4 == 0, "the pyramid copy moves whole 16-byte units");
static_assert(StagedGeom<TSDF_STORAGE_F32, kStagedThreadsMax>::kBytes <= 227 * 1024,
              "shared memory per CTA");

// Per-lane constants of the frame (the lane's quad: lx = 4 (lane & 1) + j,
// lz = (lane >> 1) & 7, ly = (lane >> 4) + 2 i in slab i, as in
// make_unit_consts).
struct StagedConsts {
  unsigned long long dbias;  // address of depth pixel 0 minus 4 x the offset bias
  unsigned off_bias;         // pixel offset of (0, 0) as computed from the floor bits
  unsigned width;
  void* sdf;
  unsigned char* w;
  int pool;
  float lbase[3], dk[3];
  float fx, fy;
  unsigned maxw4;
  f2 J01, J23;        // voxel indices along x of the two pairs of a quad
  f2 DZ, PDX, PDY;    // one voxel step along x: camera z, fx X, fy Y
  f2 CXH, CYH;        // cx + 1/2, cy + 1/2
  f2 MAG;             // 2^23 (floor by a round-down add)
  f2 INVMU, MU;       // 1 / mu, mu
  float xlo, xhi, ylo, yhi;  // x + 1/2 in [1.5, W - 1.5], y + 1/2 in [1.5, H - 1.5]
};

__device__ __forceinline__ void make_staged_consts(const FrameConst& fc, const SceneView& sv,
                                                   int lane, StagedConsts& K) {
  const float lx0 = (float)(4 * (lane & 1));
  const float lz = (float)((lane >> 1) & 7);
  const float ly0 = (float)(lane >> 4);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    K.lbase[r] = fmaf(fc.A_hi[3 * r], lx0, fmaf(fc.A_hi[3 * r + 1], ly0, fc.A_hi[3 * r + 2] * lz));
    K.dk[r] = 2.0f * fc.A_hi[3 * r + 1];
  }
  K.fx = fc.fx;
  K.fy = fc.fy;
  K.maxw4 = (unsigned)fc.max_weight * 0x01010101u;
  K.width = (unsigned)fc.width;
  // offset from the floor bits: vb * W + ub = v W + u + bias (mod 2^32), with
  // bias = 2^23-float bits x (W + 1) = k 2^24 for some k < 256; as W H < 2^24
  // the sum never wraps, so pixel (u, v) sits at dbias + 4 (vb W + ub)
  K.off_bias = kFloorBits * ((unsigned)fc.width + 1u);
  const float* depth = sv.depth_san + fc.set * sv.depth_san_stride;
  K.dbias = (unsigned long long)(uintptr_t)depth - 4ull * (unsigned long long)K.off_bias;
  K.sdf = sv.sdf;
  K.w = sv.w;
  K.pool = sv.pool;
  K.J01 = f2_make(0.0f, 1.0f);
  K.J23 = f2_make(2.0f, 3.0f);
  K.DZ = f2_dup(fc.A_hi[6]);
  K.PDX = f2_dup(fc.fx * fc.A_hi[0]);
  K.PDY = f2_dup(fc.fy * fc.A_hi[3]);
  K.CXH = f2_dup(fc.cx + 0.5f);
  K.CYH = f2_dup(fc.cy + 0.5f);
  K.MAG = f2_dup(kFloorMagic);
  K.INVMU = f2_dup(fc.inv_mu);
  K.MU = f2_dup(fc.mu);
  K.xlo = 1.5f;
  K.ylo = 1.5f;
  K.xhi = fc.xmax + 0.5f;
  K.yhi = fc.ymax + 0.5f;
}

// Selection of allocated block `ptr` (packed key `key`) with its record
// flags (see select_block).
__device__ __forceinline__ bool select_staged(const FrameConst& fc, const StagedCull& C,
                                              const FrameAlloc& fa, const unsigned* pyr,
                                              bool pyr_shared, int ptr, unsigned long long key,
                                              VisRec& r) {
  int bx, by, bz;
  unpack_key(key, bx, by, bz);
  const float o[3] = {8.0f * bx, 8.0f * by, 8.0f * bz};
  const bool fresh = ptr >= fa.fresh_from;
  bool interior = false, vis = fresh;
  if (fresh || fa.dmax_bits != 0u) {
    float c0[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
      c0[q] = fmaf(fc.A_hi[3 * q], o[0],
                   fmaf(fc.A_hi[3 * q + 1], o[1], fmaf(fc.A_hi[3 * q + 2], o[2], fc.t_hi[q])));
    vis = block_screen(fc, C, pyr, pyr_shared, c0, __uint_as_float(fa.dmax_bits) + fc.mu, !fresh,
                       interior);
    vis = vis || fresh;
  }
  if (vis) {
    r.ptr = ptr;
    origin_df(fc, o, r.chi, r.clo);
    r.fresh = (fresh ? kRecFresh : 0) | (interior ? kRecInterior : 0);
  }
  return vis;
}

// A fresh block (handed out by this frame's allocation) starts from the
// initial voxel state (sdf 1, weight 0). For float and int16 storage the
// slot receives that state by the same bulk copy as any other block, from
// the one-block images below, so the update itself needs no case for it;
// FP16 sets it in registers instead (measured: the copy is 1.6 % faster
// for float, 1.2 % for int16 and 1.2 % slower for FP16, frame by frame on
// the Kinect sequence).
template <int S>
constexpr bool kFreshCopy = S != TSDF_STORAGE_F16;

#define TSDF_REP8(x) x, x, x, x, x, x, x, x
#define TSDF_REP64(x) \
  TSDF_REP8(x), TSDF_REP8(x), TSDF_REP8(x), TSDF_REP8(x), TSDF_REP8(x), TSDF_REP8(x), \
      TSDF_REP8(x), TSDF_REP8(x)
#define TSDF_REP512(x) \
  TSDF_REP64(x), TSDF_REP64(x), TSDF_REP64(x), TSDF_REP64(x), TSDF_REP64(x), TSDF_REP64(x), \
      TSDF_REP64(x), TSDF_REP64(x)
__device__ __align__(128) const float g_fresh_sdf_f32[kBlockVoxels] = {TSDF_REP512(1.0f)};
__device__ __align__(128) const short g_fresh_sdf_i16[kBlockVoxels] = {TSDF_REP512(32767)};
__device__ __align__(128) const unsigned char g_fresh_w[kBlockVoxels] = {};
#undef TSDF_REP512
#undef TSDF_REP64
#undef TSDF_REP8

// One lane issues the bulk copies of a block's voxel data (the scene's sdf
// and weight arrays, `pool` blocks) into a slot: the block's own, or the
// initial state for a fresh block (none when the form sets it in registers).
template <int S>
__device__ __forceinline__ void stage_block(const void* sdf, const unsigned char* w, int pool,
                                            const VisRec* rec, unsigned char* slot,
                                            unsigned long long* bar) {
  using G = StagedGeom<S, kStagedThreadsMax>;
  const int ptr = rec->ptr;
  if (ptr < 0 || ptr >= pool) return;
  const void* src_sdf = reinterpret_cast<const unsigned char*>(sdf) + (size_t)ptr * G::kSdfBytes;
  const unsigned char* src_w = w + (size_t)ptr * kBlockVoxels;
  if (rec->fresh & kRecFresh) {
    if constexpr (!kFreshCopy<S>) return;
    src_sdf = S == TSDF_STORAGE_F32 ? static_cast<const void*>(g_fresh_sdf_f32)
                                    : static_cast<const void*>(g_fresh_sdf_i16);
    src_w = g_fresh_w;
  }
  mbar_arrive_expect_tx(bar, G::kSlotBytes);
  bulk_g2s(slot, src_sdf, G::kSdfBytes, bar);
  bulk_g2s(slot + G::kSdfBytes, src_w, kBlockVoxels, bar);
}

// Two stored values (elements 0 and 1 of `v`) as a float pair, and back:
// the same values as Storage<S>::load / store element by element, in fewer
// instructions. int16: the pair's bits, each with its top bit flipped, sit
// in the low half of 2^23 (float bits 0x4B000000), so the float is 2^23 +
// 2^15 + q exactly; one packed subtraction and one packed multiply give
// both q / 32767 values as Storage<I16>::load does. FP16: one packed
// round-to-nearest conversion stores both.
template <int S>
__device__ __forceinline__ f2 load_pair(const typename Storage<S>::T* v) {
  if constexpr (S == TSDF_STORAGE_I16) {
    unsigned b;
    memcpy(&b, v, 4);
    b ^= 0x80008000u;
    const f2 q = f2_sub(f2_make(__uint_as_float(__byte_perm(b, kFloorBits, 0x7610)),
                                __uint_as_float(__byte_perm(b, kFloorBits, 0x7632))),
                        f2_dup(8421376.0f));
    return f2_mul(q, f2_dup(__uint_as_float(0x38000101u)));
  } else {
    return f2_make(Storage<S>::load(v[0]), Storage<S>::load(v[1]));
  }
}

template <int S>
__device__ __forceinline__ void store_pair(f2 x, typename Storage<S>::T* v) {
  if constexpr (S == TSDF_STORAGE_I16) {
    const f2 t = f2_mul(x, f2_dup(32767.0f));
    const unsigned b = __byte_perm((unsigned)__float2int_rz(f2_lo(t)),
                                   (unsigned)__float2int_rz(f2_hi(t)), 0x5410);
    memcpy(v, &b, 4);
  } else if constexpr (S == TSDF_STORAGE_F16) {
    unsigned b;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(b) : "f"(f2_hi(x)), "f"(f2_lo(x)));
    memcpy(v, &b, 4);
  } else {
    v[0] = f2_lo(x);
    v[1] = f2_hi(x);
  }
}

// Rule U for one block with one warp; the lane's 16 voxels are 4 slabs x a
// quad of 4 along x, as in process_block. The depth gathers are issued
// before the wait for the block's staged data. Every voxel's update flag
// u (1 when eta >= -mu, else 0) is a float that scales the weight
// reciprocal: a voxel with u = 0 gets F + (f - F) * 0 = F, bit for bit
// (f is finite: no measurement reads as kNoDepth), and every storage form's
// store(load(x)) is x, so no select is needed. The quads are
// processed without branches; stores are skipped for quads with no update
// (all quads of a fresh block are written). `ok` turns false when the wait
// for the staged data gives up (the block is then left unchanged). Returns
// the number of voxels this lane updated.
template <int S, bool kInterior>
__device__ __forceinline__ unsigned staged_block(const StagedConsts& K, const VisRec& vr,
                                                 bool fresh, int lane, const unsigned char* slot,
                                                 unsigned long long* bar, unsigned parity,
                                                 const float* s_rcp, bool& ok) {
  using St = Storage<S>;
  using T = typename St::T;
  using G = StagedGeom<S, kStagedThreadsMax>;
  // --- projections and depth gathers of the lane's 16 voxels ------------
  float d[16];
  float zl[4];  // z offset of the quad's first voxel from the block origin (hi part excluded)
  const f2 CHIZ = f2_dup(vr.chi[2]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float fi = (float)i;
    zl[i] = vr.clo[2] + fmaf(fi, K.dk[2], K.lbase[2]);
    float px, py;
    if constexpr (S == TSDF_STORAGE_F32) {
      // x and y as one pair (the same roundings; 1.2 % faster for float,
      // 1.2 % slower for int16, whose registers it crowds)
      const f2 P = f2_mul(f2_make(K.fx, K.fy),
                          f2_add(f2_make(vr.chi[0], vr.chi[1]),
                                 f2_add(f2_make(vr.clo[0], vr.clo[1]),
                                        f2_fma(f2_dup(fi), f2_make(K.dk[0], K.dk[1]),
                                               f2_make(K.lbase[0], K.lbase[1])))));
      px = f2_lo(P);
      py = f2_hi(P);
    } else {
      px = K.fx * (vr.chi[0] + (vr.clo[0] + fmaf(fi, K.dk[0], K.lbase[0])));
      py = K.fy * (vr.chi[1] + (vr.clo[1] + fmaf(fi, K.dk[1], K.lbase[1])));
    }
    const f2 ZL = f2_dup(zl[i]), PX = f2_dup(px), PY = f2_dup(py);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const f2 J = p ? K.J23 : K.J01;
      const f2 Z = f2_add(CHIZ, f2_fma(J, K.DZ, ZL));
      const float Z0 = f2_lo(Z), Z1 = f2_hi(Z);
      const f2 RZ = f2_make(rcp_approx(Z0), rcp_approx(Z1));
      const f2 X = f2_fma(f2_fma(J, K.PDX, PX), RZ, K.CXH);  // x + 1/2
      const f2 Y = f2_fma(f2_fma(J, K.PDY, PY), RZ, K.CYH);
      const f2 UB = f2_add_rd(X, K.MAG), VB = f2_add_rd(Y, K.MAG);
      const unsigned o0 = __float_as_uint(f2_lo(VB)) * K.width + __float_as_uint(f2_lo(UB));
      const unsigned o1 = __float_as_uint(f2_hi(VB)) * K.width + __float_as_uint(f2_hi(UB));
      if constexpr (kInterior) {
        d[4 * i + 2 * p] = __ldg(reinterpret_cast<const float*>(K.dbias + 4ull * o0));
        d[4 * i + 2 * p + 1] = __ldg(reinterpret_cast<const float*>(K.dbias + 4ull * o1));
      } else {
        // border block: a voxel outside [1, W-2] x [1, H-2] (or behind the
        // camera) reads no depth
        const float x0 = f2_lo(X), x1 = f2_hi(X), y0 = f2_lo(Y), y1 = f2_hi(Y);
        const bool in0 = Z0 > 0.0f && x0 >= K.xlo && x0 <= K.xhi && y0 >= K.ylo && y0 <= K.yhi;
        const bool in1 = Z1 > 0.0f && x1 >= K.xlo && x1 <= K.xhi && y1 >= K.ylo && y1 <= K.yhi;
        d[4 * i + 2 * p] =
            in0 ? __ldg(reinterpret_cast<const float*>(K.dbias + 4ull * o0)) : kNoDepth;
        d[4 * i + 2 * p + 1] =
            in1 ? __ldg(reinterpret_cast<const float*>(K.dbias + 4ull * o1)) : kNoDepth;
      }
    }
  }
  // the staged voxel data (all lanes wait: the slot is reused afterwards)
  if (kFreshCopy<S> || !fresh) {
    ok = mbar_wait_bounded(bar, parity, kStagedWaitPolls);
    if (!ok) return 0;
  }
  const T* s_sdf = reinterpret_cast<const T*>(slot) + 4 * lane;
  const unsigned* s_w = reinterpret_cast<const unsigned*>(slot + G::kSdfBytes) + lane;
  T* g_sdf = reinterpret_cast<T*>(K.sdf) + (size_t)vr.ptr * kBlockVoxels + 4 * lane;
  unsigned* g_w = reinterpret_cast<unsigned*>(K.w + (size_t)vr.ptr * kBlockVoxels) + lane;
  unsigned cnt = 0;  // updated voxels, one byte lane per voxel of a quad
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // --- rule U decisions of quad i -------------------------------------
    const f2 ZL = f2_dup(zl[i]);
    float f[4], u[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const f2 z = f2_fma(p ? K.J23 : K.J01, K.DZ, ZL);
      const f2 ETA = f2_sub(f2_sub(f2_make(d[4 * i + 2 * p], d[4 * i + 2 * p + 1]), CHIZ), z);
      const f2 FR = f2_mul(ETA, K.INVMU);
      const f2 SM = f2_add(ETA, K.MU);  // >= 0 exactly when eta >= -mu
      f[2 * p] = fminf(1.0f, f2_lo(FR));
      f[2 * p + 1] = fminf(1.0f, f2_hi(FR));
      u[2 * p] = step01(f2_lo(SM));
      u[2 * p + 1] = step01(f2_hi(SM));
    }
    // update bytes: byte j = 1 when voxel j is updated (byte 2 of 1.0f has
    // its top bit set; sign-replicating permutes gather it)
    const unsigned upd =
        (prmt_sign(__float_as_uint(u[0]), __float_as_uint(u[1]), 0x00EAu) |
         prmt_sign(__float_as_uint(u[2]), __float_as_uint(u[3]), 0xEA00u)) & 0x01010101u;
    cnt += upd;
    // the quad's voxel data: staged, or the initial state of a fresh block
    T old[4];
    unsigned wq;
    load_quad<S>(s_sdf + 128 * i, s_w + 32 * i, old, wq);
    if (!kFreshCopy<S> && fresh) {
#pragma unroll
      for (int j = 0; j < 4; ++j) old[j] = St::initial();
      wq = 0u;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      // F <- F + (f - F) u / (w + 1), both voxels of the pair at once, with
      // 1 / (w + 1) rounded once (the table)
      const f2 R = f2_mul(f2_make(u[2 * p], u[2 * p + 1]),
                          f2_make(s_rcp[__byte_perm(wq, 0u, 0x4440u + 2 * p)],
                                  s_rcp[__byte_perm(wq, 0u, 0x4441u + 2 * p)]));
      const f2 F = load_pair<S>(old + 2 * p);
      store_pair<S>(f2_fma(f2_sub(f2_make(f[2 * p], f[2 * p + 1]), F), R, F), old + 2 * p);
    }
    // w <- min(w + 1, maxW) for the updated voxels, four bytes at once:
    // stored weights never exceed maxW, so w < maxW iff the byte differs
    // from maxW (bytes of wq ^ maxW4 that are non-zero get a 1)
    const unsigned t = wq ^ K.maxw4;
    const unsigned nz = ((((t & 0x7f7f7f7fu) + 0x7f7f7f7fu) | t) >> 7) & upd;
    if (upd | (unsigned)fresh) {
      T* q = g_sdf + 128 * i;
      if constexpr (S == TSDF_STORAGE_F32) {
        *reinterpret_cast<float4*>(q) = make_float4(old[0], old[1], old[2], old[3]);
      } else {
        uint2 v;
        memcpy(&v, old, sizeof(v));
        *reinterpret_cast<uint2*>(q) = v;
      }
      g_w[32 * i] = wq + nz;
    }
  }
  return (cnt * 0x01010101u) >> 24;
}

// Registers: 128 at 512 threads (the whole register file). At 256 threads
// (beside another kernel) float storage stays at 128, leaving half of the
// SM's registers to the allocation CTAs; the 16-bit forms, whose conversions
// hold more values, take what they need (measured on the pipelined Kinect
// sequence: 34.9 instead of 41.6 us per frame for int16, while float storage
// is 31.7 us capped and 35.9 us uncapped).
template <int S, int NT>
constexpr int staged_min_blocks() {
  return NT == kStagedThreadsMax ? 1 : (S == TSDF_STORAGE_F32 ? kStagedThreadsMax / NT : 1);
}

template <int S, int NT>
__global__ void __launch_bounds__(NT, (staged_min_blocks<S, NT>())) integrate_staged_kernel(
    FrameConst fc, SceneView sv) {
  using G = StagedGeom<S, NT>;
  extern __shared__ __align__(128) unsigned char smem[];
  float* s_rcp = reinterpret_cast<float*>(smem);  // s_rcp[w] = 1 / (w + 1), rounded once
  unsigned long long* s_bar = reinterpret_cast<unsigned long long*>(smem + G::kOffBar);
  // [0] list size, [1] next record, [2] last CTA, [3] total visible
  int* s_ctr = reinterpret_cast<int*>(smem + G::kOffCtr);
  unsigned long long* s_tot = reinterpret_cast<unsigned long long*>(smem + G::kOffCtr + 16);
  unsigned long long* s_upd = reinterpret_cast<unsigned long long*>(smem + G::kOffCtr + 32);
  unsigned* s_pyr = reinterpret_cast<unsigned*>(smem + G::kOffPyr);
  unsigned long long* s_pyrbar = reinterpret_cast<unsigned long long*>(smem + G::kOffPyrBar);
  VisRec* s_list = reinterpret_cast<VisRec*>(smem + G::kOffList);
  unsigned char* s_slots = smem + G::kOffSlots;
  allow_dependents();
  init_rcp_table(s_rcp);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < G::kWarps * kStagedSlots) mbar_init(&s_bar[threadIdx.x], 1);
  if (threadIdx.x == 0) {
    s_ctr[0] = 0;
    s_ctr[1] = 0;
  }
  mbar_init_fence();
  StagedConsts K;
  make_staged_consts(fc, sv, lane, K);
  const int G_ = gridDim.x, T_ = blockDim.x;
  const int first = blockIdx.x;
  wait_prior_grid();  // the allocation kernel's results
  // one round trip for everything the selection needs: the frame's
  // allocation counts, the depth-max pyramid (copied to shared memory when
  // it fits) and the first candidate keys (loaded for every in-pool index;
  // those beyond the frame's high-water mark are ignored)
  unsigned long long key_pre[kStagedKeyPrefetch];
#pragma unroll
  for (int k = 0; k < kStagedKeyPrefetch; ++k) {
    const int ptr = first + G_ * (threadIdx.x + T_ * k);
    key_pre[k] = ptr < sv.pool ? __ldcg(&sv.key_of_ptr[ptr]) : kKeyEmpty;
  }
  const FrameAlloc fa = frame_alloc(sv, fc.set);
  const unsigned* g_pyr = pyramid_set(sv, fc.set);
  int pyr_words = 0;
  if (fc.use_tiles) {
    int wl, hl;
    pyr_words = pyramid_level(fc.tiles_x, fc.tiles_y, kPyramidLevels, wl, hl);
  }
  const bool pyr_shared = pyr_words <= kStagedPyrWords;
  // The selection's culling constants: built once here, or (FP16, whose
  // conversions hold more values) rebuilt per round inside the selection,
  // which keeps its processing loop out of local memory.
  constexpr bool kCullPerRound = S == TSDF_STORAGE_F16;
  StagedCull C0;
  if constexpr (!kCullPerRound) make_staged_cull(fc, C0);
  // the pyramid arrives by one bulk copy (whole 16-byte units: the set holds
  // 2 kTileCap words, far more than kStagedPyrWords, a multiple of 4)
  const bool pyr_copy = pyr_shared && pyr_words > 0;
  if (pyr_copy && threadIdx.x == 0) {
    mbar_init(s_pyrbar, 1);
    mbar_init_fence();
    const unsigned bytes = (unsigned)((pyr_words + 3) & ~3) * 4u;
    mbar_arrive_expect_tx(s_pyrbar, bytes);
    bulk_g2s(s_pyr, g_pyr, bytes, s_pyrbar);
  }
  const unsigned* pyr = pyr_shared ? s_pyr : g_pyr;
  __syncthreads();
  if (pyr_copy && !mbar_wait_bounded(s_pyrbar, 0, kStagedWaitPolls) && threadIdx.x == 0)
    set_status(sv.sc, kStTimeout);
  unsigned long long updated = 0;
  int visible = 0;
  bool ok = true;
  unsigned phase = 0;  // bit s: parity of the next completion of this warp's slot s
  unsigned long long* bar = s_bar + warp * kStagedSlots;
  unsigned char* slots = s_slots + (size_t)warp * kStagedSlots * G::kSlotBytes;
  // candidate iteration k tests pool block first + G (threadIdx.x + T k)
  const int n_iter =
      fa.high_water > first ? (fa.high_water - first + G_ * T_ - 1) / (G_ * T_) : 0;
  const int iters_per_round = kStagedListCap / T_;
  for (int k0 = 0; k0 < n_iter; k0 += iters_per_round) {
    const int k1 = min(n_iter, k0 + iters_per_round);
    // --- 1. selection into the list --------------------------------------
    StagedCull C = C0;
    if constexpr (kCullPerRound) make_staged_cull(fc, C);
    for (int k = k0; k < k1; ++k) {
      const int ptr = first + G_ * (threadIdx.x + T_ * k);
      VisRec r;
      bool sel = false;
      if (ptr < fa.high_water) {
        unsigned long long key = kKeyEmpty;
#pragma unroll
        for (int j = 0; j < kStagedKeyPrefetch; ++j)
          if (j == k) key = key_pre[j];
        if (k >= kStagedKeyPrefetch) key = __ldcg(&sv.key_of_ptr[ptr]);
        sel = select_staged(fc, C, fa, pyr, pyr_shared, ptr, key, r);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, sel);
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(&s_ctr[0], __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (sel) s_list[base + __popc(bal & ((1u << lane) - 1u))] = r;
    }
    __syncthreads();
    const int n = s_ctr[0];
    visible += n;
    // --- 2. integration: warps take records in order -----------------------
    auto grab = [&]() {
      int i = 0;
      if (lane == 0) i = atomicAdd(&s_ctr[1], 1);
      i = __shfl_sync(0xffffffffu, i, 0);
      return i < n ? i : -1;
    };
    int r0 = grab(), r1 = grab();
    int sl0 = 0, sl1 = 1, sl2 = 2;
    if (lane == 0) {
      if (r0 >= 0) stage_block<S>(K.sdf, K.w, K.pool, &s_list[r0], slots + sl0 * G::kSlotBytes, bar + sl0);
      if (r1 >= 0) stage_block<S>(K.sdf, K.w, K.pool, &s_list[r1], slots + sl1 * G::kSlotBytes, bar + sl1);
    }
    while (r0 >= 0) {
      const int r2 = ok ? grab() : -1;
      if (lane == 0 && r2 >= 0)
        stage_block<S>(K.sdf, K.w, K.pool, &s_list[r2], slots + sl2 * G::kSlotBytes, bar + sl2);
      const VisRec rec = s_list[r0];
      const bool fresh = (rec.fresh & kRecFresh) != 0;
      const bool valid = rec.ptr >= 0 && rec.ptr < K.pool;
      if (valid && ok) {
        const unsigned par = (phase >> sl0) & 1u;
        const unsigned char* slot = slots + sl0 * G::kSlotBytes;
        updated += (rec.fresh & kRecInterior)
                       ? staged_block<S, true>(K, rec, fresh, lane, slot, bar + sl0, par, s_rcp, ok)
                       : staged_block<S, false>(K, rec, fresh, lane, slot, bar + sl0, par, s_rcp, ok);
        if (kFreshCopy<S> || !fresh) phase ^= 1u << sl0;
      } else if (!valid && lane == 0) {
        set_status(sv.sc, kStInternal);  // inconsistent record: skip it
      }
      // every lane has consumed the slot (its shared loads completed into
      // registers) before lane 0 refills it
      ok = __all_sync(0xffffffffu, ok);
      r0 = r1;
      r1 = r2;
      const int t = sl0;
      sl0 = sl1;
      sl1 = sl2;
      sl2 = t;
    }
    if (!ok) {
      // a wait gave up: let the copies still in flight land before the CTA
      // leaves (bounded again), and report the timeout
      if (lane == 0) set_status(sv.sc, kStTimeout);
      for (int s = 0; s < kStagedSlots; ++s)
        mbar_wait_bounded(bar + s, (phase >> s) & 1u, kStagedWaitPolls);
    }
    __syncthreads();  // the list and its counters are reused next round
    if (threadIdx.x == 0) {
      s_ctr[0] = 0;
      s_ctr[1] = 0;
    }
    __syncthreads();
  }
  // the CTA's counts: one atomic (packed with the arrival) per CTA
#pragma unroll
  for (int off = 16; off; off >>= 1) updated += __shfl_xor_sync(0xffffffffu, updated, off);
  if (lane == 0) s_upd[warp] = updated;
  __syncthreads();
  AllocCounters* a = &sv.fc->a[fc.set];
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < G::kWarps; ++w) t += s_upd[w];
    int last = 0;
    if (sv.pool < kPackMaxPool) {
      const unsigned long long mine = (1ull << kPackArriveShift) |
                                      ((unsigned long long)visible << kPackVisShift) | t;
      const unsigned long long all = atomicAdd(&a->integ_packed, mine) + mine;
      last = (int)(all >> kPackArriveShift) == G_;
      s_ctr[3] = (int)((all >> kPackVisShift) & ((1ull << (kPackArriveShift - kPackVisShift)) - 1));
      s_tot[0] = all & ((1ull << kPackVisShift) - 1);
    } else {
      if (t) atomicAdd(&a->n_updated, t);
      if (visible) atomicAdd(&a->n_visible, visible);
      __threadfence();
      last = atomicAdd(&a->integ_arrive, 1) == G_ - 1;
      if (last) {
        __threadfence();
        s_ctr[3] = __ldcg(&a->n_visible);
        s_tot[0] = __ldcg(&a->n_updated);
      }
    }
    s_ctr[2] = last;
  }
  __syncthreads();
  if (s_ctr[2]) {
    __threadfence();
    close_frame_with(fc, sv, fa.n_new, s_ctr[3], s_tot[0]);
  }
}

// ----------------------------------------------------------------------------
// Staged batched integration: one CTA per SM for a batch of scenes. The
// allocated blocks of every scene of this storage form are one range
// (scene i owns [hw[i], hw[i + 1])); each CTA selects its interleaved share
// of the range into its shared-memory list of (scene, block) records (the
// scene's slot in the record's flags) and its warps take records from that
// list with the staged pipeline of the single-scene kernel: a warp rebuilds
// its per-scene constants when a record belongs to another scene than the
// last one, and lane 0 stages each block from its own scene's arrays.
// Counts are kept per scene in shared memory; the last CTA closes every
// scene's frame.
constexpr int kRecSlotShift = 8;  // record flags: scene slot << 8 | fresh | interior

template <int S, int NT>
struct StagedBatchGeom {
  using B = StagedGeom<S, NT>;
  // rcp table | mbarriers | counters | scene prefix | counts | allocations |
  // list | slots
  static constexpr int kOffBar = 1024;
  static constexpr int kOffCtr = kOffBar + B::kWarps * kStagedSlots * 8;
  static constexpr int kOffHw = 2048;
  static constexpr int kOffUpd = kOffHw + 4 * (kMaxBatch + 2);
  static constexpr int kOffVis = kOffUpd + 8 * kMaxBatch;
  static constexpr int kOffFa = kOffVis + 4 * kMaxBatch;
  static constexpr int kOffList = (kOffFa + (int)sizeof(FrameAlloc) * kMaxBatch + 127) / 128 * 128;
  static constexpr int kOffSlots = kOffList + kStagedListCap * (int)sizeof(VisRec);
  static constexpr int kBytes = kOffSlots + B::kWarps * kStagedSlots * B::kSlotBytes;
};
static_assert(StagedBatchGeom<TSDF_STORAGE_F32, kStagedThreadsMax>::kOffCtr + 16 <= 2048,
              "shared layout");
static_assert(StagedBatchGeom<TSDF_STORAGE_F32, kStagedThreadsMax>::kBytes <= 227 * 1024,
              "shared memory per CTA");

template <int S, int NT>
__global__ void __launch_bounds__(NT, (staged_min_blocks<S, NT>())) integrate_batch_staged_kernel(
    const SlotDesc* slots, int n) {
  using G = StagedBatchGeom<S, NT>;
  using B = StagedGeom<S, NT>;
  extern __shared__ __align__(128) unsigned char smem[];
  float* s_rcp = reinterpret_cast<float*>(smem);
  unsigned long long* s_bar = reinterpret_cast<unsigned long long*>(smem + G::kOffBar);
  int* s_ctr = reinterpret_cast<int*>(smem + G::kOffCtr);  // list size, next record, last CTA
  int* s_hw = reinterpret_cast<int*>(smem + G::kOffHw);
  unsigned long long* s_upd = reinterpret_cast<unsigned long long*>(smem + G::kOffUpd);
  int* s_vis = reinterpret_cast<int*>(smem + G::kOffVis);
  FrameAlloc* s_fa = reinterpret_cast<FrameAlloc*>(smem + G::kOffFa);
  VisRec* s_list = reinterpret_cast<VisRec*>(smem + G::kOffList);
  unsigned char* s_slots = smem + G::kOffSlots;
  allow_dependents();
  init_rcp_table(s_rcp);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < B::kWarps * kStagedSlots) mbar_init(&s_bar[threadIdx.x], 1);
  if (threadIdx.x == 0) {
    s_ctr[0] = 0;
    s_ctr[1] = 0;
    s_hw[0] = 0;
  }
  mbar_init_fence();
  wait_prior_grid();  // the allocation kernel's results
  // every scene's allocation results; a scene of another storage form owns
  // no part of the range
  for (int i = threadIdx.x; i < n; i += NT) {
    const FrameAlloc fa = frame_alloc(slots[i].sv, slots[i].fc.set);
    s_fa[i] = fa;
    s_hw[i + 1] = slots[i].sv.storage == S ? fa.high_water : 0;
    s_upd[i] = 0ull;
    s_vis[i] = 0;
  }
  __syncthreads();
  if (warp == 0) {  // inclusive prefix of s_hw[1..n], 32 at a time
    int carry = 0;
    for (int b = 0; b < n; b += 32) {
      int v = b + lane < n ? s_hw[b + lane + 1] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (b + lane < n) s_hw[b + lane + 1] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  const int total = s_hw[n];
  const int G_ = gridDim.x;
  const int first = blockIdx.x;
  const int n_iter = total > first ? (total - first + G_ * NT - 1) / (G_ * NT) : 0;
  const int iters_per_round = kStagedListCap / NT;
  bool ok = true;
  unsigned phase = 0;
  unsigned long long* bar = s_bar + warp * kStagedSlots;
  unsigned char* wslots = s_slots + (size_t)warp * kStagedSlots * B::kSlotBytes;
  int kslot = -1;  // the scene whose constants K holds (warp-uniform)
  StagedConsts K;
  for (int k0 = 0; k0 < n_iter; k0 += iters_per_round) {
    const int k1 = min(n_iter, k0 + iters_per_round);
    // --- 1. selection into the list (records carry their scene) -----------
    for (int k = k0; k < k1; ++k) {
      const int g = first + G_ * (threadIdx.x + NT * k);
      VisRec r;
      bool sel = false;
      int slot = 0;
      if (g < total) {
        int lo = 0, hi = n - 1;  // last scene with s_hw[scene] <= g
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_hw[mid] <= g) lo = mid; else hi = mid - 1;
        }
        slot = lo;
        const SlotDesc* d = &slots[slot];
        const int ptr = g - s_hw[slot];
        StagedCull C;
        make_staged_cull(d->fc, C);
        sel = select_staged(d->fc, C, s_fa[slot], pyramid_set(d->sv, s_fa[slot].par), false, ptr,
                            __ldcg(&d->sv.key_of_ptr[ptr]), r);
        if (sel) {
          r.fresh |= slot << kRecSlotShift;
          atomicAdd(&s_vis[slot], 1);
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, sel);
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(&s_ctr[0], __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (sel) s_list[base + __popc(bal & ((1u << lane) - 1u))] = r;
    }
    __syncthreads();
    const int nl = s_ctr[0];
    // --- 2. integration ---------------------------------------------------
    auto grab = [&]() {
      int i = 0;
      if (lane == 0) i = atomicAdd(&s_ctr[1], 1);
      i = __shfl_sync(0xffffffffu, i, 0);
      return i < nl ? i : -1;
    };
    auto stage = [&](int r, int sl) {
      const VisRec* rec = &s_list[r];
      const SceneView& sv = slots[rec->fresh >> kRecSlotShift].sv;
      stage_block<S>(sv.sdf, sv.w, sv.pool, rec, wslots + sl * B::kSlotBytes, bar + sl);
    };
    int r0 = grab(), r1 = grab();
    int sl0 = 0, sl1 = 1, sl2 = 2;
    if (lane == 0) {
      if (r0 >= 0) stage(r0, sl0);
      if (r1 >= 0) stage(r1, sl1);
    }
    while (r0 >= 0) {
      const int r2 = ok ? grab() : -1;
      if (lane == 0 && r2 >= 0) stage(r2, sl2);
      const VisRec rec = s_list[r0];
      const int bs = rec.fresh >> kRecSlotShift;
      if (bs != kslot) {
        kslot = bs;
        make_staged_consts(slots[bs].fc, slots[bs].sv, lane, K);
      }
      const bool fresh = (rec.fresh & kRecFresh) != 0;
      const bool valid = rec.ptr >= 0 && rec.ptr < K.pool;
      unsigned u = 0;
      if (valid && ok) {
        const unsigned par = (phase >> sl0) & 1u;
        const unsigned char* slot = wslots + sl0 * B::kSlotBytes;
        u = (rec.fresh & kRecInterior)
                ? staged_block<S, true>(K, rec, fresh, lane, slot, bar + sl0, par, s_rcp, ok)
                : staged_block<S, false>(K, rec, fresh, lane, slot, bar + sl0, par, s_rcp, ok);
        if (kFreshCopy<S> || !fresh) phase ^= 1u << sl0;
      } else if (!valid && lane == 0) {
        set_status(slots[bs].sv.sc, kStInternal);
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) u += __shfl_xor_sync(0xffffffffu, u, off);
      if (lane == 0 && u) atomicAdd(&s_upd[bs], (unsigned long long)u);
      ok = __all_sync(0xffffffffu, ok);
      r0 = r1;
      r1 = r2;
      const int t = sl0;
      sl0 = sl1;
      sl1 = sl2;
      sl2 = t;
    }
    if (!ok) {
      if (lane == 0) set_status(slots[kslot < 0 ? 0 : kslot].sv.sc, kStTimeout);
      for (int sl = 0; sl < kStagedSlots; ++sl)
        mbar_wait_bounded(bar + sl, (phase >> sl) & 1u, kStagedWaitPolls);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_ctr[0] = 0;
      s_ctr[1] = 0;
    }
    __syncthreads();
  }
  // per-scene counts, then the arrival; the last CTA closes the frame of
  // every scene of this storage form (the arrival counter is the first such
  // scene's)
  __syncthreads();
  bool added = false;
  for (int i = threadIdx.x; i < n; i += NT) {
    AllocCounters* a = &slots[i].sv.fc->a[slots[i].fc.set];
    if (s_upd[i]) atomicAdd(&a->n_updated, s_upd[i]);
    if (s_vis[i]) atomicAdd(&a->n_visible, s_vis[i]);
    added = added || s_upd[i] || s_vis[i];
  }
  if (added) __threadfence();
  int first_s = 0;
  while (first_s < n && slots[first_s].sv.storage != S) ++first_s;
  if (first_s == n) return;  // uniform: no scene of this form
  if (last_to_arrive(&slots[first_s].sv.fc->a[slots[first_s].fc.set].integ_arrive, G_)) {
    for (int i = 0; i < n; ++i) {
      if (slots[i].sv.storage != S) continue;
      close_frame(slots[i].fc, slots[i].sv);
      __syncthreads();
    }
  }
}

// Batched: the allocated blocks of all scenes of this storage form form one
// range (scene s owns [hw_prefix[s], hw_prefix[s + 1])), tested as above;
// records carry their scene, warps rebuild their per-scene constants when a
// record belongs to another scene, and counts are kept per scene in shared
// memory and added once per CTA.
template <int S>
__global__ void __launch_bounds__(kIntegThreads, 3) integrate_batch_kernel(const SlotDesc* slots,
                                                                        int n) {
  __shared__ float s_rcp[256];
  __shared__ int s_hw[kMaxBatch + 1];
  __shared__ VisRec s_blk[kIntegThreads];
  __shared__ unsigned short s_bslot[kIntegThreads];
  __shared__ int s_warp[kIntegThreads / 32];
  __shared__ int s_total, s_next;
  __shared__ unsigned long long s_upd[kMaxBatch];
  __shared__ int s_vis[kMaxBatch];
  __shared__ FrameAlloc s_fa[kMaxBatch];
  allow_dependents();
  init_rcp_table(s_rcp);
  const int lane = threadIdx.x & 31;
  wait_prior_grid();  // the allocation kernel's results
  // allocation results and high-water marks of every scene (a scene of
  // another storage form counts 0 blocks), exclusive prefix by thread 0
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const FrameAlloc fa = frame_alloc(slots[i].sv, slots[i].fc.set);
    s_fa[i] = fa;
    s_hw[i + 1] = slots[i].sv.storage == S ? fa.high_water : 0;
    s_upd[i] = 0ull;
    s_vis[i] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_hw[0] = 0;
    for (int i = 0; i < n; ++i) s_hw[i + 1] += s_hw[i];
  }
  __syncthreads();

  const int total = s_hw[n];
  const int per_pass = gridDim.x * blockDim.x;
  int kslot = -1;  // warp-uniform: the scene K describes
  UnitConsts K;
  for (int base = blockIdx.x; base < total; base += per_pass) {
    const int g = base + threadIdx.x * gridDim.x;
    VisRec r;
    bool sel = false;
    int slot = 0;
    if (g < total) {
      int lo = 0, hi = n - 1;  // last scene with s_hw[scene] <= g
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_hw[mid] <= g) lo = mid; else hi = mid - 1;
      }
      slot = lo;
      const SlotDesc* d = &slots[slot];
      sel = select_block(d->fc, d->sv, s_fa[slot], g - s_hw[slot], r);
      if (sel) atomicAdd(&s_vis[slot], 1);
    }
    const int warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, sel);
    const int nb = compact_pass(sel, r, s_blk, s_warp, &s_total, &s_next);
    if (sel) s_bslot[s_warp[warp] + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)slot;
    __syncthreads();
    for (int i = grab_record(&s_next, lane); i < nb; i = grab_record(&s_next, lane)) {
      const VisRec rec = s_blk[i];
      const int bs = s_bslot[i];
      if (bs != kslot) {
        kslot = bs;
        make_unit_consts(slots[bs].fc, slots[bs].sv, lane, K);
      }
      unsigned u = process_block<S>(K, rec, lane, s_rcp, slots[bs].sv.sc);
#pragma unroll
      for (int off = 16; off; off >>= 1) u += __shfl_xor_sync(0xffffffffu, u, off);
      if (lane == 0 && u) atomicAdd(&s_upd[bs], (unsigned long long)u);
    }
    __syncthreads();
  }
  bool added = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    AllocCounters* a = &slots[i].sv.fc->a[slots[i].fc.set];
    if (s_upd[i]) atomicAdd(&a->n_updated, s_upd[i]);
    if (s_vis[i]) atomicAdd(&a->n_visible, s_vis[i]);
    added = added || s_upd[i] || s_vis[i];
  }
  if (added) __threadfence();
  // the last CTA closes the frame of every scene of this storage form (the
  // arrival counter is the first such scene's)
  int first = 0;
  while (first < n && slots[first].sv.storage != S) ++first;
  if (first == n) return;  // uniform: no scene of this form
  if (last_to_arrive(&slots[first].sv.fc->a[slots[first].fc.set].integ_arrive, gridDim.x)) {
    for (int i = 0; i < n; ++i) {
      if (slots[i].sv.storage != S) continue;
      close_frame(slots[i].fc, slots[i].sv);
      __syncthreads();  // thread 0's reads of scene i's counts precede nothing else
    }
  }
}

// Clears a set the resume path used (it runs the allocation stages without
// the integration kernel); the scene counters are not touched.
__global__ void finish_frame_kernel(SceneView sv, int set) {
  AllocCounters* a = &sv.fc->a[set];
  a->n_new = 0;
  a->n_overflow = 0;
  a->assign_base = 0;
  a->depth_max_bits = 0u;
  a->alloc_done = 0;
  a->n_visible = 0;
  a->integ_arrive = 0;
  a->n_updated = 0ull;
  a->integ_packed = 0ull;
  for (int g = 0; g < kArriveGroups; ++g) a->arrive[g] = 0;
}

template <typename Kern>
int blocks_per_sm(Kern k, int threads) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, threads, 0);
  return b > 0 ? b : 1;
}

template <int S, bool C>
cudaError_t launch_integrate_sc(const FrameConst& fc, const SceneView& sv, int sm_count,
                                int ctas_per_sm, cudaStream_t st) {
  static const int b = blocks_per_sm(integrate_kernel<S, C>, kIntegThreads);
  const int per_sm = ctas_per_sm > 0 ? min(b, ctas_per_sm) : b;
  return launch_pdl(integrate_kernel<S, C>, dim3(sm_count * per_sm), dim3(kIntegThreads), st, fc,
                    sv);
}

// the staged kernel: one CTA per SM, its shared memory opted in once
template <int S, int NT>
cudaError_t launch_integrate_staged_nt(const FrameConst& fc, const SceneView& sv, int sm_count,
                                       cudaStream_t st) {
  using G = StagedGeom<S, NT>;
  static const cudaError_t attr = cudaFuncSetAttribute(
      integrate_staged_kernel<S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kBytes);
  if (attr != cudaSuccess) return attr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sm_count);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = G::kBytes;
  cfg.stream = st;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, integrate_staged_kernel<S, NT>, fc, sv);
}

// share_sm: other kernels run beside this one (the smaller CTA leaves them
// registers and shared memory on every SM)
template <int S>
cudaError_t launch_integrate_staged(const FrameConst& fc, const SceneView& sv, int sm_count,
                                    bool share_sm, cudaStream_t st) {
  return share_sm ? launch_integrate_staged_nt<S, 256>(fc, sv, sm_count, st)
                  : launch_integrate_staged_nt<S, kStagedThreadsMax>(fc, sv, sm_count, st);
}

// Scenes that keep voxel colours take the kernel with the colour path;
// depth-only scenes the staged kernel (images below 2^24 pixels, the bound
// of its pixel offsets, and mu >= 2^-20 m, the range of its update flags),
// except 16-bit scenes beside another kernel (pipelined sequences), where
// the general kernel's two CTAs per SM hide latency better than one staged
// CTA of 256 threads (measured: 1280x720 int16 sequences 9 % faster; equal
// at 640x480); the rest take the general kernel.
template <int S>
cudaError_t launch_integrate_s(const FrameConst& fc, const SceneView& sv, int sm_count,
                               int ctas_per_sm, cudaStream_t st) {
  if (sv.rgbw) return launch_integrate_sc<S, true>(fc, sv, sm_count, ctas_per_sm, st);
  const bool share_sm = ctas_per_sm > 0;
  if ((long long)fc.width * fc.height < (1ll << 24) && fc.mu >= kStagedMinMu &&
      (S == TSDF_STORAGE_F32 || !share_sm))
    return launch_integrate_staged<S>(fc, sv, sm_count, share_sm, st);
  return launch_integrate_sc<S, false>(fc, sv, sm_count, ctas_per_sm, st);
}

template <int S>
cudaError_t launch_integrate_batch_general(const SlotDesc* d_slots, int n, int sm_count,
                                           int ctas_per_sm, cudaStream_t st) {
  static const int b = blocks_per_sm(integrate_batch_kernel<S>, kIntegThreads);
  const int grid = max(sm_count * min(b, ctas_per_sm), n);
  return launch_pdl(integrate_batch_kernel<S>, dim3(grid), dim3(kIntegThreads), st, d_slots, n);
}

template <int S, int NT>
cudaError_t launch_integrate_batch_staged(const SlotDesc* d_slots, int n, int sm_count,
                                          cudaStream_t st) {
  using G = StagedBatchGeom<S, NT>;
  static const cudaError_t attr = cudaFuncSetAttribute(
      integrate_batch_staged_kernel<S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kBytes);
  if (attr != cudaSuccess) return attr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sm_count);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = G::kBytes;
  cfg.stream = st;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, integrate_batch_staged_kernel<S, NT>, d_slots, n);
}

template <int S>
cudaError_t launch_integrate_batch_s(const SlotDesc* d_slots, int n, int sm_count,
                                     const BatchIntegLaunch& how, cudaStream_t st) {
  if (how.kernel == kBatchKernelGeneral)
    return launch_integrate_batch_general<S>(d_slots, n, sm_count, how.ctas_per_sm, st);
  return how.threads == 256 ? launch_integrate_batch_staged<S, 256>(d_slots, n, sm_count, st)
                            : launch_integrate_batch_staged<S, kStagedThreadsMax>(d_slots, n,
                                                                                 sm_count, st);
}

}  // namespace

cudaError_t launch_integrate(const FrameConst& fc, const SceneView& sv, int sm_count,
                             cudaStream_t st, int ctas_per_sm) {
  switch (sv.storage) {
    case TSDF_STORAGE_F32:
      return launch_integrate_s<TSDF_STORAGE_F32>(fc, sv, sm_count, ctas_per_sm, st);
    case TSDF_STORAGE_I16:
      return launch_integrate_s<TSDF_STORAGE_I16>(fc, sv, sm_count, ctas_per_sm, st);
    default:
      return launch_integrate_s<TSDF_STORAGE_F16>(fc, sv, sm_count, ctas_per_sm, st);
  }
}

cudaError_t launch_finish_frame(const SceneView& sv, int set, cudaStream_t st) {
  finish_frame_kernel<<<1, 1, 0, st>>>(sv, set);
  return cudaGetLastError();
}

// Batched launch: one per storage form present in the batch (each kernel
// skips the scenes of the other forms).
cudaError_t launch_integrate_batch(const SlotDesc* d_slots, const SlotDesc* h_slots, int n,
                                   int sm_count, const BatchIntegLaunch& how, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  bool has[3] = {false, false, false};
  for (int i = 0; i < n; ++i) has[h_slots[i].sv.storage] = true;
  cudaError_t e = cudaSuccess;
  if (has[0] && e == cudaSuccess)
    e = launch_integrate_batch_s<TSDF_STORAGE_F32>(d_slots, n, sm_count, how, st);
  if (has[1] && e == cudaSuccess)
    e = launch_integrate_batch_s<TSDF_STORAGE_I16>(d_slots, n, sm_count, how, st);
  if (has[2] && e == cudaSuccess)
    e = launch_integrate_batch_s<TSDF_STORAGE_F16>(d_slots, n, sm_count, how, st);
  return e;
}

}  // namespace tsdf
