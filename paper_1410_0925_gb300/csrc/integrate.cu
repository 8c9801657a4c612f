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
// block selection

// Can rule U write any voxel l in [0,7]^3 of the block whose origin voxel has
// the (float) camera point c0? Conservative: the voxels lie in the box spanned
// by the lattice offsets 0..7; its 8 corners bound every voxel's camera z and,
// when all are in front of the camera, the voxels' image points (perspective
// maps the box onto the hull of the corners' images).
__device__ __forceinline__ bool block_visible(const FrameConst& fc, const unsigned* tile_max,
                                              const float c0[3], float zfar) {
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

// ----------------------------------------------------------------------------
// integration

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Per-lane constants of one scene's frame for the integration of its blocks.
struct UnitConsts {
  const float* depth;  // sanitised depth, pitch = width, -inf = no measurement
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
        d[4 * i + j] = fminf(1.0f, eta * K.inv_mu);  // -inf where no measurement
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
};

// (The high-water mark comes from the frame's own commit, not from free_top,
// which the next frame's allocation may already be moving.)
__device__ __forceinline__ FrameAlloc frame_alloc(const SceneView& sv, int set) {
  FrameAlloc f;
  f.par = set;
  const AllocCounters* a = &sv.fc->a[set];
  f.fresh_from = sv.pool - __ldcg(&a->assign_base);
  f.high_water = f.fresh_from + __ldcg(&a->n_new);
  f.dmax_bits = __ldcg(&a->depth_max_bits);
  return f;
}

// Fold a frame's counts into its scene's counters and clear the frame's set
// (counters, and the pyramid levels built by atomics: levels 0 is rewritten
// by every allocation tile). Run by one CTA after every CTA that integrated
// the frame has added its counts.
__device__ void close_frame(const FrameConst& fc, const SceneView& sv) {
  AllocCounters* a = &sv.fc->a[fc.set];
  if (threadIdx.x == 0) {
    const int vis = __ldcg(&a->n_visible);
    const unsigned long long upd = __ldcg(&a->n_updated);
    SceneCounters* sc = sv.sc;
    sc->frames += 1;
    sc->last_new = (unsigned long long)__ldcg(&a->n_new);
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
  }
  for (int i = threadIdx.x; i < kArriveGroups; i += blockDim.x) a->arrive[i] = 0;
  if (fc.use_tiles) {
    unsigned* pyr = pyramid_set(sv, fc.set);
    int wl, hl;
    const int lo = fc.tiles_x * fc.tiles_y;
    const int hi = pyramid_level(fc.tiles_x, fc.tiles_y, kPyramidLevels, wl, hl);
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) pyr[i] = 0u;
  }
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

// Step 1 for allocated block `ptr`: does it need integrating, and its record.
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
    vis = block_visible(fc, pyramid_set(sv, fa.par), c0, __uint_as_float(fa.dmax_bits) + fc.mu);
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

// scenes that keep voxel colours take the kernel with the colour path
template <int S>
cudaError_t launch_integrate_s(const FrameConst& fc, const SceneView& sv, int sm_count,
                               int ctas_per_sm, cudaStream_t st) {
  return sv.rgbw ? launch_integrate_sc<S, true>(fc, sv, sm_count, ctas_per_sm, st)
                 : launch_integrate_sc<S, false>(fc, sv, sm_count, ctas_per_sm, st);
}

template <int S>
cudaError_t launch_integrate_batch_s(const SlotDesc* d_slots, int n, int sm_count,
                                     int ctas_per_sm, cudaStream_t st) {
  static const int b = blocks_per_sm(integrate_batch_kernel<S>, kIntegThreads);
  const int grid = max(sm_count * min(b, ctas_per_sm), n);
  return launch_pdl(integrate_batch_kernel<S>, dim3(grid), dim3(kIntegThreads), st, d_slots, n);
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
                                   int sm_count, int ctas_per_sm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  bool has[3] = {false, false, false};
  for (int i = 0; i < n; ++i) has[h_slots[i].sv.storage] = true;
  cudaError_t e = cudaSuccess;
  if (has[0] && e == cudaSuccess)
    e = launch_integrate_batch_s<TSDF_STORAGE_F32>(d_slots, n, sm_count, ctas_per_sm, st);
  if (has[1] && e == cudaSuccess)
    e = launch_integrate_batch_s<TSDF_STORAGE_I16>(d_slots, n, sm_count, ctas_per_sm, st);
  if (has[2] && e == cudaSuccess)
    e = launch_integrate_batch_s<TSDF_STORAGE_F16>(d_slots, n, sm_count, ctas_per_sm, st);
  return e;
}

}  // namespace tsdf
