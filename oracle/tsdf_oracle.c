/*
 * tsdf_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see
 * tsdf_oracle.h). Everything here follows the InfiniTAM report:
 *   - voxel type and fixed-point conversion: Section 3.1 (ITMVoxel listing);
 *   - dense volume: Section 3.2;
 *   - block grouping (8x8x8 voxels): Section 3.3;
 *   - allocation band [d - mu, d + mu] along each pixel ray: Section 4.2;
 *   - per-voxel update rule (projective truncated SDF, running average with
 *     a capped weight): Section 4.3;
 *   - swapping between device and host copies: Section 5.
 * Readings where the report is silent are marked "reading:".
 */
#include "tsdf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define BLOCK 8
#define BLOCK_VOXELS 512

/* ------------------------------------------------------------------ */
/* small linear algebra                                                */
/* ------------------------------------------------------------------ */

/* Rigid or affine 4x4 (row-major) applied to a point. Last row must be
 * (0, 0, 0, 1); checked by the callers. */
static void apply_affine(const double M[16], const double p[3], double out[3])
{
    for (int r = 0; r < 3; ++r)
        out[r] = M[4 * r + 0] * p[0] + M[4 * r + 1] * p[1] +
                 M[4 * r + 2] * p[2] + M[4 * r + 3];
}

static int is_affine(const double M[16])
{
    return M[12] == 0.0 && M[13] == 0.0 && M[14] == 0.0 && M[15] == 1.0;
}

/* General 4x4 inverse by Gauss-Jordan elimination with partial pivoting.
 * reading: the pose is given world->camera (the listing multiplies model
 * points by M_d); the band segment needs camera->world, so it is inverted
 * here in FP64. Returns 0 if singular. */
static int invert4(const double M[16], double out[16])
{
    double a[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c)
            a[r][c] = c < 4 ? M[4 * r + c] : (c - 4 == r ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (a[piv][c] == 0.0) return 0;
        if (piv != c)
            for (int k = 0; k < 8; ++k) {
                double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t;
            }
        double inv = 1.0 / a[c][c];
        for (int k = 0; k < 8; ++k) a[c][k] *= inv;
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            double f = a[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 8; ++k) a[r][k] -= f * a[c][k];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) out[4 * r + c] = a[r][c + 4];
    return 1;
}

static int key_cmp3(const int32_t *a, const int32_t *b)
{
    for (int i = 0; i < 3; ++i) {
        if (a[i] < b[i]) return -1;
        if (a[i] > b[i]) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* storage forms (Section 3.1)                                         */
/* ------------------------------------------------------------------ */

int16_t or_float_to_i16(double x)
{
    /* SDF_floatToValue: (short)(x * 32767), i.e. truncation toward zero */
    return (int16_t)(x * 32767.0);
}

double or_i16_to_float(int16_t q)
{
    /* SDF_valueToFloat: x / 32767 */
    return (double)q / 32767.0;
}

double or_round_f16(double x)
{
    /* reading: the report has no half-precision voxel; FP16 storage rounds
     * to the nearest binary16 value, ties to even (IEEE 754 default). */
    if (x == 0.0 || !isfinite(x)) return x;
    double ax = fabs(x);
    int e;
    frexp(ax, &e);              /* ax = m * 2^e, m in [0.5, 1) */
    int q_exp = e - 11;         /* 11 significant bits */
    if (q_exp < -24) q_exp = -24; /* binary16 subnormal quantum 2^-24 */
    double q = ldexp(1.0, q_exp);
    double r = nearbyint(ax / q) * q; /* default rounding: ties to even */
    if (r > 65504.0) r = INFINITY;
    return x < 0 ? -r : r;
}

static double store_value(int storage, double F)
{
    switch (storage) {
    case OR_STORAGE_I16: return or_i16_to_float(or_float_to_i16(F));
    case OR_STORAGE_F16: return or_round_f16(F);
    default: return F;
    }
}

/* reading: the initial sdf is the short type's 32767 (= 1.0 as a value) and
 * 1.0 for the float and half forms; the weight starts at 0. */
static const double SDF_INITIAL = 1.0;

/* ------------------------------------------------------------------ */
/* per-frame context                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    const float *depth;
    const uint8_t *rgb;  /* RGBX colour registered to depth, or NULL */
    int width, height;
    double fx, fy, cx, cy;
    double M[16];     /* world -> camera */
    double Minv[16];  /* camera -> world */
} frame_ctx;

static int make_frame(frame_ctx *fc, const float *depth, int width,
                      int height, const double intr[4], const double M[16])
{
    if (!depth || width < 3 || height < 3 || !intr || !M) return -1;
    if (!is_affine(M)) return -1;
    fc->depth = depth;
    fc->rgb = NULL;
    fc->width = width;
    fc->height = height;
    fc->fx = intr[0]; fc->fy = intr[1]; fc->cx = intr[2]; fc->cy = intr[3];
    if (!(fc->fx != 0.0) || !(fc->fy != 0.0)) return -1;
    memcpy(fc->M, M, sizeof(fc->M));
    if (!invert4(M, fc->Minv)) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* allocation band (Section 4.2, first stage)                          */
/* ------------------------------------------------------------------ */

/* Does the closed segment P0-P1 meet the closed box [lo, hi]? Slab test
 * (Kay & Kajiya): intersect the parameter intervals of the three slabs. */
static int segment_meets_box(const double P0[3], const double P1[3],
                             const double lo[3], const double hi[3])
{
    double t0 = 0.0, t1 = 1.0;
    for (int a = 0; a < 3; ++a) {
        double d = P1[a] - P0[a];
        if (d == 0.0) {
            if (P0[a] < lo[a] || P0[a] > hi[a]) return 0;
            continue;
        }
        double ta = (lo[a] - P0[a]) / d;
        double tb = (hi[a] - P0[a]) / d;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* World-space end points of pixel (u, v)'s band segment: camera points
 * sigma * ((u - cx)/fx, (v - cy)/fy, 1) for sigma = d - mu and d + mu.
 * reading: sigma is camera z (the same quantity eta = d - z compares), and
 * the segment is not clipped to positive depth. */
static void band_segment(const frame_ctx *fc, int u, int v, double d,
                         double mu, double P0[3], double P1[3])
{
    double r[3] = { ((double)u - fc->cx) / fc->fx,
                    ((double)v - fc->cy) / fc->fy, 1.0 };
    double qa[3], qb[3];
    for (int i = 0; i < 3; ++i) {
        qa[i] = (d - mu) * r[i];
        qb[i] = (d + mu) * r[i];
    }
    apply_affine(fc->Minv, qa, P0);
    apply_affine(fc->Minv, qb, P1);
}

static void block_box(const int32_t key[3], double s, double grow,
                      double lo[3], double hi[3])
{
    for (int i = 0; i < 3; ++i) {
        lo[i] = (double)BLOCK * key[i] * s - grow;
        hi[i] = (double)BLOCK * (key[i] + 1) * s + grow;
    }
}

/* hit bits of one block against one segment */
static int hit_bits(const double P0[3], const double P1[3],
                    const int32_t key[3], double s, double db)
{
    double lo[3], hi[3];
    int bits = 0;
    block_box(key, s, db, lo, hi);
    if (!segment_meets_box(P0, P1, lo, hi)) return 0;
    bits |= OR_HIT_GROWN;
    block_box(key, s, 0.0, lo, hi);
    if (segment_meets_box(P0, P1, lo, hi)) bits |= OR_HIT_EXACT;
    block_box(key, s, -db, lo, hi);
    if (segment_meets_box(P0, P1, lo, hi)) bits |= OR_HIT_SHRUNK;
    return bits;
}

static int valid_depth(float d)
{
    /* reading: a pixel carries a measurement iff its depth is finite and
     * > 0 (the listing rejects depth <= 0; NaN / inf are treated as
     * missing too) */
    return isfinite(d) && d > 0.0f;
}

typedef struct { int32_t key[3]; int bits; } hit_rec;

typedef struct { hit_rec *v; size_t n, cap; } hit_vec;

static int hit_push(hit_vec *h, const int32_t key[3], int bits)
{
    if (h->n == h->cap) {
        size_t nc = h->cap ? 2 * h->cap : 4096;
        hit_rec *nv = (hit_rec *)realloc(h->v, nc * sizeof(hit_rec));
        if (!nv) return -1;
        h->v = nv;
        h->cap = nc;
    }
    memcpy(h->v[h->n].key, key, sizeof(int32_t) * 3);
    h->v[h->n].bits = bits;
    h->n++;
    return 0;
}

static int hit_cmp(const void *a, const void *b)
{
    return key_cmp3(((const hit_rec *)a)->key, ((const hit_rec *)b)->key);
}

/* All blocks met (grown box) by some pixel's band segment in this frame,
 * one record per block with the OR of its hit bits, sorted by key. */
static int frame_hits(const frame_ctx *fc, double s, double mu, double db,
                      hit_vec *out)
{
    out->n = 0;
    const double inv_block = 1.0 / ((double)BLOCK * s);
    for (int v = 0; v < fc->height; ++v) {
        for (int u = 0; u < fc->width; ++u) {
            float dd = fc->depth[(size_t)v * fc->width + u];
            if (!valid_depth(dd)) continue;
            double P0[3], P1[3];
            band_segment(fc, u, v, (double)dd, mu, P0, P1);
            long long bl[3], bh[3];
            for (int a = 0; a < 3; ++a) {
                double mn = P0[a] < P1[a] ? P0[a] : P1[a];
                double mx = P0[a] < P1[a] ? P1[a] : P0[a];
                bl[a] = (long long)floor((mn - db) * inv_block);
                bh[a] = (long long)floor((mx + db) * inv_block);
            }
            int32_t key[3];
            for (long long bz = bl[2]; bz <= bh[2]; ++bz)
                for (long long by = bl[1]; by <= bh[1]; ++by)
                    for (long long bx = bl[0]; bx <= bh[0]; ++bx) {
                        key[0] = (int32_t)bx;
                        key[1] = (int32_t)by;
                        key[2] = (int32_t)bz;
                        int bits = hit_bits(P0, P1, key, s, db);
                        if (bits && hit_push(out, key, bits)) return -1;
                    }
        }
    }
    qsort(out->v, out->n, sizeof(hit_rec), hit_cmp);
    size_t w = 0;
    for (size_t i = 0; i < out->n; ++i) {
        if (w > 0 && key_cmp3(out->v[w - 1].key, out->v[i].key) == 0)
            out->v[w - 1].bits |= out->v[i].bits;
        else
            out->v[w++] = out->v[i];
    }
    out->n = w;
    return 0;
}

/* ------------------------------------------------------------------ */
/* per-voxel update (Section 4.3)                                      */
/* ------------------------------------------------------------------ */

static int near_value(double x, double b, double delta)
{
    return fabs(x - b) < delta;
}

static int near_half_integer_rounding(double x, double delta)
{
    /* (int)(x + 0.5) changes where x + 0.5 crosses an integer */
    double t = x + 0.5;
    double f = t - floor(t);
    return f < delta || f > 1.0 - delta;
}

/* Colour of a voxel (the voxel type's clr and w_color, Section 3.1), updated
 * like the depth: the report lists only the depth function and says a
 * similar one also updates the colour. reading: the colour is updated for
 * exactly the voxels rule U updates, from the same (nearest) pixel of a
 * colour image registered to the depth image; per channel the listing's
 * average new = (w old + obs) / (w + 1) with the uncapped count, evaluated in
 * float as the listing does (w old + obs is an exact integer, so one IEEE
 * division decides the value), stored rounded to the nearest integer
 * (floor(x + 1/2); truncation as for the sdf would drag every colour down and
 * freeze it once the weight is capped); then w <- min(w + 1, maxW). */
static void update_colour(const or_params *p, const uint8_t *obs, uint8_t *rgbw)
{
    const int wc = rgbw[3];
    const float den = (float)(wc + 1);
    for (int c = 0; c < 3; ++c) {
        const float num = (float)wc * (float)rgbw[c] + (float)obs[c];
        const float x = num / den;
        rgbw[c] = (uint8_t)floorf(x + 0.5f);
    }
    rgbw[3] = (uint8_t)(wc + 1 > p->max_weight ? p->max_weight : wc + 1);
}

/* Section 4.3 fuses one frame into a voxel v in three parts, each written
 * out below as its own function:
 *
 *   1. the measurement that the frame holds for v: the depth D(u) at the
 *      pixel u nearest to the projection of v's camera point x_c = M v
 *      (A1, A12, A17), defined when x_c lies in front of the camera, u lies
 *      inside the image window [1, W-2] x [1, H-2] and D(u) is a valid depth
 *      (A15);
 *   2. the projective signed distance eta = D(u) - z(x_c) along the viewing
 *      axis, truncated: f = min(1, eta / mu) when eta >= -mu; a voxel more
 *      than mu behind the measured surface is occluded and receives nothing;
 *   3. the weighted running average of the observations, with the count of
 *      observations capped at maxW (A9, A16) and the stored form's rounding
 *      (A8, A10, A14).
 *
 * Every threshold decision on the way (z = 0, the window's edges, the
 * rounding to the nearest pixel, eta = -mu) sets *flag when the exact value
 * lies within its margin, so that the FP32 device path may take the other
 * side. */

/* Part 1: the pixel of frame fc that observes camera point pc, or 0 when
 * there is none. */
static int observing_pixel(const or_params *p, const frame_ctx *fc,
                           const double pc[3], int *ix, int *iy, int *flag)
{
    const double z = pc[2];
    if (fabs(z) < p->delta_z) *flag = 1;
    if (!(z > 0.0)) return 0;                       /* behind the camera */

    const double u[2] = { fc->fx * pc[0] / z + fc->cx, fc->fy * pc[1] / z + fc->cy };
    const double hi[2] = { fc->width - 2, fc->height - 2 };
    int inside = 1;
    for (int a = 0; a < 2; ++a) {
        if (near_value(u[a], 1.0, p->delta_px) || near_value(u[a], hi[a], p->delta_px))
            *flag = 1;
        inside = inside && u[a] >= 1.0 && u[a] <= hi[a];
    }
    if (!inside) return 0;
    for (int a = 0; a < 2; ++a)
        if (near_half_integer_rounding(u[a], p->delta_px)) *flag = 1;
    *ix = (int)floor(u[0] + 0.5);                   /* nearest pixel */
    *iy = (int)floor(u[1] + 0.5);
    return 1;
}

/* Part 2: the truncated projective signed distance, or 0 when the voxel is
 * occluded (eta < -mu). */
static int truncated_sdf(const or_params *p, double eta, double *f, int *flag)
{
    if (near_value(eta, -p->mu, p->delta_eta)) *flag = 1;
    if (eta < -p->mu) return 0;
    *f = fmin(eta / p->mu, 1.0);
    return 1;
}

/* Part 3: fold observation f into the stored (F, W). The average counts the
 * new observation among W + 1 (uncapped); the stored count saturates at
 * maxW, so later observations keep a weight of 1 / (maxW + 1). */
static void fold_observation(const or_params *p, double f, double *F, int *W)
{
    const int w = *W;
    *F = store_value(p->storage, ((double)w * (*F) + f) / (double)(w + 1));
    *W = w + 1 < p->max_weight ? w + 1 : p->max_weight;
}

/* One voxel (integer coordinate v) in one frame: parts 1-3 above. F/W hold
 * the stored value (as a real) and weight; rgbw (may be NULL) the voxel's
 * colour and colour weight, updated when the frame has colour. Returns 1 if
 * the voxel was written. */
static int update_voxel(const or_params *p, const frame_ctx *fc,
                        const long long v[3], double *F, int *W, int *flag,
                        uint8_t *rgbw)
{
    const double s = p->voxel_size;
    const double pm[3] = { (double)v[0] * s, (double)v[1] * s, (double)v[2] * s };
    double pc[3];
    apply_affine(fc->M, pm, pc);
    int ix, iy;
    if (!observing_pixel(p, fc, pc, &ix, &iy, flag)) return 0;
    const size_t pix = (size_t)iy * fc->width + ix;
    if (!valid_depth(fc->depth[pix])) return 0;
    double f;
    if (!truncated_sdf(p, (double)fc->depth[pix] - pc[2], &f, flag)) return 0;
    fold_observation(p, f, F, W);
    if (fc->rgb && rgbw) update_colour(p, fc->rgb + 4 * pix, rgbw);
    return 1;
}

/* ------------------------------------------------------------------ */
/* block-form scene                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t key[3];
    int allocated;
    int t_alloc, t_poss, t_rob;   /* -1 = never */
    double *sdf;
    uint8_t *w;
    uint8_t *vflag;
    uint8_t *rgbw;   /* [512][4]: r, g, b, colour weight */
    /* swapping (Section 5): the host copy of a swapped-out block */
    int on_host;     /* a host copy exists                              */
    int swapped;     /* was swapped out at least once                   */
    int swap_amb;    /* some swap decision about it lay within a margin */
    double *h_sdf;
    uint8_t *h_w, *h_vflag, *h_rgbw;
} or_block;

struct or_scene {
    or_params p;
    or_block **blocks;   /* every block ever met by a grown box, sorted */
    size_t n, cap;
    long long n_alloc;
    long long n_updates;
    int frame;
    hit_vec hits;
};

or_scene *or_create(const or_params *p)
{
    if (!p || !(p->voxel_size > 0) || !(p->mu > 0) || p->max_weight < 1 ||
        p->max_weight > 255 || p->storage < 0 || p->storage > 2)
        return NULL;
    or_scene *s = (or_scene *)calloc(1, sizeof(or_scene));
    if (!s) return NULL;
    s->p = *p;
    return s;
}

void or_destroy(or_scene *s)
{
    if (!s) return;
    for (size_t i = 0; i < s->n; ++i) {
        free(s->blocks[i]->sdf);
        free(s->blocks[i]->w);
        free(s->blocks[i]->vflag);
        free(s->blocks[i]->rgbw);
        free(s->blocks[i]->h_sdf);
        free(s->blocks[i]->h_w);
        free(s->blocks[i]->h_vflag);
        free(s->blocks[i]->h_rgbw);
        free(s->blocks[i]);
    }
    free(s->blocks);
    free(s->hits.v);
    free(s);
}

/* binary search: index of key, or -(insertion point) - 1 */
static long long find_block(const or_scene *s, const int32_t key[3])
{
    size_t lo = 0, hi = s->n;
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        int c = key_cmp3(s->blocks[mid]->key, key);
        if (c == 0) return (long long)mid;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return -(long long)lo - 1;
}

/* merge the sorted new records (keys not yet present) into the block list */
static int insert_blocks(or_scene *s, or_block **nb, size_t m)
{
    if (m == 0) return 0;
    or_block **merged = (or_block **)malloc((s->n + m) * sizeof(or_block *));
    if (!merged) return -1;
    size_t i = 0, j = 0, k = 0;
    while (i < s->n || j < m) {
        if (j == m || (i < s->n && key_cmp3(s->blocks[i]->key, nb[j]->key) < 0))
            merged[k++] = s->blocks[i++];
        else
            merged[k++] = nb[j++];
    }
    free(s->blocks);
    s->blocks = merged;
    s->n += m;
    s->cap = s->n;
    return 0;
}

static int allocate_block_data(or_block *b)
{
    b->sdf = (double *)malloc(BLOCK_VOXELS * sizeof(double));
    b->w = (uint8_t *)calloc(BLOCK_VOXELS, 1);
    b->vflag = (uint8_t *)calloc(BLOCK_VOXELS, 1);
    b->rgbw = (uint8_t *)calloc(4 * BLOCK_VOXELS, 1);  /* colour 0, weight 0 */
    if (!b->sdf || !b->w || !b->vflag || !b->rgbw) return -1;
    for (int i = 0; i < BLOCK_VOXELS; ++i) b->sdf[i] = SDF_INITIAL;
    return 0;
}

static int integrate_frame(or_scene *s, const float *depth, const uint8_t *rgb, int width,
                           int height, const double intr[4], const double world_to_cam[16])
{
    if (!s) return -1;
    frame_ctx fc;
    if (make_frame(&fc, depth, width, height, intr, world_to_cam)) return -1;
    fc.rgb = rgb;
    const int t = s->frame;
    int status = 0;

    /* 1. allocation set of this frame (before integration, Section 2.1) */
    if (frame_hits(&fc, s->p.voxel_size, s->p.mu, s->p.delta_b, &s->hits))
        return -3;
    size_t nh = s->hits.n;
    or_block **fresh = (or_block **)malloc((nh ? nh : 1) * sizeof(or_block *));
    if (!fresh) return -3;
    size_t nfresh = 0;
    for (size_t i = 0; i < nh; ++i) {
        const hit_rec *h = &s->hits.v[i];
        long long at = find_block(s, h->key);
        or_block *b;
        if (at >= 0) {
            b = s->blocks[at];
        } else {
            b = (or_block *)calloc(1, sizeof(or_block));
            if (!b) { free(fresh); return -3; }
            memcpy(b->key, h->key, sizeof(b->key));
            b->t_alloc = b->t_poss = b->t_rob = -1;
            fresh[nfresh++] = b;
        }
        if ((h->bits & OR_HIT_GROWN) && b->t_poss < 0) b->t_poss = t;
        if ((h->bits & OR_HIT_SHRUNK) && b->t_rob < 0) b->t_rob = t;
        /* a swapped-out block that a segment only grazes: the GPU may give
         * it a fresh device block in this frame or not */
        if (b->on_host && !b->allocated && !(h->bits & OR_HIT_SHRUNK)) b->swap_amb = 1;
    }
    if (insert_blocks(s, fresh, nfresh)) { free(fresh); return -3; }
    free(fresh);

    /* new exact hits, already in key order; reading: if the pool cannot hold
     * them all, the smallest keys are allocated and the rest wait */
    for (size_t i = 0; i < nh; ++i) {
        const hit_rec *h = &s->hits.v[i];
        if (!(h->bits & OR_HIT_EXACT)) continue;
        or_block *b = s->blocks[find_block(s, h->key)];
        if (b->allocated) continue;
        if (s->p.pool_blocks > 0 && s->n_alloc >= s->p.pool_blocks) {
            status = 1;
            continue;
        }
        if (allocate_block_data(b)) return -3;
        b->allocated = 1;
        if (b->t_alloc < 0) b->t_alloc = t;  /* first allocation (not a swap-in) */
        s->n_alloc++;
    }

    /* 2. integration: every voxel of every allocated block */
    for (size_t i = 0; i < s->n; ++i) {
        or_block *b = s->blocks[i];
        if (!b->allocated) continue;
        for (int lz = 0; lz < BLOCK; ++lz)
            for (int ly = 0; ly < BLOCK; ++ly)
                for (int lx = 0; lx < BLOCK; ++lx) {
                    int li = lx + BLOCK * ly + BLOCK * BLOCK * lz;
                    long long v[3] = { (long long)BLOCK * b->key[0] + lx,
                                       (long long)BLOCK * b->key[1] + ly,
                                       (long long)BLOCK * b->key[2] + lz };
                    int W = b->w[li], flag = 0;
                    s->n_updates += update_voxel(&s->p, &fc, v, &b->sdf[li], &W, &flag,
                                                 b->rgbw + 4 * li);
                    b->w[li] = (uint8_t)W;
                    if (flag) b->vflag[li] = 1;
                }
    }
    s->frame++;
    return status;
}

int or_integrate(or_scene *s, const float *depth, int width, int height,
                 const double intr[4], const double world_to_cam[16])
{
    return integrate_frame(s, depth, NULL, width, height, intr, world_to_cam);
}

int or_integrate_rgb(or_scene *s, const float *depth, const uint8_t *rgb, int width,
                     int height, const double intr[4], const double world_to_cam[16])
{
    if (!rgb) return -1;
    return integrate_frame(s, depth, rgb, width, height, intr, world_to_cam);
}

int or_read_colour(const or_scene *s, uint8_t *rgbw)
{
    if (!s || !rgbw) return -1;
    size_t k = 0;
    for (size_t i = 0; i < s->n; ++i) {
        const or_block *b = s->blocks[i];
        if (!b->allocated) continue;
        memcpy(rgbw + 4 * BLOCK_VOXELS * k, b->rgbw, 4 * BLOCK_VOXELS);
        ++k;
    }
    return 0;
}

long long or_num_blocks(const or_scene *s) { return s ? s->n_alloc : -1; }

long long or_total_updates(const or_scene *s) { return s ? s->n_updates : -1; }

long long or_num_ghosts(const or_scene *s)
{
    if (!s) return -1;
    long long g = 0;
    for (size_t i = 0; i < s->n; ++i)
        if (s->blocks[i]->t_alloc < 0 && s->blocks[i]->t_poss >= 0) ++g;
    return g;
}

int or_read(const or_scene *s, int32_t *keys, double *sdf, uint8_t *w,
            uint8_t *vflag, uint8_t *bflag, int32_t *t_alloc)
{
    if (!s) return -1;
    size_t k = 0;
    for (size_t i = 0; i < s->n; ++i) {
        const or_block *b = s->blocks[i];
        if (!b->allocated) continue;
        if (keys) memcpy(keys + 3 * k, b->key, 3 * sizeof(int32_t));
        if (sdf) memcpy(sdf + BLOCK_VOXELS * k, b->sdf, BLOCK_VOXELS * sizeof(double));
        if (w) memcpy(w + BLOCK_VOXELS * k, b->w, BLOCK_VOXELS);
        if (vflag) memcpy(vflag + BLOCK_VOXELS * k, b->vflag, BLOCK_VOXELS);
        if (bflag) {
            uint8_t f = 0;
            if (b->t_rob < 0) f |= OR_BLOCK_MEMBERSHIP_AMBIGUOUS;
            if (b->t_poss != b->t_rob) f |= OR_BLOCK_HISTORY_AMBIGUOUS;
            if (b->swap_amb) f |= OR_BLOCK_SWAP_AMBIGUOUS;
            if (b->swapped) f |= OR_BLOCK_SWAPPED;
            bflag[k] = f;
        }
        if (t_alloc) t_alloc[k] = b->t_alloc;
        ++k;
    }
    return 0;
}

int or_read_ghosts(const or_scene *s, int32_t *keys)
{
    if (!s || !keys) return -1;
    size_t k = 0;
    for (size_t i = 0; i < s->n; ++i) {
        const or_block *b = s->blocks[i];
        if (b->t_alloc >= 0 || b->t_poss < 0) continue;
        memcpy(keys + 3 * k, b->key, 3 * sizeof(int32_t));
        ++k;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* swapping (Section 5)                                                */
/* ------------------------------------------------------------------ */

/* Is a block inside or near the view? reading: the active part of the map is
 * what lies in or close to the view frustum; a block counts as visible when
 *   - some corner of its box [8bs, 8(b+1)s]^3 is in front of the camera
 *     (camera z > 0), and
 *   - either some corner is not (the block straddles the camera plane), or
 *     the bounding box of the eight projected corners meets the image
 *     rectangle of pixel centres grown by `margin` pixels on every side,
 *     [-1/2 - margin, W - 1/2 + margin] x [-1/2 - margin, H - 1/2 + margin],
 *     and (if max_depth > 0) the nearest corner is no farther than max_depth.
 * *amb is set when a corner's camera z lies within delta_z of 0 or of
 * max_depth, or a bounding-box edge within delta_px of its bound. */
static int block_visible(const or_params *p, const frame_ctx *fc, double margin,
                         double max_depth, const int32_t key[3], int *amb)
{
    const double s = p->voxel_size;
    double qz[8], u[8], v[8];
    int n_front = 0;
    for (int c = 0; c < 8; ++c) {
        double P[3], q[3];
        for (int a = 0; a < 3; ++a)
            P[a] = (double)BLOCK * (key[a] + ((c >> a) & 1)) * s;
        apply_affine(fc->M, P, q);
        qz[c] = q[2];
        if (fabs(q[2]) < p->delta_z) *amb = 1;
        if (q[2] > 0.0) {
            ++n_front;
            u[c] = fc->fx * q[0] / q[2] + fc->cx;
            v[c] = fc->fy * q[1] / q[2] + fc->cy;
        }
    }
    if (n_front == 0) return 0;
    if (n_front < 8) return 1;
    double umin = u[0], umax = u[0], vmin = v[0], vmax = v[0], zmin = qz[0];
    for (int c = 1; c < 8; ++c) {
        if (u[c] < umin) umin = u[c];
        if (u[c] > umax) umax = u[c];
        if (v[c] < vmin) vmin = v[c];
        if (v[c] > vmax) vmax = v[c];
        if (qz[c] < zmin) zmin = qz[c];
    }
    const double lo_u = -0.5 - margin, hi_u = fc->width - 0.5 + margin;
    const double lo_v = -0.5 - margin, hi_v = fc->height - 0.5 + margin;
    if (near_value(umax, lo_u, p->delta_px) || near_value(umin, hi_u, p->delta_px) ||
        near_value(vmax, lo_v, p->delta_px) || near_value(vmin, hi_v, p->delta_px))
        *amb = 1;
    if (max_depth > 0.0 && near_value(zmin, max_depth, p->delta_z)) *amb = 1;
    return umax >= lo_u && umin <= hi_u && vmax >= lo_v && vmin <= hi_v &&
           (max_depth <= 0.0 || zmin <= max_depth);
}

int or_block_visible(const or_params *p, int width, int height, const double intr[4],
                     const double world_to_cam[16], double margin_px, double max_depth,
                     const int32_t key[3], int *ambiguous)
{
    frame_ctx fc;
    static const float dummy = 0.0f;
    if (!p || !key || make_frame(&fc, &dummy, width, height, intr, world_to_cam)) return -1;
    int amb = 0;
    const int vis = block_visible(p, &fc, margin_px, max_depth, key, &amb);
    if (ambiguous) *ambiguous = amb;
    return vis;
}

/* One swap candidate as the oracle sees it: `own` = a candidate in the
 * oracle's own (exact FP64) evaluation; `sure` = a candidate whatever the GPU
 * decides within the margins and whatever ghosts it holds. */
typedef struct { or_block *b; int own, sure, maybe; } swap_cand;

/* reading: a call moves at most `capacity` blocks, the candidates with the
 * smallest (x, y, z) keys first (as the pool-exhaustion rule of the
 * allocation). Candidates come in key order. Marks swap_amb on every oracle
 * block whose selection the GPU could decide otherwise, and returns the
 * oracle's own selection in sel[] (a prefix of its own candidates). */
static size_t select_candidates(swap_cand *c, size_t n, long long capacity, or_block **sel)
{
    long long n_sure = 0, n_maybe = 0, n_own = 0;
    size_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        if (c[i].sure) {
            /* certainly a candidate: certainly selected while even every
             * uncertain one before it would fit, certainly not once the sure
             * ones before it fill the capacity */
            if (!(n_sure + n_maybe < capacity) && n_sure < capacity && c[i].b)
                c[i].b->swap_amb = 1;
            ++n_sure;
        } else if (c[i].maybe) {
            if (c[i].b && n_sure < capacity) c[i].b->swap_amb = 1;
            ++n_maybe;
        }
        if (c[i].own) {
            if (n_own < capacity) sel[k++] = c[i].b;
            ++n_own;
        }
    }
    return k;
}

static int swap_push(swap_cand **v, size_t *n, size_t *cap, swap_cand c)
{
    if (*n == *cap) {
        size_t nc = *cap ? 2 * *cap : 1024;
        swap_cand *nv = (swap_cand *)realloc(*v, nc * sizeof(swap_cand));
        if (!nv) return -1;
        *v = nv;
        *cap = nc;
    }
    (*v)[(*n)++] = c;
    return 0;
}

static int swap_view(frame_ctx *fc, int width, int height, const double intr[4],
                     const double M[16])
{
    static const float dummy = 0.0f;  /* the view needs no depth */
    return make_frame(fc, &dummy, width, height, intr, M);
}

int or_swap_out(or_scene *s, int width, int height, const double intr[4],
                const double world_to_cam[16], double margin_px, double max_depth,
                long long capacity, long long *n_moved)
{
    frame_ctx fc;
    if (!s || capacity < 1 || !(margin_px >= 0.0) ||
        swap_view(&fc, width, height, intr, world_to_cam))
        return -1;
    swap_cand *c = NULL;
    size_t nc = 0, cc = 0;
    or_block **sel = (or_block **)malloc((s->n ? s->n : 1) * sizeof(or_block *));
    if (!sel) return -3;
    for (size_t i = 0; i < s->n; ++i) {
        or_block *b = s->blocks[i];
        /* reading: a device block whose host copy is still to be merged is
         * not swapped out (it is swapped in first). The GPU may also hold
         * ghosts, may lack blocks no segment met robustly, and may have
         * decided earlier swaps of a flagged block otherwise. */
        const int ghost = b->t_alloc < 0 && b->t_poss >= 0;
        const int resident = b->allocated && !b->on_host;
        if (!resident && !ghost && !b->swap_amb) continue;
        const int certain = resident && !b->swap_amb && b->t_rob >= 0;
        int amb = 0;
        const int vis = block_visible(&s->p, &fc, margin_px, max_depth, b->key, &amb);
        const int own = resident && !vis;
        const int sure = certain && !vis && !amb;
        const int maybe = !sure && (!vis || amb);
        if (!own && !maybe) continue;
        if (swap_push(&c, &nc, &cc, (swap_cand){ ghost ? NULL : b, own, sure, maybe })) {
            free(c); free(sel);
            return -3;
        }
    }
    const size_t k = select_candidates(c, nc, capacity, sel);
    for (size_t i = 0; i < k; ++i) {
        or_block *b = sel[i];
        b->h_sdf = b->sdf; b->h_w = b->w; b->h_vflag = b->vflag; b->h_rgbw = b->rgbw;
        b->sdf = NULL; b->w = NULL; b->vflag = NULL; b->rgbw = NULL;
        b->allocated = 0;
        b->on_host = 1;
        b->swapped = 1;
        s->n_alloc--;
    }
    free(c);
    free(sel);
    if (n_moved) *n_moved = (long long)k;
    return 0;
}

/* Secondary integration of a host voxel into a device voxel. reading: an
 * empty side (weight 0) yields the other unchanged; otherwise the two running
 * averages combine by their weights, F = (w_h F_h + w_d F_d) / (w_h + w_d),
 * and w = min(w_h + w_d, maxW). For int16 storage the average is taken on
 * the stored integers and truncated toward zero (the C conversion of the
 * voxel type), so it is exact; FP16 rounds the real value to nearest even. */
static void merge_voxel(const or_params *p, double Fh, int wh, double *Fd, uint8_t *wd)
{
    if (wh == 0) return;
    if (*wd == 0) {
        *Fd = Fh;
        *wd = (uint8_t)wh;
        return;
    }
    const int w = wh + *wd;
    if (p->storage == OR_STORAGE_I16) {
        const long qh = lround(Fh * 32767.0), qd = lround(*Fd * 32767.0);
        *Fd = or_i16_to_float((int16_t)((wh * qh + (long)*wd * qd) / w));
    } else {
        *Fd = store_value(p->storage, ((double)wh * Fh + (double)*wd * *Fd) / (double)w);
    }
    *wd = (uint8_t)(w > p->max_weight ? p->max_weight : w);
}

/* reading: colours combine by their colour weights, per channel the integer
 * average rounded half up, weight min(sum, maxW); an empty side yields the
 * other. */
static void merge_colour(const or_params *p, const uint8_t *h, uint8_t *d)
{
    const int wh = h[3], wd = d[3];
    if (wh == 0) return;
    if (wd == 0) {
        memcpy(d, h, 4);
        return;
    }
    const int w = wh + wd;
    for (int c = 0; c < 3; ++c) {
        const int num = wh * h[c] + wd * d[c];
        d[c] = (uint8_t)((2 * num + w) / (2 * w));
    }
    d[3] = (uint8_t)(w > p->max_weight ? p->max_weight : w);
}

int or_swap_merge_voxel(const or_params *p, double Fh, int wh, double *Fd, int *wd)
{
    if (!p || !Fd || !wd || wh < 0 || wh > 255 || *wd < 0 || *wd > 255) return -1;
    uint8_t w = (uint8_t)*wd;
    merge_voxel(p, Fh, wh, Fd, &w);
    *wd = w;
    return 0;
}

int or_swap_merge_colour(const or_params *p, const uint8_t h[4], uint8_t d[4])
{
    if (!p || !h || !d) return -1;
    merge_colour(p, h, d);
    return 0;
}

int or_swap_in(or_scene *s, int width, int height, const double intr[4],
               const double world_to_cam[16], double margin_px, double max_depth,
               long long capacity, long long *n_moved, long long *n_merged)
{
    frame_ctx fc;
    if (!s || capacity < 1 || !(margin_px >= 0.0) ||
        swap_view(&fc, width, height, intr, world_to_cam))
        return -1;
    /* reading: blocks that are only visible (no fresh device block yet) are
     * brought in only if the pool has room for a full call's worth of new
     * blocks. The GPU's device block count may differ from the oracle's by
     * the ghosts it holds and the robust-less blocks it lacks: if that range
     * straddles the rule, the decision is uncertain. */
    long long ghosts = 0, fragile = 0;
    for (size_t i = 0; i < s->n; ++i) {
        const or_block *b = s->blocks[i];
        if (b->t_alloc < 0 && b->t_poss >= 0) ++ghosts;
        if (b->allocated && (b->t_rob < 0 || b->swap_amb)) ++fragile;
        if (!b->allocated && b->swap_amb) ++ghosts;
    }
    int prefetch = 1, prefetch_amb = 0;
    if (s->p.pool_blocks > 0) {
        prefetch = s->p.pool_blocks - s->n_alloc >= capacity;
        const int lo = s->p.pool_blocks - (s->n_alloc + ghosts) >= capacity;
        const int hi = s->p.pool_blocks - (s->n_alloc - fragile) >= capacity;
        prefetch_amb = lo != hi;
    }
    swap_cand *c = NULL;
    size_t nc = 0, cc = 0;
    or_block **sel = (or_block **)malloc((s->n ? s->n : 1) * sizeof(or_block *));
    if (!sel) return -3;
    for (size_t i = 0; i < s->n; ++i) {
        or_block *b = s->blocks[i];
        /* a host block with a fresh device block is always a candidate; one
         * without is a candidate when visible and the pool has room. The GPU
         * may also hold host copies of ghosts and of flagged blocks. */
        const int ghost = b->t_alloc < 0 && b->t_poss >= 0;
        if (!b->on_host && !ghost && !b->swap_amb) continue;
        int amb = 0;
        const int vis = block_visible(&s->p, &fc, margin_px, max_depth, b->key, &amb);
        const int own = b->on_host && (b->allocated || (prefetch && vis));
        const int sure = b->on_host && !b->swap_amb &&
                         (b->allocated || (prefetch && !prefetch_amb && vis && !amb));
        const int maybe = !sure && (b->allocated || ghost || b->swap_amb ||
                                    ((prefetch || prefetch_amb) && (vis || amb)));
        if (!own && !maybe) continue;
        if (swap_push(&c, &nc, &cc, (swap_cand){ ghost ? NULL : b, own, sure, maybe })) {
            free(c); free(sel);
            return -3;
        }
    }
    const size_t k = select_candidates(c, nc, capacity, sel);
    long long merged = 0;
    for (size_t i = 0; i < k; ++i) {
        or_block *b = sel[i];
        if (b->allocated) {
            for (int l = 0; l < BLOCK_VOXELS; ++l) {
                merge_voxel(&s->p, b->h_sdf[l], b->h_w[l], &b->sdf[l], &b->w[l]);
                b->vflag[l] |= b->h_vflag[l];
                merge_colour(&s->p, b->h_rgbw + 4 * l, b->rgbw + 4 * l);
            }
            free(b->h_sdf); free(b->h_w); free(b->h_vflag); free(b->h_rgbw);
            ++merged;
        } else {
            b->sdf = b->h_sdf; b->w = b->h_w; b->vflag = b->h_vflag; b->rgbw = b->h_rgbw;
            b->allocated = 1;
            s->n_alloc++;
        }
        b->h_sdf = NULL; b->h_w = NULL; b->h_vflag = NULL; b->h_rgbw = NULL;
        b->on_host = 0;
    }
    free(c);
    free(sel);
    if (n_moved) *n_moved = (long long)k;
    if (n_merged) *n_merged = merged;
    return 0;
}

long long or_num_host_blocks(const or_scene *s)
{
    if (!s) return -1;
    long long n = 0;
    for (size_t i = 0; i < s->n; ++i) n += s->blocks[i]->on_host;
    return n;
}

int or_read_host(const or_scene *s, int32_t *keys, double *sdf, uint8_t *w,
                 uint8_t *rgbw, uint8_t *vflag, uint8_t *bflag)
{
    if (!s) return -1;
    size_t k = 0;
    for (size_t i = 0; i < s->n; ++i) {
        const or_block *b = s->blocks[i];
        if (!b->on_host) continue;
        if (keys) memcpy(keys + 3 * k, b->key, 3 * sizeof(int32_t));
        if (sdf) memcpy(sdf + BLOCK_VOXELS * k, b->h_sdf, BLOCK_VOXELS * sizeof(double));
        if (w) memcpy(w + BLOCK_VOXELS * k, b->h_w, BLOCK_VOXELS);
        if (rgbw) memcpy(rgbw + 4 * BLOCK_VOXELS * k, b->h_rgbw, 4 * BLOCK_VOXELS);
        if (vflag) memcpy(vflag + BLOCK_VOXELS * k, b->h_vflag, BLOCK_VOXELS);
        if (bflag) {
            uint8_t f = OR_BLOCK_SWAPPED;
            if (b->t_rob < 0) f |= OR_BLOCK_MEMBERSHIP_AMBIGUOUS;
            if (b->t_poss != b->t_rob) f |= OR_BLOCK_HISTORY_AMBIGUOUS;
            if (b->swap_amb) f |= OR_BLOCK_SWAP_AMBIGUOUS;
            bflag[k] = f;
        }
        ++k;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* dense-volume form (Section 3.2)                                     */
/* ------------------------------------------------------------------ */

struct or_dense {
    or_params p;
    int origin[3], size[3];
    int nb[3];                /* blocks per axis */
    double *sdf;
    uint8_t *w;
    uint8_t *mask;            /* block allocated */
    hit_vec hits;
};

or_dense *or_dense_create(const or_params *p, const int origin[3],
                          const int size[3])
{
    if (!p || !origin || !size) return NULL;
    for (int a = 0; a < 3; ++a)
        if (size[a] <= 0 || size[a] % BLOCK || origin[a] % BLOCK) return NULL;
    or_dense *d = (or_dense *)calloc(1, sizeof(or_dense));
    if (!d) return NULL;
    d->p = *p;
    size_t n = (size_t)size[0] * size[1] * size[2];
    for (int a = 0; a < 3; ++a) {
        d->origin[a] = origin[a];
        d->size[a] = size[a];
        d->nb[a] = size[a] / BLOCK;
    }
    d->sdf = (double *)malloc(n * sizeof(double));
    d->w = (uint8_t *)calloc(n, 1);
    d->mask = (uint8_t *)calloc((size_t)d->nb[0] * d->nb[1] * d->nb[2], 1);
    if (!d->sdf || !d->w || !d->mask) { or_dense_destroy(d); return NULL; }
    for (size_t i = 0; i < n; ++i) d->sdf[i] = SDF_INITIAL;
    return d;
}

void or_dense_destroy(or_dense *d)
{
    if (!d) return;
    free(d->sdf);
    free(d->w);
    free(d->mask);
    free(d->hits.v);
    free(d);
}

int or_dense_integrate(or_dense *d, const float *depth, int width, int height,
                       const double intr[4], const double world_to_cam[16])
{
    if (!d) return -1;
    frame_ctx fc;
    if (make_frame(&fc, depth, width, height, intr, world_to_cam)) return -1;
    if (frame_hits(&fc, d->p.voxel_size, d->p.mu, d->p.delta_b, &d->hits))
        return -3;
    int outside = 0;
    for (size_t i = 0; i < d->hits.n; ++i) {
        const hit_rec *h = &d->hits.v[i];
        if (!(h->bits & OR_HIT_EXACT)) continue;
        long long b[3];
        int in = 1;
        for (int a = 0; a < 3; ++a) {
            b[a] = (long long)h->key[a] - d->origin[a] / BLOCK;
            if (b[a] < 0 || b[a] >= d->nb[a]) in = 0;
        }
        if (!in) { outside = 1; continue; }
        d->mask[(b[2] * d->nb[1] + b[1]) * d->nb[0] + b[0]] = 1;
    }
    /* every voxel of the grid, in x-fastest order */
    for (int z = 0; z < d->size[2]; ++z)
        for (int y = 0; y < d->size[1]; ++y)
            for (int x = 0; x < d->size[0]; ++x) {
                long long v[3] = { (long long)d->origin[0] + x,
                                   (long long)d->origin[1] + y,
                                   (long long)d->origin[2] + z };
                long long b[3] = { x / BLOCK, y / BLOCK, z / BLOCK };
                if (!d->mask[(b[2] * d->nb[1] + b[1]) * d->nb[0] + b[0]])
                    continue;
                size_t li = ((size_t)z * d->size[1] + y) * d->size[0] + x;
                int W = d->w[li], flag = 0;
                update_voxel(&d->p, &fc, v, &d->sdf[li], &W, &flag, NULL);
                d->w[li] = (uint8_t)W;
            }
    return outside;
}

int or_dense_read(const or_dense *d, double *sdf, uint8_t *w)
{
    if (!d) return -1;
    size_t n = (size_t)d->size[0] * d->size[1] * d->size[2];
    if (sdf) memcpy(sdf, d->sdf, n * sizeof(double));
    if (w) memcpy(w, d->w, n);
    return 0;
}

/* ------------------------------------------------------------------ */
/* single-block / single-voxel re-simulation (sampled checks)          */
/* ------------------------------------------------------------------ */

int or_block_hit_frames(const int32_t key[3], const float *depth,
                        int n_frames, int width, int height,
                        const double intr[4], const double *poses,
                        const or_params *p, uint8_t *hits)
{
    if (!key || !depth || !poses || !p || !hits || n_frames < 0) return -2;
    const double s = p->voxel_size, db = p->delta_b;
    for (int t = 0; t < n_frames; ++t) {
        frame_ctx fc;
        const float *D = depth + (size_t)t * width * height;
        if (make_frame(&fc, D, width, height, intr, poses + 16 * t)) return -2;
        /* Only pixels whose centre lies in the image of the grown box can
         * have a ray point inside it: when every box corner is in front of
         * the camera, the image of the box is inside the bounding rectangle
         * of the projected corners. Otherwise every pixel is tested. */
        int u0 = 0, u1 = width - 1, v0 = 0, v1 = height - 1;
        double lo[3], hi[3];
        block_box(key, s, db, lo, hi);
        int all_front = 1;
        double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
        for (int c = 0; c < 8; ++c) {
            double pw[3] = { (c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1],
                             (c & 4) ? hi[2] : lo[2] };
            double pc[3];
            apply_affine(fc.M, pw, pc);
            if (!(pc[2] > 1e-9)) { all_front = 0; break; }
            double x = fc.fx * pc[0] / pc[2] + fc.cx;
            double y = fc.fy * pc[1] / pc[2] + fc.cy;
            if (x < xmin) xmin = x;
            if (x > xmax) xmax = x;
            if (y < ymin) ymin = y;
            if (y > ymax) ymax = y;
        }
        if (all_front) {
            double a = floor(xmin) - 1, b = ceil(xmax) + 1;
            double c = floor(ymin) - 1, e = ceil(ymax) + 1;
            u0 = a < 0 ? 0 : (a > width - 1 ? width : (int)a);
            u1 = b > width - 1 ? width - 1 : (b < 0 ? -1 : (int)b);
            v0 = c < 0 ? 0 : (c > height - 1 ? height : (int)c);
            v1 = e > height - 1 ? height - 1 : (e < 0 ? -1 : (int)e);
        }
        int bits = 0;
        for (int v = v0; v <= v1; ++v)
            for (int u = u0; u <= u1; ++u) {
                float dd = D[(size_t)v * width + u];
                if (!valid_depth(dd)) continue;
                double P0[3], P1[3];
                band_segment(&fc, u, v, (double)dd, p->mu, P0, P1);
                bits |= hit_bits(P0, P1, key, s, db);
            }
        hits[t] = (uint8_t)bits;
    }
    return 0;
}

typedef struct { int alloc; double F; int W; } vstate;

static int vstate_cmp(const void *a, const void *b)
{
    const vstate *x = (const vstate *)a, *y = (const vstate *)b;
    if (x->alloc != y->alloc) return x->alloc < y->alloc ? -1 : 1;
    if (x->W != y->W) return x->W < y->W ? -1 : 1;
    if (x->F < y->F) return -1;
    if (x->F > y->F) return 1;
    return 0;
}

/* All outcomes of one frame for one allocated state, both branches of every
 * decision within the margins. Appends to out (capacity cap). */
static int frame_outcomes(const or_params *p, const frame_ctx *fc,
                          const long long v[3], vstate st, vstate *out,
                          int *n, int cap)
{
#define PUSH(S) do { if (*n >= cap) return -1; out[(*n)++] = (S); } while (0)
    const double s = p->voxel_size, mu = p->mu;
    double pm[3] = { (double)v[0] * s, (double)v[1] * s, (double)v[2] * s };
    double pc[3];
    apply_affine(fc->M, pm, pc);
    int z_amb = fabs(pc[2]) < p->delta_z;
    if (pc[2] <= 0.0 || z_amb) {
        PUSH(st);                     /* rejected (or possibly rejected) */
        if (pc[2] <= 0.0) return 0;   /* a tiny positive GPU z projects far
                                         outside the image: rejected too */
    }
    double x = fc->fx * pc[0] / pc[2] + fc->cx;
    double y = fc->fy * pc[1] / pc[2] + fc->cy;
    const double xmax = fc->width - 2, ymax = fc->height - 2;
    int in = !(x < 1.0 || x > xmax || y < 1.0 || y > ymax);
    int b_amb = near_value(x, 1.0, p->delta_px) || near_value(x, xmax, p->delta_px) ||
                near_value(y, 1.0, p->delta_px) || near_value(y, ymax, p->delta_px);
    if (!in || b_amb) PUSH(st);
    if (!in && !b_amb) return 0;
    /* candidate pixel columns / rows */
    int ixs[2], iys[2], nx = 0, ny = 0;
    {
        double t = x + 0.5;
        int i0 = (int)floor(t);
        ixs[nx++] = i0;
        double f = t - floor(t);
        if (f < p->delta_px && i0 - 1 >= 0) ixs[nx++] = i0 - 1;
        else if (f > 1.0 - p->delta_px && i0 + 1 <= fc->width - 1) ixs[nx++] = i0 + 1;
        t = y + 0.5;
        i0 = (int)floor(t);
        iys[ny++] = i0;
        f = t - floor(t);
        if (f < p->delta_px && i0 - 1 >= 0) iys[ny++] = i0 - 1;
        else if (f > 1.0 - p->delta_px && i0 + 1 <= fc->height - 1) iys[ny++] = i0 + 1;
    }
    for (int a = 0; a < nx; ++a)
        for (int b = 0; b < ny; ++b) {
            int ix = ixs[a], iy = iys[b];
            if (ix < 0 || ix >= fc->width || iy < 0 || iy >= fc->height) {
                PUSH(st);
                continue;
            }
            float dm = fc->depth[(size_t)iy * fc->width + ix];
            if (!valid_depth(dm)) { PUSH(st); continue; }
            double eta = (double)dm - pc[2];
            int e_amb = near_value(eta, -mu, p->delta_eta);
            if (eta < -mu || e_amb) PUSH(st);
            if (eta < -mu && !e_amb) continue;
            double f = eta / mu;
            if (f > 1.0) f = 1.0;
            vstate ns = st;
            ns.F = store_value(p->storage,
                               ((double)st.W * st.F + f) / (double)(st.W + 1));
            ns.W = st.W + 1 > p->max_weight ? p->max_weight : st.W + 1;
            PUSH(ns);
        }
    return 0;
#undef PUSH
}

int or_voxel_candidates(const int32_t voxel[3], const float *depth,
                        int n_frames, int width, int height,
                        const double intr[4], const double *poses,
                        const or_params *p, const uint8_t *block_hits,
                        double *sdf_out, uint8_t *w_out, int max_out)
{
    if (!voxel || !depth || !poses || !p || !block_hits || max_out < 1)
        return -2;
    const int cap = 24 * max_out + 64;
    vstate *cur = (vstate *)malloc(cap * sizeof(vstate));
    vstate *nxt = (vstate *)malloc(cap * sizeof(vstate));
    if (!cur || !nxt) { free(cur); free(nxt); return -2; }
    int n = 1;
    cur[0].alloc = 0; cur[0].F = SDF_INITIAL; cur[0].W = 0;
    long long v[3] = { voxel[0], voxel[1], voxel[2] };
    int rc = 0;
    for (int t = 0; t < n_frames && rc == 0; ++t) {
        frame_ctx fc;
        if (make_frame(&fc, depth + (size_t)t * width * height, width, height,
                       intr, poses + 16 * t)) { rc = -2; break; }
        int m = 0;
        for (int i = 0; i < n && rc == 0; ++i) {
            vstate st = cur[i];
            /* allocation: certain on a robust hit, optional on a graze */
            int options[2], no = 0;
            if (st.alloc || (block_hits[t] & OR_HIT_SHRUNK)) options[no++] = 1;
            else if (block_hits[t] & OR_HIT_GROWN) { options[no++] = 0; options[no++] = 1; }
            else options[no++] = 0;
            for (int o = 0; o < no && rc == 0; ++o) {
                vstate a = st;
                a.alloc = options[o];
                if (!a.alloc) {
                    if (m >= cap) { rc = -1; break; }
                    nxt[m++] = a;
                    continue;
                }
                if (frame_outcomes(p, &fc, v, a, nxt, &m, cap)) rc = -1;
            }
        }
        if (rc) break;
        qsort(nxt, m, sizeof(vstate), vstate_cmp);
        int u = 0;
        for (int i = 0; i < m; ++i)
            if (u == 0 || vstate_cmp(&nxt[u - 1], &nxt[i]) != 0) nxt[u++] = nxt[i];
        if (u > max_out) { rc = -1; break; }
        vstate *tmp = cur; cur = nxt; nxt = tmp;
        n = u;
    }
    if (rc == 0) {
        for (int i = 0; i < n; ++i) {
            sdf_out[i] = cur[i].alloc ? cur[i].F : NAN;
            w_out[i] = cur[i].alloc ? (uint8_t)cur[i].W : 255;
        }
        rc = n;
    }
    free(cur);
    free(nxt);
    return rc;
}
