/*
 * raycast_oracle.c -- plain FP64 CPU oracle for the raycast of the InfiniTAM
 * report (Section 4.4). TEST INFRASTRUCTURE ONLY, under the same rules as
 * tsdf_oracle.c: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it, and it shares no code with the CUDA library.
 *
 * The report describes the raycast in prose; this file takes its steps in
 * that order. Where the prose leaves a detail open the choice is marked
 * "reading:".
 *
 * 1. Search range ("expected depths"). Every allocated block's closed box
 *    [8b s, 8(b+1) s]^3 is put into camera coordinates; the 2D bounding box
 *    of its eight projected corners is filled with the minimum and maximum
 *    camera depth of the corners, and a pixel keeps the smallest minimum and
 *    the largest maximum over the boxes that cover it.
 *    reading: a pixel (u, v) is covered when its centre (u, v) lies in the
 *    closed 2D box; z_near clips whole blocks: a block with a corner nearer
 *    than z_near covers no pixel (geometry within a block of the near plane
 *    is not rendered). The range is full resolution.
 *
 * 2. March (the five-state machine), along the ray through the pixel centre,
 *    parametrised by the distance t from the camera centre in voxel units:
 *    P(t) = O + t D, D a unit vector; the search starts at the range's z_lo
 *    and ends past z_hi.
 *      SEARCH_BLOCK_COARSE: steps of one block (8 voxels) while the block
 *        containing P is not allocated; on reaching an allocated block, one
 *        step of 8 voxels back and SEARCH_BLOCK_FINE.
 *      SEARCH_BLOCK_FINE: steps of mu while the value at P cannot be read;
 *        a readable negative value is WRONG_SIDE (no surface), a readable
 *        non-negative one starts SEARCH_SURFACE.
 *      SEARCH_SURFACE: steps of the value times mu, the value being a
 *        conservative estimate of the distance to the surface; an unreadable
 *        sample returns to SEARCH_BLOCK_FINE; a negative value is
 *        BEHIND_SURFACE, which ends the march.
 *    reading: values are read by trilinear interpolation of the 8 voxels of
 *    the cell floor(P) + {0,1}^3, readable when all 8 lie in allocated blocks
 *    (an unobserved voxel reads its initial value 1); a surface step is at
 *    least one voxel.
 *
 * 3. Refinement: two steps of (interpolated value) x mu from the first
 *    negative sample (the second only if its start can be read); the surface
 *    point is P at the result.
 *
 * Ambiguity flags: the CUDA path computes in FP32 and can take the other
 * side of a decision that sits within a margin of its threshold (a pixel
 * centre on a projected box edge, a block near z_near, a sample near a block
 * or cell boundary where the readable / allocated answer changes, a value
 * near 0, the last sample near the end of the range). Such pixels are
 * flagged; unflagged pixels must agree exactly in hit / no hit.
 */
#include "tsdf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define BLOCK 8
#define BLOCK_VOXELS 512

struct or_volume {
    long long n;
    int32_t *keys; /* [n][3], sorted by (x, y, z) */
    double *sdf;   /* [n][512] in the sorted order */
};

typedef struct {
    int32_t k[3];
    long long src;
} keyed;

static int cmp_key3(const int32_t *a, const int32_t *b)
{
    for (int i = 0; i < 3; ++i)
        if (a[i] != b[i])
            return a[i] < b[i] ? -1 : 1;
    return 0;
}

static int cmp_keyed(const void *a, const void *b)
{
    return cmp_key3(((const keyed *)a)->k, ((const keyed *)b)->k);
}

or_volume *or_volume_create(const int32_t *keys, const double *sdf, long long n)
{
    if (n < 0 || (n > 0 && (!keys || !sdf)))
        return NULL;
    or_volume *v = calloc(1, sizeof(*v));
    if (!v)
        return NULL;
    keyed *order = calloc((size_t)(n > 0 ? n : 1), sizeof(keyed));
    v->keys = malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(int32_t));
    v->sdf = malloc((size_t)(n > 0 ? n : 1) * BLOCK_VOXELS * sizeof(double));
    if (!order || !v->keys || !v->sdf) {
        free(order);
        or_volume_destroy(v);
        return NULL;
    }
    for (long long i = 0; i < n; ++i) {
        memcpy(order[i].k, keys + 3 * i, 3 * sizeof(int32_t));
        order[i].src = i;
    }
    qsort(order, (size_t)n, sizeof(keyed), cmp_keyed);
    for (long long i = 0; i < n; ++i) {
        if (i > 0 && cmp_key3(order[i - 1].k, order[i].k) == 0) {
            free(order);
            or_volume_destroy(v);
            return NULL; /* duplicate key */
        }
        memcpy(v->keys + 3 * i, order[i].k, 3 * sizeof(int32_t));
        memcpy(v->sdf + (size_t)i * BLOCK_VOXELS,
               sdf + (size_t)order[i].src * BLOCK_VOXELS,
               BLOCK_VOXELS * sizeof(double));
    }
    v->n = n;
    free(order);
    return v;
}

void or_volume_destroy(or_volume *v)
{
    if (!v)
        return;
    free(v->keys);
    free(v->sdf);
    free(v);
}

/* index of block b in the sorted array, or -1 (binary search) */
static long long find_block(const or_volume *v, const long b[3])
{
    int32_t k[3] = {(int32_t)b[0], (int32_t)b[1], (int32_t)b[2]};
    long long lo = 0, hi = v->n - 1;
    while (lo <= hi) {
        long long mid = lo + (hi - lo) / 2;
        int c = cmp_key3(v->keys + 3 * mid, k);
        if (c == 0)
            return mid;
        if (c < 0)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* floor(x / 8) for integers of either sign */
static long floor_div8(long x)
{
    return x >= 0 ? x / BLOCK : -((-x + BLOCK - 1) / BLOCK);
}

/* stored value of integer voxel (x, y, z); 0 if its block is absent */
static int voxel_value(const or_volume *v, long x, long y, long z, double *out)
{
    const long b[3] = {floor_div8(x), floor_div8(y), floor_div8(z)};
    const long long i = find_block(v, b);
    if (i < 0)
        return 0;
    const long lx = x - BLOCK * b[0], ly = y - BLOCK * b[1], lz = z - BLOCK * b[2];
    *out = v->sdf[(size_t)i * BLOCK_VOXELS + lx + BLOCK * ly + BLOCK * BLOCK * lz];
    return 1;
}

/* the eight voxel values of the cell with lower corner c (corner k at
 * c + (k & 1, k >> 1 & 1, k >> 2 & 1)); 0 if one of them is absent */
static int cell_values(const or_volume *v, const long c[3], double val[8])
{
    for (int k = 0; k < 8; ++k)
        if (!voxel_value(v, c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + ((k >> 2) & 1),
                         &val[k]))
            return 0;
    return 1;
}

/* Trilinear interpolation at P (voxel units); also (each may be NULL) the
 * largest difference between two voxels of the cell along one edge (a bound
 * on how fast the value can change per voxel of position) and the gradient
 * of the interpolant at P. */
static int read_interp(const or_volume *v, const double P[3], double *sdf, double *edge,
                       double grad[3])
{
    long c[3];
    double f[3], val[8];
    for (int i = 0; i < 3; ++i) {
        c[i] = (long)floor(P[i]);
        f[i] = P[i] - (double)c[i];
    }
    if (!cell_values(v, c, val))
        return 0;
    const double x00 = (1.0 - f[0]) * val[0] + f[0] * val[1];
    const double x10 = (1.0 - f[0]) * val[2] + f[0] * val[3];
    const double x01 = (1.0 - f[0]) * val[4] + f[0] * val[5];
    const double x11 = (1.0 - f[0]) * val[6] + f[0] * val[7];
    const double y0 = (1.0 - f[1]) * x00 + f[1] * x10;
    const double y1 = (1.0 - f[1]) * x01 + f[1] * x11;
    *sdf = (1.0 - f[2]) * y0 + f[2] * y1;
    if (edge) {
        double e = 0.0;
        for (int k = 0; k < 8; ++k)
            for (int a = 0; a < 3; ++a)
                if (!(k & (1 << a))) {
                    const double d = fabs(val[k | (1 << a)] - val[k]);
                    if (d > e)
                        e = d;
                }
        *edge = e;
    }
    if (grad) {
        grad[0] = (1 - f[1]) * (1 - f[2]) * (val[1] - val[0]) + f[1] * (1 - f[2]) * (val[3] - val[2]) +
                  (1 - f[1]) * f[2] * (val[5] - val[4]) + f[1] * f[2] * (val[7] - val[6]);
        grad[1] = (1 - f[0]) * (1 - f[2]) * (val[2] - val[0]) + f[0] * (1 - f[2]) * (val[3] - val[1]) +
                  (1 - f[0]) * f[2] * (val[6] - val[4]) + f[0] * f[2] * (val[7] - val[5]);
        grad[2] = (1 - f[0]) * (1 - f[1]) * (val[4] - val[0]) + f[0] * (1 - f[1]) * (val[5] - val[1]) +
                  (1 - f[0]) * f[1] * (val[6] - val[2]) + f[0] * f[1] * (val[7] - val[3]);
    }
    return 1;
}

int or_volume_read(const or_volume *v, const double P[3], double *sdf)
{
    if (!v || !P || !sdf)
        return -1;
    return read_interp(v, P, sdf, NULL, NULL);
}

/* Position within `margin` of a lattice of spacing `cell`: per axis the
 * neighbouring index an FP32 evaluation might pick (-1, 0 or +1). */
static int near_boundary(const double P[3], double cell, double margin, long base[3], int alt[3])
{
    int any = 0;
    for (int i = 0; i < 3; ++i) {
        base[i] = (long)floor(P[i] / cell);
        const double r = P[i] - cell * (double)base[i];
        alt[i] = r < margin ? -1 : (r > cell - margin ? 1 : 0);
        any |= alt[i] != 0;
    }
    return any;
}

/* Could the allocated / not allocated answer for the block containing P
 * change within the position margin? */
static int block_ambiguous(const or_volume *v, const double P[3], double margin)
{
    long base[3];
    int alt[3];
    if (!near_boundary(P, BLOCK, margin, base, alt))
        return 0;
    const int here = find_block(v, base) >= 0;
    for (int m = 1; m < 8; ++m) {
        long b[3];
        int used = 1;
        for (int i = 0; i < 3; ++i) {
            if (m & (1 << i)) {
                if (!alt[i])
                    used = 0;
                b[i] = base[i] + alt[i];
            } else {
                b[i] = base[i];
            }
        }
        if (used && (find_block(v, b) >= 0) != here)
            return 1;
    }
    return 0;
}

/* Could the readable / unreadable answer at P change within the margin? */
static int read_ambiguous(const or_volume *v, const double P[3], double margin)
{
    long base[3];
    int alt[3];
    double val[8];
    if (!near_boundary(P, 1.0, margin, base, alt))
        return 0;
    const int here = cell_values(v, base, val);
    for (int m = 1; m < 8; ++m) {
        long c[3];
        int used = 1;
        for (int i = 0; i < 3; ++i) {
            if (m & (1 << i)) {
                if (!alt[i])
                    used = 0;
                c[i] = base[i] + alt[i];
            } else {
                c[i] = base[i];
            }
        }
        if (used && cell_values(v, c, val) != here)
            return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* poses                                                               */
/* ------------------------------------------------------------------ */

static int pose_ok(const double M[16])
{
    for (int i = 0; i < 16; ++i)
        if (!isfinite(M[i]))
            return 0;
    return M[12] == 0.0 && M[13] == 0.0 && M[14] == 0.0 && M[15] == 1.0;
}

/* inverse of the affine map x -> R x + t (row-major 4x4 with last row
 * 0 0 0 1): Li = R^-1 (adjugate / determinant), ti = -Li t */
static int invert_affine(const double M[16], double Li[9], double ti[3])
{
    const double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8],
                 h = M[9], k = M[10];
    const double det = a * (e * k - f * h) - b * (d * k - f * g) + c * (d * h - e * g);
    if (!(fabs(det) > 1e-300))
        return 0;
    Li[0] = (e * k - f * h) / det;
    Li[1] = (c * h - b * k) / det;
    Li[2] = (b * f - c * e) / det;
    Li[3] = (f * g - d * k) / det;
    Li[4] = (a * k - c * g) / det;
    Li[5] = (c * d - a * f) / det;
    Li[6] = (d * h - e * g) / det;
    Li[7] = (b * g - a * h) / det;
    Li[8] = (a * e - b * d) / det;
    for (int r = 0; r < 3; ++r)
        ti[r] = -(Li[3 * r] * M[3] + Li[3 * r + 1] * M[7] + Li[3 * r + 2] * M[11]);
    return 1;
}

static int params_ok(const or_ray_params *p)
{
    return p && p->voxel_size > 0.0 && p->mu > 0.0 && p->z_near > 0.0 && p->delta_px >= 0.0 &&
           p->delta_z >= 0.0 && p->delta_v >= 0.0 && p->delta_sdf >= 0.0;
}

/* ------------------------------------------------------------------ */
/* 1. search range                                                     */
/* ------------------------------------------------------------------ */

static void fill_rect(double *lo, double *hi, int W, int u0, int u1, int v0, int v1, double zlo,
                      double zhi)
{
    for (int y = v0; y <= v1; ++y)
        for (int x = u0; x <= u1; ++x) {
            const size_t i = (size_t)y * W + x;
            if (zlo < lo[i])
                lo[i] = zlo;
            if (zhi > hi[i])
                hi[i] = zhi;
        }
}

/* pixel centres u with a <= u <= b, clipped to [0, n - 1]; empty if u0 > u1 */
static void pixel_span(double a, double b, int n, int *u0, int *u1)
{
    const double lo = ceil(a), hi = floor(b);
    *u0 = lo < 0.0 ? 0 : (lo > n ? n : (int)lo);
    *u1 = hi > n - 1 ? n - 1 : (hi < -1.0 ? -1 : (int)hi);
}

int or_expected_depth(const or_volume *v, int W, int H, const double intr[4], const double M[16],
                      const or_ray_params *p, double *range, uint8_t *flags)
{
    if (!v || W < 1 || H < 1 || !intr || !M || !range || !params_ok(p) || !pose_ok(M))
        return -1;
    const size_t np = (size_t)W * H;
    double *ex_lo = malloc(np * sizeof(double)), *ex_hi = malloc(np * sizeof(double));
    double *su_lo = malloc(np * sizeof(double)), *su_hi = malloc(np * sizeof(double));
    double *mb_lo = malloc(np * sizeof(double)), *mb_hi = malloc(np * sizeof(double));
    if (!ex_lo || !ex_hi || !su_lo || !su_hi || !mb_lo || !mb_hi) {
        free(ex_lo); free(ex_hi); free(su_lo); free(su_hi); free(mb_lo); free(mb_hi);
        return -3;
    }
    for (size_t i = 0; i < np; ++i) {
        ex_lo[i] = su_lo[i] = mb_lo[i] = INFINITY;
        ex_hi[i] = su_hi[i] = mb_hi[i] = -INFINITY;
    }
    const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    const double s = p->voxel_size, zn = p->z_near, dpx = p->delta_px, dz = p->delta_z;
    for (long long b = 0; b < v->n; ++b) {
        double cam[8][3], zmin = INFINITY, zmax = -INFINITY;
        for (int k = 0; k < 8; ++k) {
            const double w[3] = {(BLOCK * (double)v->keys[3 * b] + BLOCK * (k & 1)) * s,
                                 (BLOCK * (double)v->keys[3 * b + 1] + BLOCK * ((k >> 1) & 1)) * s,
                                 (BLOCK * (double)v->keys[3 * b + 2] + BLOCK * ((k >> 2) & 1)) * s};
            for (int r = 0; r < 3; ++r)
                cam[k][r] = M[4 * r] * w[0] + M[4 * r + 1] * w[1] + M[4 * r + 2] * w[2] + M[4 * r + 3];
            if (cam[k][2] < zmin)
                zmin = cam[k][2];
            if (cam[k][2] > zmax)
                zmax = cam[k][2];
        }
        if (zmin < zn - dz)
            continue; /* a corner nearer than the near plane: clipped */
        /* within the margin the FP32 path may clip it or not */
        const int near_amb = zmin < zn + dz;
        double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
        for (int k = 0; k < 8; ++k) {
            const double u = fx * cam[k][0] / cam[k][2] + cx;
            const double vv = fy * cam[k][1] / cam[k][2] + cy;
            if (u < umin) umin = u;
            if (u > umax) umax = u;
            if (vv < vmin) vmin = vv;
            if (vv > vmax) vmax = vv;
        }
        int u0, u1, v0, v1;
        pixel_span(umin, umax, W, &u0, &u1);
        pixel_span(vmin, vmax, H, &v0, &v1);
        if (zmin >= zn && u0 <= u1 && v0 <= v1)
            fill_rect(ex_lo, ex_hi, W, u0, u1, v0, v1, zmin, zmax);
        pixel_span(umin + dpx, umax - dpx, W, &u0, &u1);
        pixel_span(vmin + dpx, vmax - dpx, H, &v0, &v1);
        if (!near_amb && u0 <= u1 && v0 <= v1)
            fill_rect(su_lo, su_hi, W, u0, u1, v0, v1, zmin, zmax);
        pixel_span(umin - dpx, umax + dpx, W, &u0, &u1);
        pixel_span(vmin - dpx, vmax + dpx, H, &v0, &v1);
        if (u0 <= u1 && v0 <= v1)
            fill_rect(mb_lo, mb_hi, W, u0, u1, v0, v1, zmin, zmax);
    }
    for (size_t i = 0; i < np; ++i) {
        range[2 * i] = ex_lo[i];
        range[2 * i + 1] = ex_hi[i];
        if (flags)
            flags[i] = (su_lo[i] != mb_lo[i] || su_hi[i] != mb_hi[i]) ? OR_RAY_RANGE_AMBIGUOUS : 0;
    }
    free(ex_lo); free(ex_hi); free(su_lo); free(su_hi); free(mb_lo); free(mb_hi);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 2-3. march and refinement                                           */
/* ------------------------------------------------------------------ */

enum { SEARCH_BLOCK_COARSE, SEARCH_BLOCK_FINE, SEARCH_SURFACE };

typedef struct {
    double O[3], D[3]; /* P(t) = O + t D, voxel units, |D| = 1 */
    double t_lo, t_hi;
} ray;

static void at(const ray *r, double t, double P[3])
{
    for (int i = 0; i < 3; ++i)
        P[i] = r->O[i] + t * r->D[i];
}

/* Is a sign decision on this interpolated value too close to call? The
 * margin grows with how fast the value changes across the cell. */
static int sign_ambiguous(double sdf, double edge, const or_ray_params *p)
{
    return fabs(sdf) < p->delta_sdf + edge * p->delta_v;
}

/* Error growth of one step whose length is mu * (value read at the sample):
 * a distance error e before it becomes |1 + mu dsdf/dt| e, plus what an
 * error in the sample's position does to the value read (at most the cell's
 * steepest edge difference times sqrt(3) per voxel) and a rounding term. */
static double grow(double B, double mu_v, const double grad[3], const double D[3], double edge)
{
    const double slope = grad[0] * D[0] + grad[1] * D[1] + grad[2] * D[2];
    return fabs(1.0 + mu_v * slope) * B + mu_v * sqrt(3.0) * edge + 1.0;
}

/* March one ray; returns 1 with the surface at t_out, 0 without one.
 * *gain receives a bound on how much a per-sample position error (of an
 * evaluation in lower precision) can have moved the surface point, in units
 * of that error: the start and steps of constant length carry it unchanged,
 * steps whose length is a value read scale it (grow), and the final point
 * adds its own. */
static int march(const or_volume *v, const ray *r, const or_ray_params *p, double *t_out,
                 int *amb, int *n_steps, double *gain)
{
    const double mu_v = p->mu / p->voxel_size, dv = p->delta_v;
    double t = r->t_lo, P[3], sdf, edge, grad[3], B = 1.0;
    int state = SEARCH_BLOCK_COARSE;
    *n_steps = 0;
    for (;;) {
        if (fabs(t - r->t_hi) < dv)
            *amb = 1;
        if (t > r->t_hi)
            return 0;
        at(r, t, P);
        ++*n_steps;
        if (state == SEARCH_BLOCK_COARSE) {
            if (block_ambiguous(v, P, dv))
                *amb = 1;
            const long b[3] = {(long)floor(P[0] / BLOCK), (long)floor(P[1] / BLOCK),
                               (long)floor(P[2] / BLOCK)};
            if (find_block(v, b) >= 0) {
                t -= BLOCK; /* one step back, then the finer search */
                state = SEARCH_BLOCK_FINE;
            } else {
                t += BLOCK;
            }
            continue;
        }
        if (read_ambiguous(v, P, dv))
            *amb = 1;
        if (!read_interp(v, P, &sdf, &edge, grad)) {
            state = SEARCH_BLOCK_FINE;
            t += mu_v;
            continue;
        }
        if (sign_ambiguous(sdf, edge, p))
            *amb = 1;
        if (state == SEARCH_BLOCK_FINE && sdf < 0.0)
            return 0; /* WRONG_SIDE: entered a block from behind its surface */
        state = SEARCH_SURFACE;
        if (sdf < 0.0) {
            /* BEHIND_SURFACE: two interpolation steps back onto the surface */
            B = grow(B, mu_v, grad, r->D, edge);
            t += sdf * mu_v;
            at(r, t, P);
            if (read_ambiguous(v, P, dv))
                *amb = 1;
            if (read_interp(v, P, &sdf, &edge, grad)) {
                B = grow(B, mu_v, grad, r->D, edge);
                t += sdf * mu_v;
            }
            *t_out = t;
            *gain = B + 1.0;
            return 1;
        }
        const double step = sdf * mu_v;
        if (step > 1.0) {
            B = grow(B, mu_v, grad, r->D, edge);
            t += step;
        } else {
            t += 1.0;
        }
    }
}

int or_raycast(const or_volume *v, int W, int H, const double intr[4], const double M[16],
               const or_ray_params *p, const double *range, const uint8_t *range_flags,
               const int64_t *pixels, long long n, double *points, uint8_t *flags,
               int32_t *steps, double *gain)
{
    if (!v || W < 1 || H < 1 || !intr || !M || !range || !points || n < 0 || !params_ok(p) ||
        !pose_ok(M))
        return -1;
    double Li[9], ti[3];
    if (!invert_affine(M, Li, ti))
        return -1;
    const double s = p->voxel_size;
    for (long long j = 0; j < n; ++j) {
        const long long pix = pixels ? pixels[j] : j;
        if (pix < 0 || pix >= (long long)W * H)
            return -2;
        const int u = (int)(pix % W), vv = (int)(pix / W);
        double *out = points + 4 * j;
        out[0] = out[1] = out[2] = out[3] = 0.0;
        uint8_t fl = range_flags ? (range_flags[pix] & OR_RAY_RANGE_AMBIGUOUS) : 0;
        int nst = 0;
        double g = 0.0;
        const double z_lo = range[2 * pix], z_hi = range[2 * pix + 1];
        if (z_lo <= z_hi) {
            /* camera ray through the pixel centre, at camera depth 1 */
            const double rc[3] = {(u - intr[2]) / intr[0], (vv - intr[3]) / intr[1], 1.0};
            double E[3];
            for (int i = 0; i < 3; ++i)
                E[i] = Li[3 * i] * rc[0] + Li[3 * i + 1] * rc[1] + Li[3 * i + 2] * rc[2];
            const double len = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
            ray r;
            for (int i = 0; i < 3; ++i) {
                r.O[i] = ti[i] / s;
                r.D[i] = E[i] / len;
            }
            /* camera depth z is at distance z * len along the ray */
            r.t_lo = z_lo * len / s;
            r.t_hi = z_hi * len / s;
            double t_hit;
            int amb = 0;
            if (march(v, &r, p, &t_hit, &amb, &nst, &g)) {
                double P[3];
                at(&r, t_hit, P);
                out[0] = P[0] * s;
                out[1] = P[1] * s;
                out[2] = P[2] * s;
                out[3] = 1.0;
            }
            if (amb)
                fl |= OR_RAY_MARCH_AMBIGUOUS;
        }
        if (flags)
            flags[j] = fl;
        if (steps)
            steps[j] = nst;
        if (gain)
            gain[j] = g;
    }
    return 0;
}
