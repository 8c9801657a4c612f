/*
 * icp_oracle.c -- plain FP64 CPU oracle for the depth tracker's linearised
 * point-to-plane system (InfiniTAM report, Section 4.1). TEST
 * INFRASTRUCTURE ONLY, under the same rules as tsdf_oracle.c: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it,
 * and it shares no code with the CUDA library.
 *
 * The tracker renders a point map V and a normal map N of the model from
 * the reference pose (Section 4.4), projects every point p of the new depth
 * image onto them and measures its distance from the tangent plane there,
 * r = (T p - V)^T N, T being the current pose estimate; the pose minimising
 * the linearised sum of r^2 solves a 6x6 linear system. This file computes
 * that system's terms.
 *
 * reading (the report gives the steps, not the details):
 *   - normals: N(u, v) = normalised (V(u+1, v) - V(u-1, v)) x
 *     (V(u, v+1) - V(u, v-1)); invalid on the image border, where a
 *     neighbour has no point, or where the cross product vanishes. (The
 *     sign of N does not change the system.)
 *   - association: p (camera) = d ((u - cx)/fx, (v - cy)/fy, 1) for a pixel
 *     with a finite d > 0; its world point P = T^-1 p (T = current
 *     world->camera pose); q = M_ref P in the reference camera; rejected if
 *     q.z <= 0; the reference pixel is the nearest, (floor(x + 1/2),
 *     floor(y + 1/2)) with x = fx q.x / q.z + cx, and must lie in the image
 *     and have a point and a normal; rejected if |P - V| > max_dist.
 *   - linearisation: a small motion (w, t) applied to the world point,
 *     P' = P + w x P + t, so r(w, t) = r + (P x N).w + N.t and the row is
 *     J = (P x N, N).
 *   - terms: H = sum J J^T (the 21 entries of its upper triangle, row by
 *     row), g = sum J r (6), E = sum r^2 and the inlier count.
 *
 * Ambiguity: a pixel whose reference-pixel rounding, image-border test,
 * q.z > 0 test or distance test lies within a margin of its threshold is
 * flagged; for each of the 29 terms the oracle reports the largest change
 * any other outcome of those decisions could make (slack), and the sum of
 * |term| over all inlier pixels (scale, for a rounding tolerance).
 */
#include "tsdf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NTERMS 29

static int finite_point(const float *p)
{
    return p[3] == 1.0f && isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
}

int or_icp_normals(const float *points, int width, int height, double *normals)
{
    if (!points || !normals || width < 3 || height < 3)
        return -1;
    for (int v = 0; v < height; ++v)
        for (int u = 0; u < width; ++u) {
            double *n = normals + 4 * ((size_t)v * width + u);
            n[0] = n[1] = n[2] = n[3] = 0.0;
            if (u == 0 || v == 0 || u == width - 1 || v == height - 1)
                continue;
            const float *c = points + 4 * ((size_t)v * width + u);
            const float *l = c - 4, *r = c + 4;
            const float *t = c - 4 * (size_t)width, *b = c + 4 * (size_t)width;
            if (!finite_point(c) || !finite_point(l) || !finite_point(r) || !finite_point(t) ||
                !finite_point(b))
                continue;
            const double du[3] = {(double)r[0] - l[0], (double)r[1] - l[1], (double)r[2] - l[2]};
            const double dv[3] = {(double)b[0] - t[0], (double)b[1] - t[1], (double)b[2] - t[2]};
            const double x[3] = {du[1] * dv[2] - du[2] * dv[1], du[2] * dv[0] - du[0] * dv[2],
                                 du[0] * dv[1] - du[1] * dv[0]};
            const double len = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            if (!(len > 0.0))
                continue;
            n[0] = x[0] / len;
            n[1] = x[1] / len;
            n[2] = x[2] / len;
            n[3] = 1.0;
        }
    return 0;
}

typedef struct {
    double Tinv[12]; /* current camera -> world, rows of [R | t] */
    double Mref[12]; /* world -> reference camera */
    double fx, fy, cx, cy;
    int width, height;
    const float *points;
    const double *normals;
    double max_dist;
} icp_ctx;

static void affine(const double A[12], const double p[3], double out[3])
{
    for (int r = 0; r < 3; ++r)
        out[r] = A[4 * r] * p[0] + A[4 * r + 1] * p[1] + A[4 * r + 2] * p[2] + A[4 * r + 3];
}

/* 29 terms of pixel with world point P against reference pixel (ix, iy);
 * returns 1 for an inlier (terms written), 0 if rejected; *near_dist set if
 * the distance test was within the margin */
static int pixel_terms(const icp_ctx *c, const double P[3], int ix, int iy, double dd,
                       double out[NTERMS], int *near_dist)
{
    if (ix < 0 || iy < 0 || ix >= c->width || iy >= c->height)
        return 0;
    const size_t k = (size_t)iy * c->width + ix;
    const float *V = c->points + 4 * k;
    const double *N = c->normals + 4 * k;
    if (!finite_point(V) || N[3] != 1.0)
        return 0;
    const double diff[3] = {P[0] - V[0], P[1] - V[1], P[2] - V[2]};
    const double dist2 = diff[0] * diff[0] + diff[1] * diff[1] + diff[2] * diff[2];
    const double m2 = c->max_dist * c->max_dist;
    if (fabs(dist2 - m2) < dd * m2)
        *near_dist = 1;
    if (dist2 > m2)
        return 0;
    const double r = diff[0] * N[0] + diff[1] * N[1] + diff[2] * N[2];
    const double J[6] = {P[1] * N[2] - P[2] * N[1], P[2] * N[0] - P[0] * N[2],
                         P[0] * N[1] - P[1] * N[0], N[0], N[1], N[2]};
    int t = 0;
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b)
            out[t++] = J[a] * J[b];
    for (int a = 0; a < 6; ++a)
        out[t++] = J[a] * r;
    out[t++] = r * r;
    out[t++] = 1.0;
    return 1;
}

static int near_rounding(double x, double delta)
{
    const double f = (x + 0.5) - floor(x + 0.5);
    return f < delta || f > 1.0 - delta;
}

int or_icp_reduce(const float *depth, int width, int height, const double intr[4],
                  const double cur_world_to_cam[16], const double ref_world_to_cam[16],
                  const float *points, const double *normals, double max_dist,
                  const double margins[3], double *sums, double *slack, double *scale,
                  uint8_t *flags)
{
    if (!depth || !intr || !cur_world_to_cam || !ref_world_to_cam || !points || !normals ||
        !sums || width < 3 || height < 3 || !(max_dist > 0.0) || !margins)
        return -1;
    const double *M = cur_world_to_cam;
    for (int i = 0; i < 16; ++i)
        if (!isfinite(M[i]) || !isfinite(ref_world_to_cam[i]))
            return -1;
    if (M[12] != 0.0 || M[13] != 0.0 || M[14] != 0.0 || M[15] != 1.0)
        return -1;
    icp_ctx c;
    /* inverse of the current pose: the adjugate of its rotation part */
    const double a = M[0], b = M[1], cc = M[2], d = M[4], e = M[5], f = M[6], g = M[8],
                 h = M[9], k = M[10];
    const double det = a * (e * k - f * h) - b * (d * k - f * g) + cc * (d * h - e * g);
    if (!(fabs(det) > 1e-300))
        return -1;
    const double Ri[9] = {(e * k - f * h) / det, (cc * h - b * k) / det, (b * f - cc * e) / det,
                          (f * g - d * k) / det, (a * k - cc * g) / det, (cc * d - a * f) / det,
                          (d * h - e * g) / det, (b * g - a * h) / det, (a * e - b * d) / det};
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q)
            c.Tinv[4 * r + q] = Ri[3 * r + q];
        c.Tinv[4 * r + 3] = -(Ri[3 * r] * M[3] + Ri[3 * r + 1] * M[7] + Ri[3 * r + 2] * M[11]);
        for (int q = 0; q < 4; ++q)
            c.Mref[4 * r + q] = ref_world_to_cam[4 * r + q];
    }
    c.fx = intr[0];
    c.fy = intr[1];
    c.cx = intr[2];
    c.cy = intr[3];
    c.width = width;
    c.height = height;
    c.points = points;
    c.normals = normals;
    c.max_dist = max_dist;
    const double dpx = margins[0], dz = margins[1], dd = margins[2];
    for (int t = 0; t < NTERMS; ++t) {
        sums[t] = 0.0;
        if (slack)
            slack[t] = 0.0;
        if (scale)
            scale[t] = 0.0;
    }
    for (int v = 0; v < height; ++v)
        for (int u = 0; u < width; ++u) {
            const size_t pix = (size_t)v * width + u;
            if (flags)
                flags[pix] = 0;
            const float dm = depth[pix];
            if (!(isfinite(dm) && dm > 0.0f))
                continue;
            const double p[3] = {dm * ((u - c.cx) / c.fx), dm * ((v - c.cy) / c.fy), (double)dm};
            double P[3], q[3];
            affine(c.Tinv, p, P);
            affine(c.Mref, P, q);
            int amb = fabs(q[2]) < dz;
            if (q[2] <= 0.0 && !amb)
                continue;
            double own[NTERMS];
            int own_in = 0, near_dist = 0;
            int ix = 0, iy = 0;
            double x = 0.0, y = 0.0;
            if (q[2] > 0.0) {
                x = c.fx * q[0] / q[2] + c.cx;
                y = c.fy * q[1] / q[2] + c.cy;
                ix = (int)floor(x + 0.5);
                iy = (int)floor(y + 0.5);
                own_in = pixel_terms(&c, P, ix, iy, dd, own, &near_dist);
                if (near_rounding(x, dpx) || near_rounding(y, dpx))
                    amb = 1;
            }
            if (near_dist)
                amb = 1;
            if (own_in) {
                for (int t = 0; t < NTERMS; ++t) {
                    sums[t] += own[t];
                    if (scale)
                        scale[t] += fabs(own[t]);
                }
            }
            if (!amb)
                continue;
            if (flags)
                flags[pix] = 1;
            if (!slack)
                continue;
            /* other outcomes: rejected (0), or any of the neighbouring
             * reference pixels the rounding could pick */
            double worst[NTERMS];
            for (int t = 0; t < NTERMS; ++t)
                worst[t] = own_in ? fabs(own[t]) : 0.0;
            if (q[2] > 0.0 || fabs(q[2]) < dz) {
                const double qz = q[2] > 0.0 ? q[2] : dz;
                const double xs = c.fx * q[0] / qz + c.cx, ys = c.fy * q[1] / qz + c.cy;
                const int bx = (int)floor(xs + 0.5), by = (int)floor(ys + 0.5);
                for (int oy = -1; oy <= 1; ++oy)
                    for (int ox = -1; ox <= 1; ++ox) {
                        double alt[NTERMS];
                        int nd = 0;
                        if (!pixel_terms(&c, P, bx + ox, by + oy, dd, alt, &nd))
                            continue;
                        for (int t = 0; t < NTERMS; ++t) {
                            const double dlt = fabs(alt[t] - (own_in ? own[t] : 0.0));
                            if (dlt > worst[t])
                                worst[t] = dlt;
                        }
                    }
            }
            for (int t = 0; t < NTERMS; ++t)
                slack[t] += worst[t];
        }
    return 0;
}

/* reading: one level of the tracker's resolution hierarchy (the report uses
 * one, without details) halves each dimension; a coarse pixel holds the mean
 * of the valid (finite, > 0) depths of its 2x2 fine pixels, 0 where none is
 * valid. The sum runs in a fixed order (top-left, top-right, bottom-left,
 * bottom-right) in float and is divided by the count, as an FP32 evaluation
 * does. Its intrinsics are fx / 2 and (cx - 1/2) / 2 (a coarse pixel centre
 * is the centre of its 2x2 block). */
int or_icp_downsample(const float *depth, int width, int height, float *out)
{
    if (!depth || !out || width < 2 || height < 2)
        return -1;
    const int w2 = width / 2, h2 = height / 2;
    for (int v = 0; v < h2; ++v)
        for (int u = 0; u < w2; ++u) {
            float sum = 0.0f;
            int n = 0;
            for (int k = 0; k < 4; ++k) {
                const float d = depth[(size_t)(2 * v + (k >> 1)) * width + 2 * u + (k & 1)];
                if (isfinite(d) && d > 0.0f) {
                    sum += d;
                    ++n;
                }
            }
            out[(size_t)v * w2 + u] = n ? sum / (float)n : 0.0f;
        }
    return 0;
}
