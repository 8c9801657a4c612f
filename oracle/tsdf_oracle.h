/*
 * tsdf_oracle.h -- plain FP64 CPU oracle for depth-frame fusion into a
 * voxel-block TSDF (InfiniTAM technical report, arXiv 1410.0925).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the slow, obviously-correct
 * definition that the CUDA path is checked against. Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it; the product path
 * never does, and it shares no code, header, helper or table with the CUDA
 * library.
 *
 * What it computes (per frame, in order):
 *   1. Allocation set (Section 4.2, first stage): for every pixel with a
 *      finite depth d > 0, the segment of its ray between camera depths
 *      d - mu and d + mu, mapped to world coordinates with the inverse pose;
 *      every 8x8x8-voxel block whose closed box [8bs, 8(b+1)s]^3 meets that
 *      segment is allocated (new blocks start at sdf = 1, w = 0; Section 3.1
 *      voxel type).
 *   2. Integration (Section 4.3):
 *      every voxel of every allocated block is projected, compared with the
 *      depth at the nearest pixel and, if it is not more than mu behind the
 *      surface, averaged in with weight 1; the weight is capped at maxW.
 * Between frames, swapping (Section 5, or_swap_out / or_swap_in below) moves
 * blocks between the device copy and a host copy.
 *
 * There is no hash table here: blocks live in an array sorted by their block
 * coordinate, which is the plain definition that hashing reproduces.
 *
 * Ambiguity flags: an FP32 GPU cannot reproduce FP64 decisions that sit on a
 * threshold (pixel rounding, image border, eta = -mu, a segment grazing a
 * block). The oracle flags such decisions within the margins in or_params and
 * provides or_voxel_candidates(), which re-simulates one voxel with both
 * outcomes of every flagged decision.
 */
#ifndef TSDF_ORACLE_H
#define TSDF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_STORAGE_F32 = 0, OR_STORAGE_I16 = 1, OR_STORAGE_F16 = 2 };

/* block flag bits (or_read) */
enum {
    OR_BLOCK_MEMBERSHIP_AMBIGUOUS = 1, /* never met by a segment robustly   */
    OR_BLOCK_HISTORY_AMBIGUOUS = 2,    /* first allocation frame not unique */
    OR_BLOCK_SWAP_AMBIGUOUS = 4,       /* a swap decision lay within a margin */
    OR_BLOCK_SWAPPED = 8               /* was swapped out at least once       */
};

/* per-frame hit bits of one block (or_block_hit_frames) */
enum { OR_HIT_GROWN = 1, OR_HIT_EXACT = 2, OR_HIT_SHRUNK = 4 };

typedef struct {
    double voxel_size;   /* s, metres                                      */
    double mu;           /* truncation band, metres                        */
    int max_weight;      /* maxW of the integration listing                */
    int storage;         /* OR_STORAGE_*                                   */
    long long pool_blocks; /* block capacity; <= 0 means unlimited          */
    double delta_px;     /* pixel-coordinate ambiguity margin (pixels)     */
    double delta_eta;    /* eta = -mu ambiguity margin (metres)            */
    double delta_b;      /* block-box grow/shrink margin (metres)          */
    double delta_z;      /* camera-z = 0 ambiguity margin (metres)         */
} or_params;

typedef struct or_scene or_scene;

or_scene *or_create(const or_params *p);
void or_destroy(or_scene *s);

/* Fuse one frame. depth: row-major float32 metres, width*height.
 * intr = {fx, fy, cx, cy}; world_to_cam = 4x4 row-major.
 * Returns 0, or 1 if the pool capacity left some new blocks unallocated
 * (those with the lexicographically largest keys), or <0 on bad input. */
int or_integrate(or_scene *s, const float *depth, int width, int height,
                 const double intr[4], const double world_to_cam[16]);

/* Fuse one frame with colour (the voxel type's clr / w_color, Section 3.1):
 * as or_integrate, and every voxel the depth rule updates also averages the
 * colour of the same (nearest) pixel of rgb, an RGBX image registered to the
 * depth (width*height*4 bytes, X ignored): per channel
 * new = (w old + obs) / (w + 1) in float, stored rounded to the nearest
 * integer, w <- min(w + 1, maxW). New blocks start at colour 0, weight 0. */
int or_integrate_rgb(or_scene *s, const float *depth, const uint8_t *rgb, int width,
                     int height, const double intr[4], const double world_to_cam[16]);
/* Colour of the allocated blocks in or_read's order: rgbw [n][512][4]
 * (r, g, b, colour weight), voxel order x + 8y + 64z. */
int or_read_colour(const or_scene *s, uint8_t *rgbw);

long long or_num_blocks(const or_scene *s);
/* Number of voxel writes of the update rule so far (a counter only). */
long long or_total_updates(const or_scene *s);
long long or_num_ghosts(const or_scene *s);

/* Canonical readback of the allocated blocks, sorted by (x, y, z).
 * keys [n][3]; sdf [n][512] (the stored value as a real number: for int16
 * storage q/32767, for fp16 the binary16 value); w, vflag [n][512];
 * bflag, t_alloc [n]. Any output pointer may be NULL. */
int or_read(const or_scene *s, int32_t *keys, double *sdf, uint8_t *w,
            uint8_t *vflag, uint8_t *bflag, int32_t *t_alloc);

/* Keys [n][3] of blocks that a grown box would have allocated but the exact
 * test never did ("ghosts"); a GPU may legitimately hold them. */
int or_read_ghosts(const or_scene *s, int32_t *keys);

/* Swapping (Section 5). The active part of the map is what lies in or near
 * the view; the rest goes to a host copy and comes back when needed.
 *   visibility: a block is visible when some corner of its box is in front
 *     of the camera and either some corner is not, or the bounding box of
 *     its projected corners meets the image rectangle of pixel centres grown
 *     by margin_px on every side (and, if max_depth > 0, its nearest corner
 *     is no farther than max_depth);
 *   or_swap_out: device blocks without a pending host copy that are not
 *     visible move to the host (at most `capacity`, smallest keys first);
 *     their hash entries keep the key, so a later band that meets one
 *     allocates a fresh device block (sdf 1, w 0);
 *   or_swap_in: host blocks that have such a fresh device block, and host
 *     blocks that are visible if the pool has `capacity` free blocks, come
 *     back (at most `capacity`, smallest keys first); a fresh device block
 *     is merged with its host copy voxel by voxel (secondary integration):
 *     an empty side yields the other, else F = (w_h F_h + w_d F_d) / (w_h +
 *     w_d) (int16: on the stored integers, truncated toward zero), w =
 *     min(w_h + w_d, maxW); colour likewise by colour weight, per channel
 *     rounded half up.
 * Blocks whose swap decisions lay within the margins (delta_px, delta_z) or
 * depend on ghosts carry OR_BLOCK_SWAP_AMBIGUOUS. Return 0 or <0 on bad
 * input; n_moved / n_merged may be NULL. */
int or_swap_out(or_scene *s, int width, int height, const double intr[4],
                const double world_to_cam[16], double margin_px, double max_depth,
                long long capacity, long long *n_moved);
int or_swap_in(or_scene *s, int width, int height, const double intr[4],
               const double world_to_cam[16], double margin_px, double max_depth,
               long long capacity, long long *n_moved, long long *n_merged);
long long or_num_host_blocks(const or_scene *s);
/* The secondary integration of one voxel (value as a real number, weights
 * 0..255; *Fd, *wd updated) and of one colour word (r, g, b, weight; d
 * updated), on their own. Return 0, or -1 on bad input. */
int or_swap_merge_voxel(const or_params *p, double Fh, int wh, double *Fd, int *wd);
int or_swap_merge_colour(const or_params *p, const uint8_t h[4], uint8_t d[4]);
/* The visibility rule on its own: 1 visible, 0 not, -1 bad input;
 * *ambiguous (may be NULL) as for the flags above. */
int or_block_visible(const or_params *p, int width, int height, const double intr[4],
                     const double world_to_cam[16], double margin_px, double max_depth,
                     const int32_t key[3], int *ambiguous);
/* The host copies, sorted by key: keys [n][3], sdf / w / vflag [n][512],
 * rgbw [n][512][4], bflag [n]; any pointer may be NULL. */
int or_read_host(const or_scene *s, int32_t *keys, double *sdf, uint8_t *w,
                 uint8_t *rgbw, uint8_t *vflag, uint8_t *bflag);
/* Dense-volume form (Section 3.2): a fixed grid of nx*ny*nz voxels whose
 * voxel (0,0,0) has integer coordinate origin[]. A voxel is updated in a
 * frame only if its block has been allocated by then (same allocation
 * definition), so on a grid that covers every allocated block it must equal
 * the block form exactly. Returns NULL on bad sizes. */
typedef struct or_dense or_dense;
or_dense *or_dense_create(const or_params *p, const int origin[3],
                          const int size[3]);
void or_dense_destroy(or_dense *d);
int or_dense_integrate(or_dense *d, const float *depth, int width, int height,
                       const double intr[4], const double world_to_cam[16]);
/* sdf / w arrays of nx*ny*nz, x fastest */
int or_dense_read(const or_dense *d, double *sdf, uint8_t *w);

/* Per-frame hit bits (OR_HIT_*) of block `key` for frames 0..n_frames-1.
 * depth: n_frames frames of width*height; poses: n_frames 4x4 row-major. */
int or_block_hit_frames(const int32_t key[3], const float *depth,
                        int n_frames, int width, int height,
                        const double intr[4], const double *poses,
                        const or_params *p, uint8_t *hits);

/* Every final (sdf, w) that one voxel can legitimately end with, taking both
 * outcomes of each flagged decision and every admissible allocation frame of
 * its block (from or_block_hit_frames' bits). Writes up to max_out states;
 * returns the count, or -1 if more than max_out distinct states arose, or
 * -2 on bad input. Unallocated final states are reported with w = 255 and
 * sdf = NaN. */
int or_voxel_candidates(const int32_t voxel[3], const float *depth,
                        int n_frames, int width, int height,
                        const double intr[4], const double *poses,
                        const or_params *p, const uint8_t *block_hits,
                        double *sdf_out, uint8_t *w_out, int max_out);

/* Storage conversions, exported so they can be pinned on their own.
 * int16: trunc(x * 32767) (C cast), value = q / 32767 (Section 3.1).
 * fp16: round to nearest binary16, ties to even. */
int16_t or_float_to_i16(double x);
double or_i16_to_float(int16_t q);
double or_round_f16(double x);

/* ------------------------------------------------------------------ */
/* Raycast (Section 4.4): raycast_oracle.c                             */
/* ------------------------------------------------------------------ */

/* A block volume in canonical form: keys [n][3] (block coordinates, any
 * order, no duplicates) and sdf [n][512] (the stored value of each voxel as a
 * real number, voxel order x + 8y + 64z). The volume copies both. */
typedef struct or_volume or_volume;
or_volume *or_volume_create(const int32_t *keys, const double *sdf, long long n);
void or_volume_destroy(or_volume *v);

typedef struct {
    double voxel_size;  /* s, metres                                       */
    double mu;          /* truncation band, metres                         */
    double z_near;      /* near plane of the search range, metres (> 0)    */
    double delta_px;    /* box-projection coverage margin, pixels          */
    double delta_z;     /* near-plane clipping margin, metres (< z_near)   */
    double delta_v;     /* sample-position margin, voxels                  */
    double delta_sdf;   /* sign margin of an interpolated value            */
} or_ray_params;

/* pixel flag bits (or_expected_depth, or_raycast) */
enum { OR_RAY_RANGE_AMBIGUOUS = 1, OR_RAY_MARCH_AMBIGUOUS = 2 };

/* Trilinear read at a point in voxel units (P = world position / s).
 * Returns 1 and the value if all eight voxels of the cell floor(P) + {0,1}^3
 * lie in blocks of the volume, else 0. */
int or_volume_read(const or_volume *v, const double P[3], double *sdf);

/* Search range per pixel (the expected depths). range [H][W][2] receives
 * (z_lo, z_hi) in camera depth (+inf, -inf where no block covers the
 * pixel); flags [H][W] (may be NULL) receives OR_RAY_RANGE_AMBIGUOUS. */
int or_expected_depth(const or_volume *v, int width, int height, const double intr[4],
                      const double world_to_cam[16], const or_ray_params *p,
                      double *range, uint8_t *flags);

/* Cast the rays of n pixels (pixel indices y * width + x; pixels == NULL
 * means all width * height pixels in order) through the search range of
 * or_expected_depth. points [n][4] receives the surface point in world
 * metres and 1, or (0, 0, 0, 0) without a surface; flags [n] (may be NULL)
 * OR_RAY_MARCH_AMBIGUOUS and the pixel's range flag; steps [n] (may be
 * NULL) the number of samples taken; gain [n] (may be NULL) a bound on how
 * far a per-sample position error e (of an evaluation of the same march in
 * lower precision) can move the surface point: at most gain * e (0 without a
 * surface). Steps whose length is mu times a value read scale an earlier
 * error by |1 + mu dsdf/dt| and add the value's own sensitivity to e; the
 * start and constant steps carry it unchanged. */
int or_raycast(const or_volume *v, int width, int height, const double intr[4],
               const double world_to_cam[16], const or_ray_params *p,
               const double *range, const uint8_t *range_flags,
               const int64_t *pixels, long long n, double *points, uint8_t *flags,
               int32_t *steps, double *gain);

/* ------------------------------------------------------------------ */
/* Depth tracker terms (Section 4.1): icp_oracle.c                     */
/* ------------------------------------------------------------------ */

/* Normal map of a point map: points [H][W][4] float (x, y, z world metres,
 * 1 where valid; the raycast's output); normals [H][W][4] receives the
 * normalised cross product of the central differences along x and y, and 1,
 * or zeros on the border / where a neighbour has no point. */
int or_icp_normals(const float *points, int width, int height, double *normals);

/* The 29 terms of the linearised point-to-plane system for a depth image
 * (width * height floats) seen from cur_world_to_cam against the reference
 * maps rendered from ref_world_to_cam (points float [H][W][4], normals
 * double [H][W][4] as or_icp_normals): sums[0..20] = upper triangle of
 * sum J J^T row by row, sums[21..26] = sum J r, sums[27] = sum r^2,
 * sums[28] = inlier count, J = (P x N, N), r = (P - V).N. margins =
 * {pixel (rounding and border), reference depth (q.z = 0), relative
 * distance (|P - V|^2 = max_dist^2)}. slack[29] (may be NULL): per term,
 * the sum over flagged pixels of the largest change another outcome of
 * their flagged decisions could make; scale[29] (may be NULL): the sum of
 * |term| over inliers; flags [H][W] (may be NULL): 1 for flagged pixels. */
int or_icp_reduce(const float *depth, int width, int height, const double intr[4],
                  const double cur_world_to_cam[16], const double ref_world_to_cam[16],
                  const float *points, const double *normals, double max_dist,
                  const double margins[3], double *sums, double *slack, double *scale,
                  uint8_t *flags);

/* One level of the tracker's depth hierarchy: out [height/2][width/2]
 * receives per 2x2 block the mean of its valid depths (float, fixed order),
 * 0 where none is valid. */
int or_icp_downsample(const float *depth, int width, int height, float *out);

#ifdef __cplusplus
}
#endif
#endif
