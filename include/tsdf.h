/*
 * tsdf.h -- C ABI of the GB300 voxel-block TSDF fusion library (libtsdf.so).
 *
 * The library fuses depth frames into a truncated signed distance function
 * stored in 8x8x8-voxel blocks that are addressed through a spatial hash
 * table with an excess (overflow) list, following the InfiniTAM report
 * (Prisacariu et al., arXiv 1410.0925):
 *   - voxel record and fixed-point sdf:          Section 3.1 (ITMVoxel listing)
 *   - voxel blocks, hash table, excess list:      Section 3.3
 *   - allocation (band search, block reservation,
 *     visible-block list):                        Section 4.2
 *   - per-voxel integration rule:                 Section 4.3
 *   - voxel colour:                               Sections 3.1, 4.3
 *   - depth tracker (normals, point-to-plane
 *     terms, Gauss-Newton, depth hierarchy):      Section 4.1
 *   - raycast:                                    Section 4.4
 *   - swapping to a host block array:             Section 5
 *   - the processing pipeline of one camera:      Section 2.1
 *   - main-engine usage (create, write a frame,
 *     process it):                                Section 6
 *
 * Conventions shared by every call:
 *   - Units are metres. Block coordinates b are int16 triples; block b holds
 *     the voxels v = 8b + l, l in [0,8)^3, with linear index
 *     l.x + 8 l.y + 64 l.z in every block array this API reads or writes
 *     (the device keeps another order internally). Voxel v sits at the world
 *     point v * voxel_size.
 *   - Poses are 4x4 row-major double world->camera matrices (the matrix the
 *     integration listing applies to model points); the last row must be
 *     (0, 0, 0, 1).
 *   - Depth images are row-major float32 metres; a pixel is a measurement
 *     iff its value is finite and > 0 (0 and NaN mean "no measurement").
 *   - Every call returns TSDF_OK (0) or a negative TSDF_ERR_* status.
 *     Conditions met by device code (pool or excess list exhausted, a band
 *     block outside the int16 key range, a bounded device loop that gave up)
 *     are recorded in a device status word and returned by the next call
 *     that synchronises (tsdf_sync, tsdf_get_stats, tsdf_num_blocks,
 *     tsdf_read_blocks, tsdf_load_blocks); reporting clears them. The scene
 *     stays usable afterwards.
 *   - All device work of a scene is enqueued on the scene's CUDA stream; no
 *     call synchronises unless its comment says so.
 *   - The library never falls back to a CPU implementation: without a
 *     usable CUDA device, tsdf_scene_create returns TSDF_ERR_CUDA. The only
 *     calls that compute on the host are tsdf_swap_visibility and
 *     tsdf_swap_merge_voxels, which run the swap kernels' own arithmetic on
 *     the CPU for tools and tests; no scene operation uses them.
 */
#ifndef TSDF_H
#define TSDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSDF_OK 0
#define TSDF_ERR_INVALID_ARG (-1)
#define TSDF_ERR_OUT_OF_MEMORY (-2)
#define TSDF_ERR_POOL_EXHAUSTED (-3)   /* block pool had too few free blocks  */
#define TSDF_ERR_EXCESS_EXHAUSTED (-4) /* excess list (or its frame buffer) full */
#define TSDF_ERR_CUDA (-5)             /* a CUDA runtime call failed          */
#define TSDF_ERR_TIMEOUT (-6)          /* a bounded device loop gave up       */
#define TSDF_ERR_CAPACITY (-7)         /* caller buffer too small             */
#define TSDF_ERR_KEY_RANGE (-8)        /* a band block outside int16 coords   */
#define TSDF_ERR_INTERNAL (-9)         /* a device index failed a consistency
                                          check; the access was skipped       */

/* sdf storage forms (Section 3.1 lists short and float voxels; half is an
 * addition of this library) */
#define TSDF_STORAGE_F32 0   /* float sdf, initial 1.0                      */
#define TSDF_STORAGE_I16 1   /* short sdf = (short)(x * 32767), initial 32767 */
#define TSDF_STORAGE_F16 2   /* IEEE binary16 sdf (round to nearest even), 1.0 */

/* Scene parameters (Section 6: ITMSceneParams voxel size and truncation
 * band; Section 3.3: voxel block array and hash table sizes). */
typedef struct {
    float voxel_size;          /* s > 0, metres                                 */
    float mu;                  /* truncation band mu > 0, metres               */
    int32_t max_weight;        /* maxW of the integration listing, 1..255      */
    int32_t hash_buckets_log2; /* ordered part: 2^k buckets, 1 <= k <= 26      */
    int32_t entries_per_bucket;/* entries per bucket, 1..8 ("typically 2")     */
    int32_t excess_entries;    /* unordered excess list length, >= 1           */
    int32_t pool_blocks;       /* voxel block array length, 1..2^24            */
    int32_t storage;           /* TSDF_STORAGE_*                               */
} tsdf_scene_desc;

/* Pinhole depth camera (the listing's projParams_d and image size). */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;     /* >= 3 each */
} tsdf_intrinsics;

/* Counters since creation or the last reset. */
typedef struct {
    int64_t frames;               /* frames integrated                          */
    int64_t allocated_blocks;     /* blocks holding a pool slot                 */
    int64_t last_new_blocks;      /* blocks allocated by the last frame         */
    int64_t last_visible_blocks;  /* blocks the last frame integrated          */
    int64_t last_updated_voxels;  /* voxels whose (sdf, w) the last frame wrote */
    int64_t total_updated_voxels; /* sum over all frames                        */
    int64_t total_visible_blocks; /* sum over all frames                        */
    int64_t excess_used;          /* excess-list entries in use                 */
    int64_t kernel_launches;      /* library kernels launched (host count)      */
} tsdf_stats;

typedef struct tsdf_scene tsdf_scene;

/* Create a scene on the current CUDA device and bind it to `stream` (a
 * cudaStream_t; NULL = the legacy default stream). Allocates the hash table
 * (2^k * entries_per_bucket + excess_entries entries of 16 bytes), the voxel
 * block array (pool_blocks * 512 voxels of 5 / 3 / 3 bytes for F32 / I16 /
 * F16), the free-block stack and per-frame work buffers with cudaMalloc, and
 * initialises them (enqueued on `stream`). The scene owns all of this memory
 * until tsdf_scene_destroy. *out receives the handle.
 * Errors: INVALID_ARG for a NULL pointer or a field out of range,
 * OUT_OF_MEMORY, CUDA. */
int tsdf_scene_create(const tsdf_scene_desc *desc, void *stream,
                      tsdf_scene **out);

/* Free every device buffer of the scene (synchronises its stream first).
 * NULL is accepted and ignored. */
int tsdf_scene_destroy(tsdf_scene *scene);

/* Return the scene to its freshly created state (empty hash table, full
 * free-block stack, zero counters); enqueued, does not synchronise. */
int tsdf_scene_reset(tsdf_scene *scene);

/* Fuse n frames in order: the results are those of n tsdf_integrate calls
 * with device depth. Frame t + 1's allocation runs while frame t is being
 * integrated: allocations run on the scene's stream, integrations on a
 * second stream the scene owns, and the second stream is joined back into
 * the scene's stream before the call returns, so later work on the scene's
 * stream sees all n frames and the call can be captured into a CUDA graph
 * as a whole (the frames' per-frame state alternates between two sets; each
 * frame leaves its set clear). frames[i].scene must be this scene or NULL;
 * depth is DEVICE memory that must stay valid until the scene's stream has
 * executed the enqueued work. Stage timing (tsdf_timing_*) does not record
 * these frames. Nothing synchronises; the depth work buffers grow to the
 * largest image first (an allocation, as in tsdf_integrate). Frames whose
 * depth_on_host is 1 are copied from host memory on a copy stream the
 * scene owns into a ring of two device staging buffers (grown to the
 * largest image on first use), each copy ordered after the allocation two
 * frames back that read the same buffer, so copies run ahead of the
 * allocation stream; the host memory must stay valid, and (for copies that
 * overlap the GPU work) pinned, until the call's work completes. Errors:
 * INVALID_ARG (as tsdf_integrate, or another scene in a frame), CUDA. */
typedef struct tsdf_frame tsdf_frame;
int tsdf_integrate_frames(tsdf_scene *scene, const tsdf_frame *frames, int32_t n);

/* Rebind the scene to another stream. Work already enqueued stays on the
 * old stream: synchronise it first if ordering matters. */
int tsdf_scene_set_stream(tsdf_scene *scene, void *stream);

/* The CUDA device the scene lives on (the device current at creation): all
 * its device buffers and every device pointer given to its calls belong to
 * it. INVALID_ARG for a null scene or output. */
int tsdf_scene_device(const tsdf_scene *scene, int32_t *device);

/* Fuse one depth frame (Section 4.2 allocation, then Section 4.3 integration):
 *   1. every block met by some measured pixel's ray segment between camera
 *      depths d - mu and d + mu is found in the hash table or inserted (a free
 *      bucket entry, else an excess-list entry linked into the bucket's
 *      chain) and, if new, given a block from the free stack, initialised to
 *      sdf = 1, w = 0; no block is dropped by intra-frame collisions;
 *   2. the visible blocks are selected: every allocated block whose voxels
 *      can pass the projection test of the integration rule (a conservative
 *      test; every block new this frame is selected);
 *   3. every voxel of every visible block is updated by the rule: skip if
 *      behind the camera, outside [1, width-2] x [1, height-2], on a pixel
 *      without measurement, or eta = d - z < -mu; else
 *      sdf <- (w sdf + min(1, eta/mu)) / (w + 1), w <- min(w + 1, maxW).
 * depth: width*height floats with row pitch `pitch_elems` (>= width,
 * pitch_elems * height < 2^31). If
 * depth_on_host is nonzero, `depth` is host memory and is copied to the
 * device on the scene's stream inside this call (pinned memory makes the
 * copy asynchronous); else it is device memory that must stay valid until
 * the stream has executed the enqueued work. The pose is copied.
 * Nothing synchronises, and once a frame of this image size (or larger) has
 * been integrated nothing allocates, so the call can then be captured into
 * a CUDA graph (the scene keeps a per-frame depth work buffer, and a host
 * staging buffer for host depth, grown to the largest image seen).
 * Errors: INVALID_ARG (NULL, bad sizes,
 * pose whose last row is not (0,0,0,1) or whose rotation part is singular),
 * CUDA. */
int tsdf_integrate(tsdf_scene *scene, const float *depth, int64_t pitch_elems,
                   int depth_on_host, const tsdf_intrinsics *intr,
                   const double world_to_cam[16]);

/* Colour (the voxel type's clr and w_color of Section 3.1). The report lists
 * only the depth update and says a similar function also updates the colour;
 * here every voxel the depth rule updates also averages the colour of the same
 * (nearest) pixel of a colour image registered to the depth image: per channel
 * new = (w old + obs) / (w + 1) in float (w old + obs is an exact integer, one
 * IEEE division), stored rounded to the nearest integer, and the colour weight
 * becomes min(w + 1, maxW).
 *
 * tsdf_scene_enable_colour allocates 4 bytes per voxel (pool_blocks * 2 KB:
 * r, g, b, colour weight) and sets every colour to 0; from then on new blocks
 * start at colour 0 / weight 0 (also in frames without colour), a reset clears
 * the colours, and blocks loaded by tsdf_load_blocks read colour 0. A scene
 * with colour cannot join a batched step (tsdf_batch_prepare: INVALID_ARG).
 * Enqueued on the scene's stream; idempotent. Errors: OUT_OF_MEMORY, CUDA. */
int tsdf_scene_enable_colour(tsdf_scene *scene);

/* tsdf_integrate with colour: rgb is a DEVICE image of width * height
 * 4-byte pixels (r, g, b, unused), row pitch = width, 4-byte aligned, same
 * camera as the depth; it must stay valid until the stream has executed the
 * enqueued work. Errors: as tsdf_integrate; INVALID_ARG if colour is not
 * enabled, rgb is NULL or misaligned. */
int tsdf_integrate_rgb(tsdf_scene *scene, const float *depth, int64_t pitch_elems,
                       int depth_on_host, const uint8_t *rgb, const tsdf_intrinsics *intr,
                       const double world_to_cam[16]);

/* Canonical colour readback (synchronises), in tsdf_read_blocks' block order:
 * rgbw [n][512][4] uint8 (r, g, b, colour weight), voxel order x + 8y + 64z,
 * caller-owned HOST memory. Capacity and errors as tsdf_read_blocks;
 * INVALID_ARG if colour is not enabled. */
int tsdf_read_colour(tsdf_scene *scene, uint8_t *rgbw, int64_t capacity, int64_t *n_written);

/* Raycast (Section 4.4): render the scene's surface from a camera.
 *   1. search range: every allocated block's box [8bs, 8(b+1)s]^3 is put
 *      into camera coordinates; the pixels whose centres lie in the bounding
 *      box of its eight projected corners get the corners' camera-depth range
 *      (z_near clips whole blocks: one with a corner nearer than z_near covers
 *      no pixel, so geometry within a block of the near plane is not
 *      rendered); a pixel's range is the smallest and largest depth over the
 *      blocks covering it;
 *   2. march along the pixel centre's ray from the range's near end, in
 *      voxel units: steps of one block while the sample's block is not
 *      allocated, then one block back; steps of mu while the trilinear read
 *      fails (a read needs all eight voxels of its cell in allocated blocks;
 *      an unobserved voxel reads 1); a first successful read that is negative
 *      ends the ray without surface (entered from behind); then steps of
 *      max(value * mu, one voxel) until a negative value, or past the range;
 *   3. from the first negative sample two steps of (read value) * mu along
 *      the ray give the surface point.
 * points: DEVICE buffer of width * height float4 (16-byte aligned), row-major:
 * (x, y, z, 1) world metres on a surface, (0, 0, 0, 0) without. range: NULL
 * or a DEVICE buffer of width * height float2 (8-byte aligned) receiving
 * (z_lo, z_hi) per pixel, (+inf, -inf) where no block covers it. Enqueued on
 * the scene's stream after everything before it; nothing synchronises. The
 * first call (and a call with more 16x16 pixel tiles than any before)
 * allocates work buffers: 84 bytes per pool block and 12 bytes per tile;
 * after that the call can be captured into a CUDA graph.
 * Errors: INVALID_ARG (NULL, bad sizes, misaligned buffers, z_near not
 * positive and finite, pose as tsdf_integrate), OUT_OF_MEMORY, CUDA. */
int tsdf_raycast(tsdf_scene *scene, const tsdf_intrinsics *intr,
                 const double world_to_cam[16], float z_near, float *points,
                 float *range);

/* Counters of the most recent raycast (synchronises). */
typedef struct {
  int64_t footprints;      /* blocks whose footprint covers a pixel        */
  int64_t wide_footprints; /* of those, footprints wider than 16 tiles     */
  int64_t steps;           /* samples taken over all rays                  */
  int64_t hits;            /* rays that found a surface                    */
  int64_t guard_stops;     /* rays stopped by the 65536-sample limit       */
} tsdf_raycast_stats;
int tsdf_get_raycast_stats(tsdf_scene *scene, tsdf_raycast_stats *out);

/* Depth tracker (Section 4.1): the linearised point-to-plane system.
 * Reference maps come from a raycast at the reference pose (tsdf_raycast's
 * points); tsdf_icp_normals derives the normal map: per pixel the normalised
 * cross product (V(u+1,v) - V(u-1,v)) x (V(u,v+1) - V(u,v-1)), (0,0,0,0) on
 * the border, where a neighbour has no point, or where it vanishes (its sign
 * does not matter to the system).
 * tsdf_icp_reduce: for every pixel of a depth image with a finite d > 0, the
 * world point P = T^-1 (d ((u-cx)/fx, (v-cy)/fy, 1)) (T = cur_world_to_cam),
 * projected with ref_world_to_cam onto the nearest reference pixel (rejected
 * behind the reference camera, outside the image, without point or normal, or
 * farther than max_dist from the point V there); r = (P - V).N and
 * J = (P x N, N) (a small motion P' = P + w x P + t of the world point). sums
 * (DEVICE, 29 doubles, 8-byte aligned) receives the upper triangle of
 * sum J J^T row by row (21), sum J r (6), sum r^2 and the inlier count,
 * accumulated in FP32 per thread and CTA and as double-floats (hi + lo)
 * across CTAs, in an order that does not depend on scheduling. The host solves H x = -g (the report keeps
 * the solve on the CPU). points / normals: DEVICE width * height float4
 * (16-byte aligned); depth: DEVICE, row pitch pitch_elems. All calls are
 * enqueued on the stream given at creation and can be captured into a CUDA
 * graph; one handle runs one reduction at a time. Errors: INVALID_ARG (NULL,
 * sizes, misalignment, a pose whose last row is not 0 0 0 1 or whose rotation
 * is singular, max_dist not positive), OUT_OF_MEMORY, CUDA. */
typedef struct tsdf_icp tsdf_icp;
int tsdf_icp_create(void *stream, tsdf_icp **out);
int tsdf_icp_destroy(tsdf_icp *icp);
int tsdf_icp_normals(tsdf_icp *icp, const float *points, float *normals, int32_t width,
                     int32_t height);
int tsdf_icp_reduce(tsdf_icp *icp, const float *depth, int64_t pitch_elems,
                    const tsdf_intrinsics *intr, const double cur_world_to_cam[16],
                    const double ref_world_to_cam[16], const float *points,
                    const float *normals, float max_dist, double *sums);
/* One Gauss-Newton step on the device: solve H x = -g (Cholesky, FP64, one
 * thread) from the 29 terms in sums (DEVICE) and apply x = (w, t) as a small
 * motion of the world points, P' = exp(w) P + t (Rodrigues), to the pose
 * (DEVICE, 16 doubles, world->camera, row-major): pose <- pose
 * [exp(w) | t]^-1. With fewer than 6 inliers, or a system that is not
 * positive definite, the pose is kept and the handle's status records it. */
int tsdf_icp_solve(tsdf_icp *icp, const double *sums, double *pose);
/* `iterations` Gauss-Newton iterations with no host round trip: each
 * derives the reduction's constants from the DEVICE pose (in FP64, on the
 * device), reduces the terms (as tsdf_icp_reduce, into sums) and applies
 * tsdf_icp_solve's step to the pose. The reference pose is copied. */
int tsdf_icp_track(tsdf_icp *icp, const float *depth, int64_t pitch_elems,
                   const tsdf_intrinsics *intr, double *pose, const double ref_world_to_cam[16],
                   const float *points, const float *normals, float max_dist,
                   int32_t iterations, double *sums);
/* Synchronise; return and clear the handle's status bits: 1 a device pose was
 * not an invertible affine map, 2 a step had fewer than 6 inliers, 4 a system
 * was not positive definite. */
int tsdf_icp_status(tsdf_icp *icp, int32_t *status);
/* One level of the tracker's resolution hierarchy (the report uses one for
 * convergence): out (DEVICE, (width/2) * (height/2) floats, dense) receives
 * per 2x2 block of depth the mean of its valid (finite, > 0) depths, summed
 * in a fixed order in float, 0 where none is valid. The coarse level's
 * intrinsics are fx / 2, fy / 2, (cx - 1/2) / 2, (cy - 1/2) / 2. */
int tsdf_icp_downsample(tsdf_icp *icp, const float *depth, int64_t pitch_elems, int32_t width,
                        int32_t height, float *out);
/* Intrinsics of level `level` (0 = full resolution) of that hierarchy: each
 * level halves fx and fy, maps cx to (cx - 1/2) / 2 (a coarse pixel centre
 * is the centre of its 2x2 block) and halves width and height (rounding
 * down). Host only. INVALID_ARG for null pointers, invalid intrinsics or a
 * level outside 0..15. */
int tsdf_icp_level_intrinsics(const tsdf_intrinsics *intr, int32_t level, tsdf_intrinsics *out);
/* kernels launched through this handle so far */
int tsdf_icp_kernel_launches(tsdf_icp *icp, int64_t *n);

/* The processing pipeline of one camera (Section 2.1): every frame is
 * tracked against the model rendered from the previous pose, fused at the
 * tracked pose, and the next frame is tracked against the model rendered
 * from that pose. tsdf_engine_process, for frame t > 0:
 *   1. the depth hierarchy (tsdf_icp_downsample, `levels` levels);
 *   2. per level with iterations > 0: the model rendered from the last pose
 *      at that level's intrinsics (tsdf_raycast, z_near) and its normals;
 *   3. coarse to fine, that level's Gauss-Newton iterations on the device
 *      (tsdf_icp_track, max_dist) starting from the last pose;
 *   4. the pose read back (the one synchronisation of a frame); a pose that
 *      is not finite keeps the last one;
 * then for every frame (frame 0 at the initial pose) the fusion at the pose
 * (tsdf_integrate, or tsdf_integrate_rgb when rgb is given), and the pose is
 * written to world_to_cam_out (host). With swap_blocks > 0 the scene swaps
 * (Section 5; tsdf_scene_enable_swapping with that bound): the fusion is
 * preceded by tsdf_swap_in and followed by tsdf_swap_out, both from the
 * frame's pose with swap_margin_px, so what the view sees is on the device
 * when it is fused and rendered. depth (and rgb): DEVICE, as in
 * tsdf_integrate(_rgb). The engine owns its scene (tsdf_engine_scene lends
 * it: readback, raycasts, stats; do not destroy it) and tracker.
 * Errors: INVALID_ARG (a config field out of range: levels 1..4, each
 * level at least 3 x 3 pixels, iterations 0..100, max_dist and z_near
 * positive, swap_blocks 0..pool_blocks, swap_margin_px >= 0; rgb without
 * colour), OUT_OF_MEMORY, CUDA, and those of the calls above. */
typedef struct {
    tsdf_scene_desc scene;
    tsdf_intrinsics intr;      /* the depth camera                               */
    int32_t levels;            /* tracker hierarchy levels, 1..4                 */
    int32_t iterations[4];     /* per level (0 = full resolution); 0 skips it    */
    float max_dist;            /* tracker association distance, metres           */
    float z_near;              /* raycast near plane, metres                     */
    int32_t colour;            /* nonzero: voxel colour, process() takes rgb     */
    int32_t swap_blocks;       /* > 0: swapping, at most this many blocks a call */
    float swap_margin_px;      /* swapping visibility margin, pixels             */
} tsdf_engine_config;
typedef struct tsdf_engine tsdf_engine;
int tsdf_engine_create(const tsdf_engine_config *cfg, const double initial_world_to_cam[16],
                       void *stream, tsdf_engine **out);
int tsdf_engine_destroy(tsdf_engine *engine);
int tsdf_engine_process(tsdf_engine *engine, const float *depth, int64_t pitch_elems,
                        const uint8_t *rgb, double world_to_cam_out[16]);
/* Empty the model and start again from initial_world_to_cam (enqueued). */
int tsdf_engine_reset(tsdf_engine *engine, const double initial_world_to_cam[16]);
int tsdf_engine_scene(tsdf_engine *engine, tsdf_scene **out);
/* the tracker's status bits (tsdf_icp_status), read and cleared */
int tsdf_engine_tracker_status(tsdf_engine *engine, int32_t *status);
/* kernels launched by the engine so far (its scene's and its tracker's) */
int tsdf_engine_kernel_launches(tsdf_engine *engine, int64_t *n);

/* Swapping (Section 5): only the part of the map in or near the view stays
 * in device memory; the rest goes to a host voxel block array with one block
 * slot per hash entry (the hash entry keeps the key, marked as having no
 * device block), and comes back when needed.
 *
 * tsdf_scene_enable_swapping allocates the host array (pinned host memory
 * mapped into the device's address space: n_entries x (512 x (element size +
 * 1) + 2048 with colour) bytes, owned by the scene), the per-entry swap state
 * and work buffers. transfer_blocks (1 .. pool_blocks) bounds the blocks one
 * swap call moves. Enable colour first if it is wanted (afterwards
 * tsdf_scene_enable_colour returns INVALID_ARG). A swapping scene cannot join
 * a batched step. Errors: INVALID_ARG (already enabled, bad bound),
 * OUT_OF_MEMORY, CUDA.
 *
 * Visibility of a block from a view (intrinsics + world_to_cam, as for
 * tsdf_integrate): some corner of its box [8bs, 8(b+1)s]^3 is in front of the
 * camera, and either some corner is not (the block straddles the camera
 * plane) or the bounding box of its projected corners meets the rectangle of
 * pixel centres grown by margin_px on every side, [-1/2 - m, W - 1/2 + m] x
 * [-1/2 - m, H - 1/2 + m], and, if max_depth > 0, its nearest corner is no
 * farther than max_depth metres. Evaluated in FP64.
 *
 * tsdf_swap_out: every device block that is not visible and has no pending
 * host copy is a candidate; up to transfer_blocks of them, smallest (x, y, z)
 * keys first, are copied to the host array and leave the pool (the pool is
 * compacted, so pool indices change). A band that later meets such a block
 * gives it a fresh device block (sdf 1, w 0) in the allocation stage, which
 * then integrates new frames until the block is swapped in.
 *
 * tsdf_swap_in: candidates are the host blocks that have such a fresh device
 * block, and, if the pool has at least transfer_blocks free blocks, the host
 * blocks that are visible; up to transfer_blocks of them, smallest keys
 * first, come back. A fresh device block is merged with its host copy voxel
 * by voxel (secondary integration): a side with weight 0 yields the other;
 * else sdf = (w_h F_h + w_d F_d) / (w_h + w_d) (int16: on the stored integers,
 * truncated toward zero; FP16: rounded to nearest even), w = min(w_h + w_d,
 * maxW); colour likewise by colour weight, per channel rounded half up.
 *
 * Both calls are enqueued on the scene's stream without synchronisation
 * (capturable into a CUDA graph). Errors: INVALID_ARG (swapping not enabled,
 * bad intrinsics, pose not affine or not finite, margin < 0 or not finite,
 * max_depth not finite), CUDA. tsdf_read_blocks, tsdf_raycast and
 * tsdf_lookup_blocks see device blocks only; tsdf_load_blocks returns
 * INVALID_ARG while host copies exist; tsdf_scene_reset clears them. */
typedef struct {
    int64_t host_blocks;         /* blocks with a host copy now                */
    int64_t transfer_blocks;     /* the per-call bound                         */
    int64_t last_out_candidates; /* last swap-out: candidates, blocks moved    */
    int64_t last_out;
    int64_t last_in_candidates;  /* last swap-in: candidates, moved, merged    */
    int64_t last_in;
    int64_t last_merged;
    int64_t total_out, total_in, total_merged;
} tsdf_swap_stats;
int tsdf_scene_enable_swapping(tsdf_scene *scene, int32_t transfer_blocks);
int tsdf_swap_out(tsdf_scene *scene, const tsdf_intrinsics *intr, const double world_to_cam[16],
                  double margin_px, double max_depth);
int tsdf_swap_in(tsdf_scene *scene, const tsdf_intrinsics *intr, const double world_to_cam[16],
                 double margin_px, double max_depth);
/* Synchronises. INVALID_ARG without swapping. */
int tsdf_get_swap_stats(tsdf_scene *scene, tsdf_swap_stats *out);
/* The visibility rule above on the host (the code the swap kernels run,
 * compiled for the CPU; needs no GPU): visible[i] = 1 if block keys[i] (host
 * int16 [n][3]) is visible from the view for a scene of voxel size
 * voxel_size, else 0. Errors: INVALID_ARG as tsdf_swap_out, or a bad voxel
 * size. */
int tsdf_swap_visibility(float voxel_size, const tsdf_intrinsics *intr,
                         const double world_to_cam[16], double margin_px, double max_depth,
                         const int16_t *keys, int64_t n, uint8_t *visible);
/* The secondary integration above on the host (the per-voxel code the
 * swap-in kernel runs, compiled for the CPU; needs no GPU): merges n host
 * voxels (host_sdf in the storage's element type, host_w, optional host_rgbw
 * colour words r | g << 8 | b << 16 | weight << 24) into n device-side voxels
 * (sdf, w, rgbw, updated in place). All pointers are HOST memory; rgbw and
 * host_rgbw are both NULL or both set. Errors: INVALID_ARG (storage,
 * max_weight outside 1..255, n < 0, missing pointers). */
int tsdf_swap_merge_voxels(int32_t storage, int32_t max_weight, int64_t n, const void *host_sdf,
                           const uint8_t *host_w, const uint32_t *host_rgbw, void *sdf,
                           uint8_t *w, uint32_t *rgbw);
/* Canonical readback of the host copies (synchronises), sorted by block
 * coordinate, in tsdf_read_blocks' layout: keys [n][3] int16, sdf [n][512]
 * by storage, w [n][512], rgbw [n][512][4] (colour scenes only; any output
 * may be NULL). Capacity as tsdf_read_blocks. */
int tsdf_read_host_blocks(tsdf_scene *scene, int16_t *keys, void *sdf, uint8_t *w, uint8_t *rgbw,
                          int64_t capacity, int64_t *n_written);

/* Wait for the scene's stream; return (and clear) any recorded device
 * condition. */
int tsdf_sync(tsdf_scene *scene);

/* Synchronise and fill *out. Returns the recorded device condition, if any
 * (the stats are filled either way). */
int tsdf_get_stats(tsdf_scene *scene, tsdf_stats *out);

/* Synchronise and return the number of allocated blocks in *n. */
int tsdf_num_blocks(tsdf_scene *scene, int64_t *n);

/* Canonical readback (synchronises): every allocated block, sorted by block
 * coordinate (x, then y, then z, as signed int16), into caller-owned HOST
 * buffers: keys [n][3] int16; sdf [n][512] of float / int16 / uint16
 * (binary16 bits) by storage; w [n][512] uint8 (any of sdf, w may be NULL to
 * skip it). `capacity` is the number of blocks the buffers hold; if fewer
 * than the allocated count, nothing is written, *n_written receives the
 * required count and TSDF_ERR_CAPACITY is returned. Where blocks sit in the
 * pool and in the hash table is not observable through this call. */
int tsdf_read_blocks(tsdf_scene *scene, int16_t *keys, void *sdf, uint8_t *w,
                     int64_t capacity, int64_t *n_written);

/* Resume from a canonical readback (synchronises): insert the n blocks
 * (host buffers in tsdf_read_blocks' layout and storage) into the scene and
 * write their voxels. Keys already present are overwritten. Errors as
 * tsdf_integrate's allocation (POOL_EXHAUSTED, EXCESS_EXHAUSTED), INVALID_ARG
 * for duplicate keys in the input or a weight above the scene's max_weight
 * (integration never produces one). */
int tsdf_load_blocks(tsdf_scene *scene, const int16_t *keys, const void *sdf,
                     const uint8_t *w, int64_t n);

/* Retrieval (Section 3.3, readVoxel's search): for each of n block keys
 * (host int16 [n][3]) probe its bucket, then the bucket's excess chain; write
 * the block's pool index or -1 if absent into ptr_out (host int32 [n]).
 * Synchronises. */
int tsdf_lookup_blocks(tsdf_scene *scene, const int16_t *keys, int64_t n,
                       int32_t *ptr_out);

/* Per-stage device timing (instrumentation, not part of the method).
 * tsdf_timing_begin allocates max_frames x 3 CUDA events and makes every
 * following tsdf_integrate record them around its stages (at most
 * max_frames frames; later frames are not timed). Event records are stream
 * operations, so a tsdf_integrate captured into a CUDA graph records them on
 * every replay. Stages (one kernel each): 0 band allocation, find-or-insert
 * and the frame's commit (excess list, free-stack pop), 1 visible-block
 * selection, new-block initialisation and integration (and the frame's
 * counter bookkeeping). With integration_only nonzero only the two events
 * around stage 1 are recorded (less perturbation of the timed work).
 * tsdf_timing_read synchronises and writes, for the n_frames frames
 * recorded so far, the times in ms of each frame's 3 stage boundaries
 * (before stage 0, before stage 1, after stage 1) relative to the first
 * boundary recorded, ms[frame][3]; boundaries not recorded read NaN
 * (capacity = rows the buffer holds). tsdf_timing_end frees the events and
 * stops recording. tsdf_raycast records a row the same way: stage 0 its
 * search-range inputs (footprints, tile offsets, fragments), stage 1 the
 * march kernel (with integration_only, only the events around the march). */
int tsdf_timing_begin(tsdf_scene *scene, int32_t max_frames,
                      int32_t integration_only);
int tsdf_timing_read(tsdf_scene *scene, float *ms, int64_t capacity,
                     int64_t *n_frames);
int tsdf_timing_end(tsdf_scene *scene);

/* Canonical readback into caller-owned DEVICE buffers that allocates no
 * memory. The paper has no counterpart; this exists for callers that cannot
 * call cudaMalloc at that point: a real-time loop that must not take the
 * allocator's locks or its implicit device synchronisation, or a host
 * framework whose caching memory pool owns the device memory (a library
 * cudaMalloc there can fail or fragment the pool).
 * Output layout and order are those of tsdf_read_blocks (keys [n][3] int16,
 * sdf [n][512] by storage, w [n][512] uint8; sdf or w may be NULL), written
 * on the scene's stream. The call reads the block count back to the host
 * (it synchronises the scene's stream first) and synchronises the stream
 * again before returning.
 * The sort scratch is a fixed array inside the library (12 bytes per block,
 * TSDF_READ_NOALLOC_MAX_BLOCKS blocks, 3 MiB) that every GPU loading the
 * library holds until the process exits. The first call on a device looks up
 * that array's device address (once per device); make that first call
 * before any stream capture. All calls share the one array, so calls whose
 * GPU work overlaps (several scenes on different streams at once) race:
 * serialise them. Returns TSDF_ERR_CAPACITY, writing nothing, when the
 * allocated block count (written to *n_written) exceeds `capacity` or
 * exceeds TSDF_READ_NOALLOC_MAX_BLOCKS; other errors as tsdf_read_blocks. */
#define TSDF_READ_NOALLOC_MAX_BLOCKS (1 << 18)
int tsdf_read_blocks_device_noalloc(tsdf_scene *scene, int16_t *keys_dev,
                                    void *sdf_dev, uint8_t *w_dev,
                                    int64_t capacity, int64_t *n_written);

/* ---- Batched step ------------------------------------------------------
 * One fusion step (the same stages as tsdf_integrate) for many independent
 * scenes at once: one launch per stage covers every scene of the batch,
 * whatever their image sizes, voxel sizes, pools and storage forms (one
 * integration launch per storage form present). The results
 * are those of calling tsdf_integrate on each scene with its frame. The paper
 * fuses one scene at a time; batching is an addition of this library. */

/* One scene's frame of a batched step (or of a tsdf_integrate_frames
 * sequence). */
struct tsdf_frame {
    tsdf_scene *scene;        /* distinct scenes on the batch's device       */
    const float *depth;       /* depth, width*height, row pitch below        */
    int64_t pitch_elems;      /* >= width, pitch_elems * height < 2^31        */
    tsdf_intrinsics intr;
    double world_to_cam[16];  /* row-major, last row (0, 0, 0, 1)           */
    int32_t depth_on_host;    /* 0: `depth` is DEVICE memory; 1: HOST memory
                                 (pinned: copies are asynchronous, and a CUDA
                                 graph can capture them), copied to the
                                 device by the call: tsdf_integrate_frames
                                 through a staging ring on a copy stream; a
                                 batch launch into the scene's staging
                                 buffer on the batch stream, before its
                                 allocation stage. The host memory must stay
                                 valid until that copy has run.             */
};

/* Schedule of a batched step (results do not depend on any field):
 *   integrate_kernel: 0 = staged (one CTA per SM; the CTA's warps take
 *     (scene, block) records from its shared-memory queue and keep the voxel
 *     data of their next two blocks in flight by bulk asynchronous copies);
 *     1 = general (the blocks' voxel data loaded into registers);
 *   integrate_threads: the staged kernel's CTA size, 256 or 512;
 *   integrate_ctas_per_sm: the general kernel's CTAs per SM (1..8, capped by
 *     what fits on an SM); must be 1 for the staged kernel;
 *   alloc_tile: pixels per allocation CTA, 0 = 16x16, 1 = 16x8, 2 = 32x8;
 *   pipelined: 0 or 1. Pipelined (needs two or more tables): launch k + 1's
 *     allocation stage runs while launch k's integration stage still runs,
 *     the latter on a second stream the batch owns; call tsdf_batch_join
 *     before the batch stream (or a scene of the batch) is used for anything
 *     else, and inside a CUDA graph capture before the capture ends.
 *     Pipelined integrations use at most 2 general CTAs per SM, or a
 *     256-thread staged CTA. */
typedef struct {
    int32_t integrate_ctas_per_sm;
    int32_t pipelined;
    int32_t integrate_kernel;
    int32_t integrate_threads;
    int32_t alloc_tile;
} tsdf_batch_config;

typedef struct tsdf_batch tsdf_batch;

/* Create a batch for up to `capacity` (1..1024) scenes per step on the
 * current device, bound to `stream` (NULL = legacy default stream), with
 * `tables` (1..4096) slot tables used round-robin: each prepare writes the
 * current table and each launch enqueues it and moves to the next one, so a
 * CUDA graph may capture up to `tables` prepare + launch pairs (a multi-frame
 * step) with each launch reading its own table at replay. Allocates the
 * tables (pinned host copies + device copies); capacity x tables must not
 * exceed 2^20 slots. */
int tsdf_batch_create(int32_t capacity, int32_t tables, void *stream,
                      tsdf_batch **out);
/* Synchronise the batch stream and free the batch (not its scenes). */
int tsdf_batch_destroy(tsdf_batch *batch);

/* Host-only: validate the n frames and write the current slot table's host
 * copy (FP64 pose handling per scene, as tsdf_integrate). Each scene is
 * re-bound to the batch stream (its later calls are ordered after the
 * batch's work) and its per-frame depth buffer grown if needed (the only
 * allocation). Waits until the table's previous eager launch has copied it;
 * during a stream capture it cannot wait and fails instead (call
 * tsdf_batch_set_cursor before capturing: it waits for every table).
 * Errors: INVALID_ARG (n outside 1..capacity, duplicate or NULL scenes, bad
 * frames, a table still being copied during a capture), OUT_OF_MEMORY, CUDA. */
int tsdf_batch_prepare(tsdf_batch *batch, const tsdf_frame *frames, int32_t n);
/* Enqueue on the batch stream: the current table's copy (host -> device) and
 * the batched stages, then advance to the next table. Neither
 * allocates nor synchronises, so it can be captured into a CUDA graph; a
 * replay reads each captured table's host copy as it is then, so rewrite a
 * table only after the previous replay has finished with it (for example,
 * after synchronising). Errors: INVALID_ARG if the current table was not
 * prepared since its last launch, CUDA. */
int tsdf_batch_launch(tsdf_batch *batch);
/* tsdf_batch_prepare + tsdf_batch_launch. */
int tsdf_batch_integrate(tsdf_batch *batch, const tsdf_frame *frames, int32_t n);
/* Index of the table the next prepare writes (0..tables-1). */
int tsdf_batch_cursor(const tsdf_batch *batch, int32_t *cursor);
/* Make `cursor` the table the next prepare writes (for example 0 before
 * capturing a multi-frame step). Outside a capture it first waits until
 * every table's last eager launch has copied it. */
int tsdf_batch_set_cursor(tsdf_batch *batch, int32_t cursor);

int tsdf_batch_set_config(tsdf_batch *batch, const tsdf_batch_config *cfg);
/* Make the batch stream wait for every pipelined launch so far (a no-op
 * when none is pending). */
int tsdf_batch_join(tsdf_batch *batch);
int tsdf_batch_get_config(const tsdf_batch *batch, tsdf_batch_config *cfg);
/* Autotuner: time `steps` launches of the current (prepared) table for
 * every candidate schedule (the staged kernel at 256 and 512 threads, the
 * general kernel at 1, 2, 3 or as many CTAs per SM as fit, each with the
 * three allocation tiles: 18 candidates; the `pipelined` field is kept),
 * keep the fastest, apply it and report it. This integrates the prepared
 * frames (1 + steps) x 18 times into the batch's scenes: tune on scratch
 * scenes, or reset the scenes afterwards. The table stays prepared and
 * current. Synchronises. */
int tsdf_batch_autotune(tsdf_batch *batch, int32_t steps, tsdf_batch_config *best,
                        float *best_ms);
/* Stage timing of batched launches, as tsdf_timing_* for a scene: three
 * boundaries per launch (before the table copy and band allocation, before
 * the integration stage, after it), ms[launch][3] relative to the first
 * boundary recorded. The autotuner's launches are
 * timed too while timing is on. */
int tsdf_batch_timing_begin(tsdf_batch *batch, int32_t max_launches,
                            int32_t integration_only);
int tsdf_batch_timing_read(tsdf_batch *batch, float *ms, int64_t capacity,
                           int64_t *n_launches);
int tsdf_batch_timing_end(tsdf_batch *batch);
/* Kernel and copy launches enqueued by the batch so far. */
int tsdf_batch_kernel_launches(const tsdf_batch *batch, int64_t *n);

/* ---- Serving ------------------------------------------------------------
 * Fusion sessions (one scene each) admitted by device memory and fused by
 * continuous batching: every step launches one batched fusion step with the
 * oldest queued frame of every admitted session that has one, so sessions
 * join and leave the batch from one step to the next, and a session's frames
 * are fused in submission order. The paper fuses one live sequence; serving
 * many is an addition of this library. Host calls from one thread. */

/* Admission controller (host only, no device work): a FIFO of sessions with
 * a byte cost. Admit takes sessions from the head while the admitted
 * sessions' bytes stay within the budget and their count within max_active;
 * a head that does not fit waits (no later session overtakes it). */
typedef struct tsdf_admission tsdf_admission;
int tsdf_admission_create(int64_t budget_bytes, int32_t max_active,
                          tsdf_admission **out);
int tsdf_admission_destroy(tsdf_admission *adm);
/* INVALID_ARG: bytes < 0 or above the budget, or id already known. */
int tsdf_admission_enqueue(tsdf_admission *adm, int64_t id, int64_t bytes);
/* Remove a queued (not admitted) id. */
int tsdf_admission_cancel(tsdf_admission *adm, int64_t id);
/* Admit up to `capacity` sessions; their ids in admission order. */
int tsdf_admission_admit(tsdf_admission *adm, int64_t *ids, int32_t capacity,
                         int32_t *n);
/* An admitted id leaves and gives its bytes back. */
int tsdf_admission_release(tsdf_admission *adm, int64_t id);
int tsdf_admission_stats(const tsdf_admission *adm, int64_t *active_bytes,
                         int32_t *n_active, int32_t *n_queued);

/* Device bytes tsdf_scene_create allocates for `desc` plus the per-frame
 * depth buffer of a width x height image (the admission cost of a session). */
int tsdf_scene_device_bytes(const tsdf_scene_desc *desc, int32_t width,
                            int32_t height, int64_t *bytes);

#define TSDF_SESSION_QUEUED 0    /* waiting for admission                    */
#define TSDF_SESSION_ACTIVE 1    /* admitted, has a scene on the device      */
#define TSDF_SESSION_FINISHED 2  /* closed and every submitted frame fused   */
#define TSDF_SESSION_FAILED 3    /* its scene could not be created (status)  */

typedef struct {
    int64_t pool_budget_bytes;  /* admitted sessions' device bytes, at most   */
    int32_t max_active;         /* admitted sessions at once, 1..1024         */
    int32_t max_queued_frames;  /* per session, submitted and not launched    */
    int32_t max_inflight_steps; /* launched steps not yet retired, 1..8       */
    int32_t reserved;
} tsdf_server_config;

typedef struct {
    int32_t admitted;         /* sessions admitted by this step             */
    int32_t launched_frames;  /* frames in this step's batched launch       */
    int32_t active_sessions;  /* admitted and not released                  */
    int32_t queued_sessions;  /* waiting for admission                      */
    int32_t inflight_steps;
    int32_t reserved;
    int64_t active_bytes;     /* admitted sessions' device bytes            */
    int64_t cached_bytes;     /* released sessions' scenes kept for reuse   */
    int64_t steps;            /* batched steps launched so far              */
    int64_t launches;         /* kernel and table-copy launches so far      */
} tsdf_server_step_info;

/* A fused frame: server-clock times (ms, steady clock) of its submission and
 * of the device completion of the step that fused it. */
typedef struct {
    int64_t ticket;
    int64_t session;
    double submit_ms;
    double done_ms;
} tsdf_frame_done;

typedef struct {
    int32_t state;            /* TSDF_SESSION_*                             */
    int32_t status;           /* creation error of a FAILED session         */
    int64_t device_bytes;
    int64_t frames_submitted;
    int64_t frames_launched;
    int64_t frames_done;
    double open_ms, admit_ms, finish_ms;  /* server clock; 0 = not yet      */
    /* FINISHED sessions: the scene's totals after the last frame (read
     * asynchronously behind it) and its device condition (TSDF_ERR_* or 0) */
    int64_t updated_voxels;
    int64_t allocated_blocks;
    int32_t device_status;
    int32_t reserved;
} tsdf_session_info;

typedef struct tsdf_server tsdf_server;

/* A server on the current device, its work on `stream`. Released sessions'
 * scenes are kept for sessions of the same buffer and image sizes (reset,
 * not reallocated); they are freed when a new scene would not fit the budget
 * otherwise, by tsdf_server_trim and by tsdf_server_destroy. */
int tsdf_server_create(const tsdf_server_config *cfg, void *stream,
                       tsdf_server **out);
int tsdf_server_destroy(tsdf_server *server);
/* Queue a session for admission; frames up to width x height. INVALID_ARG
 * if its device bytes exceed the budget. */
int tsdf_server_open(tsdf_server *server, const tsdf_scene_desc *desc,
                     int32_t width, int32_t height, int64_t *session);
/* Queue a frame (DEVICE depth, caller-owned until the frame is reported
 * done). Allowed before admission. CAPACITY when max_queued_frames frames
 * wait already; INVALID_ARG after close or for a larger image. */
int tsdf_server_submit(tsdf_server *server, int64_t session,
                       const float *depth, int64_t pitch_elems,
                       const tsdf_intrinsics *intr,
                       const double world_to_cam[16], int64_t *ticket);
/* No more frames: the session becomes FINISHED once its last frame is fused
 * and its final counters are read (asynchronously, behind the last frame):
 * at the retirement seen by a later step or poll. */
int tsdf_server_close(tsdf_server *server, int64_t session);
/* Retire completed steps, admit, and launch one step (nothing when no
 * admitted session has a queued frame). Blocks only while
 * max_inflight_steps steps are in flight. */
int tsdf_server_step(tsdf_server *server, tsdf_server_step_info *info);
/* Frames fused since the last poll (retiring completed steps first; with
 * wait_all, after every launched step completed). */
int tsdf_server_poll(tsdf_server *server, int32_t wait_all,
                     tsdf_frame_done *done, int32_t capacity, int32_t *n);
int tsdf_server_session_info(const tsdf_server *server, int64_t session,
                             tsdf_session_info *info);
/* The session's scene (ACTIVE or FINISHED), for readback with
 * tsdf_read_blocks and the other scene calls; owned by the server. */
int tsdf_server_scene(tsdf_server *server, int64_t session,
                      tsdf_scene **scene);
/* Forget a QUEUED (cancel), FINISHED or FAILED session and give its memory
 * back to admission; INVALID_ARG while it is still fusing. */
int tsdf_server_release(tsdf_server *server, int64_t session);
/* Free every cached scene. */
int tsdf_server_trim(tsdf_server *server);

/* Human-readable text of a status code (static storage). */
const char *tsdf_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* TSDF_H */
