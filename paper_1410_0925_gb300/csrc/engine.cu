// engine.cu -- the processing pipeline of one camera (Section 2.1: tracking,
// allocation and integration, swapping, raycast), as one object: every frame is
// tracked against the model rendered from the previous pose, fused at the
// tracked pose, and the model is rendered from that pose for the next frame.
// Host code over the library's own calls; one synchronisation per frame
// (the tracked pose is read back for the host).
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "scene_impl.h"

using namespace tsdf;

namespace {
constexpr int kMaxLevels = 4;
}

struct tsdf_engine {
  tsdf_engine_config cfg;
  cudaStream_t stream;
  int device;
  tsdf_scene* scene;
  tsdf_icp* icp;
  tsdf_intrinsics intr[kMaxLevels];   // per hierarchy level (0 = full resolution)
  float* depth_lvl[kMaxLevels];       // levels 1.. (level 0 is the caller's depth)
  float* points[kMaxLevels];          // reference maps per level
  float* normals[kMaxLevels];
  double* pose_dev;                   // 16 doubles
  double* sums_dev;                   // 29 doubles
  double* pose_host;                  // pinned, 16 doubles
  double pose[16];                    // the last tracked pose (world -> camera)
  long long frames;
};

namespace {

void engine_free(tsdf_engine* e) {
  if (!e) return;
  for (int l = 0; l < kMaxLevels; ++l) {
    cudaFree(e->depth_lvl[l]);
    cudaFree(e->points[l]);
    cudaFree(e->normals[l]);
  }
  cudaFree(e->pose_dev);
  cudaFree(e->sums_dev);
  cudaFreeHost(e->pose_host);
  tsdf_icp_destroy(e->icp);
  tsdf_scene_destroy(e->scene);
  free(e);
}

bool config_ok(const tsdf_engine_config* c) {
  if (!c || c->levels < 1 || c->levels > kMaxLevels) return false;
  if (!(c->max_dist > 0.0f) || !std::isfinite(c->max_dist)) return false;
  if (!(c->z_near > 0.0f) || !std::isfinite(c->z_near)) return false;
  for (int l = 0; l < c->levels; ++l)
    if (c->iterations[l] < 0 || c->iterations[l] > 100) return false;
  if (c->swap_blocks < 0 || c->swap_blocks > c->scene.pool_blocks) return false;
  if (!(c->swap_margin_px >= 0.0f) || !std::isfinite(c->swap_margin_px)) return false;
  if (validate_intr(&c->intr)) return false;
  // every level keeps at least 3 x 3 pixels
  return (c->intr.width >> (c->levels - 1)) >= 3 && (c->intr.height >> (c->levels - 1)) >= 3;
}

}  // namespace

int tsdf_engine_create(const tsdf_engine_config* cfg, const double initial_world_to_cam[16],
                       void* stream, tsdf_engine** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!config_ok(cfg) || !initial_world_to_cam) return TSDF_ERR_INVALID_ARG;
  const double* M = initial_world_to_cam;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(M[i])) return TSDF_ERR_INVALID_ARG;
  if (M[12] != 0.0 || M[13] != 0.0 || M[14] != 0.0 || M[15] != 1.0) return TSDF_ERR_INVALID_ARG;
  tsdf_engine* e = (tsdf_engine*)calloc(1, sizeof(tsdf_engine));
  if (!e) return TSDF_ERR_OUT_OF_MEMORY;
  e->cfg = *cfg;
  e->stream = (cudaStream_t)stream;
  memcpy(e->pose, M, sizeof(e->pose));
  int rc = tsdf_scene_create(&cfg->scene, stream, &e->scene);
  if (!rc && cfg->colour) rc = tsdf_scene_enable_colour(e->scene);
  if (!rc && cfg->swap_blocks > 0) rc = tsdf_scene_enable_swapping(e->scene, cfg->swap_blocks);
  if (!rc) rc = tsdf_icp_create(stream, &e->icp);
  if (rc) {
    engine_free(e);
    return rc;
  }
  cudaError_t err = cudaGetDevice(&e->device);
  for (int l = 0; l < cfg->levels && err == cudaSuccess; ++l) {
    tsdf_intrinsics in;
    if (tsdf_icp_level_intrinsics(&cfg->intr, l, &in)) {
      engine_free(e);
      return TSDF_ERR_INVALID_ARG;
    }
    if (l > 0)
      err = cudaMalloc((void**)&e->depth_lvl[l], (size_t)in.width * in.height * sizeof(float));
    e->intr[l] = in;
    const size_t px = (size_t)in.width * in.height * 4 * sizeof(float);
    if (err == cudaSuccess) err = cudaMalloc((void**)&e->points[l], px);
    if (err == cudaSuccess) err = cudaMalloc((void**)&e->normals[l], px);
  }
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->pose_dev, 16 * sizeof(double));
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->sums_dev, 32 * sizeof(double));
  if (err == cudaSuccess) err = cudaMallocHost((void**)&e->pose_host, 16 * sizeof(double));
  if (err != cudaSuccess) {
    engine_free(e);
    return cuda_fail(err);
  }
  *out = e;
  return TSDF_OK;
}

int tsdf_engine_destroy(tsdf_engine* e) {
  if (!e) return TSDF_OK;
  cudaSetDevice(e->device);
  cudaStreamSynchronize(e->stream);
  engine_free(e);
  return TSDF_OK;
}

int tsdf_engine_process(tsdf_engine* e, const float* depth, int64_t pitch_elems,
                        const uint8_t* rgb, double world_to_cam_out[16]) {
  if (!e || !depth || !world_to_cam_out || pitch_elems < e->cfg.intr.width)
    return TSDF_ERR_INVALID_ARG;
  if (rgb && !e->cfg.colour) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(e->device));
  int rc = TSDF_OK;
  if (e->frames > 0) {
    // tracking: the depth hierarchy, the model rendered from the previous
    // pose at every level, then coarse-to-fine Gauss-Newton on the device
    const float* lvl_depth[kMaxLevels];
    int64_t lvl_pitch[kMaxLevels];
    lvl_depth[0] = depth;
    lvl_pitch[0] = pitch_elems;
    for (int l = 1; l < e->cfg.levels; ++l) {
      rc = tsdf_icp_downsample(e->icp, lvl_depth[l - 1], lvl_pitch[l - 1], e->intr[l - 1].width,
                               e->intr[l - 1].height, e->depth_lvl[l]);
      if (rc) return rc;
      lvl_depth[l] = e->depth_lvl[l];
      lvl_pitch[l] = e->intr[l].width;
    }
    for (int l = 0; l < e->cfg.levels; ++l) {
      if (e->cfg.iterations[l] == 0) continue;
      if ((rc = tsdf_raycast(e->scene, &e->intr[l], e->pose, e->cfg.z_near, e->points[l], nullptr)))
        return rc;
      if ((rc = tsdf_icp_normals(e->icp, e->points[l], e->normals[l], e->intr[l].width,
                                 e->intr[l].height)))
        return rc;
    }
    memcpy(e->pose_host, e->pose, 16 * sizeof(double));
    TSDF_CUDA(cudaMemcpyAsync(e->pose_dev, e->pose_host, 16 * sizeof(double),
                              cudaMemcpyHostToDevice, e->stream));
    for (int l = e->cfg.levels - 1; l >= 0; --l) {
      if (e->cfg.iterations[l] == 0) continue;
      if ((rc = tsdf_icp_track(e->icp, lvl_depth[l], lvl_pitch[l], &e->intr[l], e->pose_dev,
                               e->pose, e->points[l], e->normals[l], e->cfg.max_dist,
                               e->cfg.iterations[l], e->sums_dev)))
        return rc;
    }
    TSDF_CUDA(cudaMemcpyAsync(e->pose_host, e->pose_dev, 16 * sizeof(double),
                              cudaMemcpyDeviceToHost, e->stream));
    TSDF_CUDA(cudaStreamSynchronize(e->stream));
    bool ok = true;
    for (int i = 0; i < 16; ++i) ok = ok && std::isfinite(e->pose_host[i]);
    if (ok) memcpy(e->pose, e->pose_host, sizeof(e->pose));  // else keep the last pose
  }
  // fusion at the tracked pose, with what the view sees brought in first
  // and what it does not moved out after (swapping)
  const bool swapping = e->cfg.swap_blocks > 0;
  const double margin = e->cfg.swap_margin_px;
  if (swapping && (rc = tsdf_swap_in(e->scene, &e->cfg.intr, e->pose, margin, 0.0))) return rc;
  rc = rgb ? tsdf_integrate_rgb(e->scene, depth, pitch_elems, 0, rgb, &e->cfg.intr, e->pose)
           : tsdf_integrate(e->scene, depth, pitch_elems, 0, &e->cfg.intr, e->pose);
  if (rc) return rc;
  if (swapping && (rc = tsdf_swap_out(e->scene, &e->cfg.intr, e->pose, margin, 0.0))) return rc;
  e->frames += 1;
  memcpy(world_to_cam_out, e->pose, sizeof(e->pose));
  return TSDF_OK;
}

int tsdf_engine_reset(tsdf_engine* e, const double initial_world_to_cam[16]) {
  if (!e || !initial_world_to_cam) return TSDF_ERR_INVALID_ARG;
  const double* M = initial_world_to_cam;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(M[i])) return TSDF_ERR_INVALID_ARG;
  if (M[12] != 0.0 || M[13] != 0.0 || M[14] != 0.0 || M[15] != 1.0) return TSDF_ERR_INVALID_ARG;
  const int rc = tsdf_scene_reset(e->scene);
  if (rc) return rc;
  memcpy(e->pose, M, sizeof(e->pose));
  e->frames = 0;
  return TSDF_OK;
}

int tsdf_engine_scene(tsdf_engine* e, tsdf_scene** out) {
  if (!e || !out) return TSDF_ERR_INVALID_ARG;
  *out = e->scene;
  return TSDF_OK;
}

int tsdf_engine_kernel_launches(tsdf_engine* e, int64_t* n) {
  if (!e || !n) return TSDF_ERR_INVALID_ARG;
  int64_t tracker = 0;
  const int rc = tsdf_icp_kernel_launches(e->icp, &tracker);
  if (rc) return rc;
  *n = e->scene->launches + tracker;
  return TSDF_OK;
}

int tsdf_engine_tracker_status(tsdf_engine* e, int32_t* status) {
  if (!e || !status) return TSDF_ERR_INVALID_ARG;
  return tsdf_icp_status(e->icp, status);
}
