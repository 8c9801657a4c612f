// batch.cu -- batched fusion step: one frame for each of many independent
// scenes (uneven image sizes, voxel sizes, pools and storage forms), one
// launch per stage for the whole batch. See include/tsdf.h.
//
// A batch owns a table of slot descriptors (each scene's device view plus the
// frame constants of this step). tsdf_batch_prepare fills a pinned host copy;
// tsdf_batch_launch copies it to the device and enqueues the three batched
// kernels, so a launch can be captured into a CUDA graph and replayed after
// preparing new frames (same scenes, same image sizes).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "scene_impl.h"

using namespace tsdf;

struct tsdf_batch {
  int capacity;
  cudaStream_t stream;
  int device;
  int sm_count;
  SlotDesc* h_slots;  // pinned
  SlotDesc* d_slots;
  int n;
  cudaEvent_t copied;  // the last eager launch's table copy
  bool copy_pending;
  tsdf_batch_config cfg;
  long long launches;
};

namespace {

bool valid_config(const tsdf_batch_config& c) {
  return (c.integrate_threads == 128 || c.integrate_threads == 256) &&
         c.visible_blocks_per_cta >= 256 && c.visible_blocks_per_cta <= (1 << 20);
}

}  // namespace

extern "C" {

int tsdf_batch_create(int32_t capacity, void* stream, tsdf_batch** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (capacity < 1 || capacity > kMaxBatch) return TSDF_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  TSDF_CUDA(cudaGetDevice(&dev));
  TSDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  tsdf_batch* b = (tsdf_batch*)calloc(1, sizeof(tsdf_batch));
  if (!b) return TSDF_ERR_OUT_OF_MEMORY;
  b->capacity = capacity;
  b->stream = (cudaStream_t)stream;
  b->device = dev;
  b->sm_count = sms;
  b->cfg.integrate_threads = 256;
  b->cfg.visible_blocks_per_cta = 4096;
  cudaError_t e = cudaMallocHost((void**)&b->h_slots, sizeof(SlotDesc) * capacity);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_slots, sizeof(SlotDesc) * capacity);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFreeHost(b->h_slots);
    cudaFree(b->d_slots);
    free(b);
    return cuda_fail(e);
  }
  *out = b;
  return TSDF_OK;
}

int tsdf_batch_destroy(tsdf_batch* b) {
  if (!b) return TSDF_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  cudaEventDestroy(b->copied);
  cudaFreeHost(b->h_slots);
  cudaFree(b->d_slots);
  free(b);
  return TSDF_OK;
}

int tsdf_batch_set_config(tsdf_batch* b, const tsdf_batch_config* c) {
  if (!b || !c || !valid_config(*c)) return TSDF_ERR_INVALID_ARG;
  b->cfg = *c;
  return TSDF_OK;
}

int tsdf_batch_get_config(const tsdf_batch* b, tsdf_batch_config* c) {
  if (!b || !c) return TSDF_ERR_INVALID_ARG;
  *c = b->cfg;
  return TSDF_OK;
}

int tsdf_batch_prepare(tsdf_batch* b, const tsdf_frame* frames, int32_t n) {
  if (!b || n < 1 || n > b->capacity || !frames) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  {
    std::vector<const tsdf_scene*> seen(n);
    for (int i = 0; i < n; ++i) seen[i] = frames[i].scene;
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return TSDF_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const tsdf_frame& f = frames[i];
    if (!f.scene || !f.depth) return TSDF_ERR_INVALID_ARG;
    if (f.scene->device != b->device) return TSDF_ERR_INVALID_ARG;
    int rc = validate_intr(&f.intr);
    if (rc) return rc;
    if (f.pitch_elems < f.intr.width ||
        f.pitch_elems * (int64_t)f.intr.height >= (int64_t)1 << 31)
      return TSDF_ERR_INVALID_ARG;
  }
  // the table's previous contents must have reached the device
  if (b->copy_pending) {
    TSDF_CUDA(cudaEventSynchronize(b->copied));
    b->copy_pending = false;
  }
  int tiles = 0, vis = 0;
  for (int i = 0; i < n; ++i) {
    const tsdf_frame& f = frames[i];
    tsdf_scene* s = f.scene;
    int rc = ensure_depth_work(s, f.intr.width, f.intr.height);
    if (rc) return rc;
    s->stream = b->stream;  // the scene's later calls order after the batch
    SlotDesc& d = b->h_slots[i];
    memset(&d, 0, sizeof(d));
    d.sv = s->sv;
    rc = make_frame_const(s, f.depth, f.pitch_elems, &f.intr, f.world_to_cam, &d.fc);
    if (rc) return rc;
    d.tile_begin = tiles;
    tiles += d.fc.tiles_x * d.fc.tiles_y;
    d.vis_begin = vis;
    d.vis_ctas = std::max(1, (s->sv.pool + b->cfg.visible_blocks_per_cta - 1) /
                                 b->cfg.visible_blocks_per_cta);
    vis += d.vis_ctas;
  }
  b->n = n;
  return TSDF_OK;
}

int tsdf_batch_launch(tsdf_batch* b) {
  if (!b || b->n < 1) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TSDF_CUDA(cudaStreamIsCapturing(b->stream, &cap));
  TSDF_CUDA(cudaMemcpyAsync(b->d_slots, b->h_slots, sizeof(SlotDesc) * b->n,
                            cudaMemcpyHostToDevice, b->stream));
  if (cap == cudaStreamCaptureStatusNone) {
    TSDF_CUDA(cudaEventRecord(b->copied, b->stream));
    b->copy_pending = true;
  }
  TSDF_CUDA(launch_alloc_batch(b->d_slots, b->h_slots, b->n, b->stream));
  TSDF_CUDA(launch_visible_batch(b->d_slots, b->h_slots, b->n, b->stream));
  TSDF_CUDA(launch_integrate_batch(b->d_slots, b->h_slots, b->n, b->sm_count,
                                   b->cfg.integrate_threads, b->stream));
  bool has[3] = {false, false, false};
  for (int i = 0; i < b->n; ++i) has[b->h_slots[i].sv.storage] = true;
  const int forms = (int)has[0] + (int)has[1] + (int)has[2];
  b->launches += 1 + 2 * forms;
  return TSDF_OK;
}

int tsdf_batch_integrate(tsdf_batch* b, const tsdf_frame* frames, int32_t n) {
  const int rc = tsdf_batch_prepare(b, frames, n);
  return rc ? rc : tsdf_batch_launch(b);
}

int tsdf_batch_kernel_launches(const tsdf_batch* b, int64_t* n) {
  if (!b || !n) return TSDF_ERR_INVALID_ARG;
  *n = b->launches;
  return TSDF_OK;
}

int tsdf_batch_autotune(tsdf_batch* b, int32_t steps, tsdf_batch_config* best, float* best_ms) {
  if (!b || b->n < 1 || steps < 1) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  const int threads[2] = {128, 256};
  const int per_cta[3] = {2048, 4096, 8192};
  cudaEvent_t e0, e1;
  TSDF_CUDA(cudaEventCreate(&e0));
  TSDF_CUDA(cudaEventCreate(&e1));
  const tsdf_batch_config saved = b->cfg;
  tsdf_batch_config winner = saved;
  float winner_ms = 1e30f;
  int rc = TSDF_OK;
  for (int ti = 0; ti < 2 && rc == TSDF_OK; ++ti) {
    for (int pi = 0; pi < 3 && rc == TSDF_OK; ++pi) {
      tsdf_batch_config c;
      c.integrate_threads = threads[ti];
      c.visible_blocks_per_cta = per_cta[pi];
      b->cfg = c;
      // the visible grid depends on the configuration: rebuild the table
      // offsets (frames unchanged)
      int vis = 0;
      for (int i = 0; i < b->n; ++i) {
        SlotDesc& d = b->h_slots[i];
        d.vis_begin = vis;
        d.vis_ctas = std::max(1, (d.sv.pool + c.visible_blocks_per_cta - 1) / c.visible_blocks_per_cta);
        vis += d.vis_ctas;
      }
      if ((rc = tsdf_batch_launch(b))) break;  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < steps && rc == TSDF_OK; ++k) rc = tsdf_batch_launch(b);
      cudaEventRecord(e1, b->stream);
      if (rc) break;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        rc = cuda_fail(e);
        break;
      }
      b->copy_pending = false;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= steps;
      if (ms < winner_ms) {
        winner_ms = ms;
        winner = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cfg = rc ? saved : winner;
  if (rc == TSDF_OK) {
    int vis = 0;
    for (int i = 0; i < b->n; ++i) {
      SlotDesc& d = b->h_slots[i];
      d.vis_begin = vis;
      d.vis_ctas = std::max(1, (d.sv.pool + b->cfg.visible_blocks_per_cta - 1) /
                                   b->cfg.visible_blocks_per_cta);
      vis += d.vis_ctas;
    }
    if (best) *best = winner;
    if (best_ms) *best_ms = winner_ms;
  }
  return rc;
}

}  // extern "C"
