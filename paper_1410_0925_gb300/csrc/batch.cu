// batch.cu -- batched fusion step: one frame for each of many independent
// scenes (uneven image sizes, voxel sizes, pools and storage forms), one
// launch per stage for the whole batch. See include/tsdf.h.
//
// A batch owns a ring of slot tables; a table holds each scene's device view
// plus the frame constants of one step. tsdf_batch_prepare fills the current
// table's pinned host copy; tsdf_batch_launch copies it to the device,
// enqueues the batched kernels and moves to the next table. A graph
// capturing K prepare + launch pairs therefore reads K distinct tables at
// every replay.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "scene_impl.h"

using namespace tsdf;

namespace {

// A host depth frame of a slot: copied into its scene's staging buffer on
// the batch stream by the launch, before the allocation stage.
struct HostDepth {
  const float* src;
  long long pitch;  // elements
  int width, height;
  float* dst;       // the scene's depth_stage (dense, pitch = width)
};

struct Table {
  SlotDesc* h;          // pinned host copy, `capacity` slots
  SlotDesc* d;          // device copy
  HostDepth* host;      // `capacity` entries, the first n_host used
  int n_host;
  int n;                // scenes prepared (0 = not prepared since last launch)
  cudaEvent_t copied;   // the table's last eager copy
  bool copy_pending;
};

}  // namespace

struct tsdf_batch {
  int capacity;
  int n_tables;
  cudaStream_t stream;
  int device;
  int sm_count;
  Table* tables;
  int cursor;
  tsdf_batch_config cfg;
  long long launches;
  StageTimer timer;  // tsdf_batch_timing_*
  // pipelined launches: integration stream, events, launches since the last
  // join
  cudaStream_t aux;
  cudaEvent_t ev_alloc[2], ev_integ[2], ev_start;
  long long pipe_k;
};

namespace {

constexpr long long kMaxSlots = 1LL << 20;

bool valid_config(const tsdf_batch_config& c) {
  if (c.pipelined != 0 && c.pipelined != 1) return false;
  if (c.alloc_tile < kAllocTile16x16 || c.alloc_tile > kAllocTile32x8) return false;
  if (c.integrate_kernel == kBatchKernelGeneral)
    return c.integrate_ctas_per_sm >= 1 && c.integrate_ctas_per_sm <= 8;
  return c.integrate_kernel == kBatchKernelStaged && c.integrate_ctas_per_sm == 1 &&
         (c.integrate_threads == 256 || c.integrate_threads == 512);
}

// The slots' allocation tiling for a tile shape: each scene's tile grid and
// its first CTA in the batch's allocation grid.
void set_alloc_tiles(Table& t, int n, int shape) {
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    FrameConst& fc = t.h[i].fc;
    fc.alloc_tile = shape;
    fc.ctiles_x = (fc.width + alloc_tile_w(shape) - 1) / alloc_tile_w(shape);
    fc.ctiles_y = (fc.height + alloc_tile_h(shape) - 1) / alloc_tile_h(shape);
    t.h[i].tile_begin = tiles;
    tiles += fc.ctiles_x * fc.ctiles_y;
  }
}

// Integration CTAs per SM of a pipelined launch: room is left for the next
// launch's allocation CTAs, which run at the same time.
constexpr int kPipelinedIntegCtasPerSm = 2;

void free_tables(tsdf_batch* b) {
  for (int k = 0; k < 2; ++k) {
    if (b->ev_alloc[k]) cudaEventDestroy(b->ev_alloc[k]);
    if (b->ev_integ[k]) cudaEventDestroy(b->ev_integ[k]);
  }
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->aux) cudaStreamDestroy(b->aux);
  b->aux = nullptr;
  if (!b->tables) return;
  for (int i = 0; i < b->n_tables; ++i) {
    Table& t = b->tables[i];
    if (t.copied) cudaEventDestroy(t.copied);
    free(t.host);
    if (t.h) cudaFreeHost(t.h);
    if (t.d) cudaFree(t.d);
  }
  free(b->tables);
  b->tables = nullptr;
}

// Enqueue table t: copy, then the two stages (timed when the batch's stage
// timer is on). Pipelined: the allocation of launch k waits for the
// integration of launch k - 2 (the previous user of its frames' sets) and
// the integration runs on the batch's second stream after the allocation,
// so launch k + 1's allocation overlaps launch k's integration.
int launch_table(tsdf_batch* b, Table& t, bool capturing, bool pipelined) {
  cudaStream_t integ = pipelined ? b->aux : b->stream;
  bool timer_capturing = false;
  cudaEvent_t* ev = b->timer.next(b->stream, &timer_capturing);
  TSDF_CUDA(b->timer.mark(ev, 0, b->stream, timer_capturing));
  const int k = (int)(b->pipe_k & 1);
  if (pipelined) {
    if (b->pipe_k == 0) {
      TSDF_CUDA(cudaEventRecord(b->ev_start, b->stream));
      TSDF_CUDA(cudaStreamWaitEvent(b->aux, b->ev_start, 0));
    }
    if (b->pipe_k >= 2) TSDF_CUDA(cudaStreamWaitEvent(b->stream, b->ev_integ[k], 0));
  }
  set_alloc_tiles(t, t.n, b->cfg.alloc_tile);
  TSDF_CUDA(cudaMemcpyAsync(t.d, t.h, sizeof(SlotDesc) * t.n, cudaMemcpyHostToDevice, b->stream));
  for (int i = 0; i < t.n_host; ++i) {
    const HostDepth& c = t.host[i];
    TSDF_CUDA(cudaMemcpy2DAsync(c.dst, c.width * sizeof(float), c.src, c.pitch * sizeof(float),
                                c.width * sizeof(float), c.height, cudaMemcpyHostToDevice,
                                b->stream));
  }
  if (!capturing) {
    TSDF_CUDA(cudaEventRecord(t.copied, b->stream));
    t.copy_pending = true;
  }
  TSDF_CUDA(launch_alloc_batch(t.d, t.h, t.n, b->stream));
  if (pipelined) {
    TSDF_CUDA(cudaEventRecord(b->ev_alloc[k], b->stream));
    TSDF_CUDA(cudaStreamWaitEvent(b->aux, b->ev_alloc[k], 0));
  }
  TSDF_CUDA(b->timer.mark(ev, 1, integ, timer_capturing));
  BatchIntegLaunch how;
  how.kernel = b->cfg.integrate_kernel;
  how.threads = pipelined ? 256 : b->cfg.integrate_threads;
  how.ctas_per_sm = pipelined ? std::min(b->cfg.integrate_ctas_per_sm, kPipelinedIntegCtasPerSm)
                              : b->cfg.integrate_ctas_per_sm;
  TSDF_CUDA(launch_integrate_batch(t.d, t.h, t.n, b->sm_count, how, integ));
  TSDF_CUDA(b->timer.mark(ev, 2, integ, timer_capturing));
  if (pipelined) {
    TSDF_CUDA(cudaEventRecord(b->ev_integ[k], b->aux));
    b->pipe_k += 1;
  }
  bool has[3] = {false, false, false};
  for (int i = 0; i < t.n; ++i) has[t.h[i].sv.storage] = true;
  const int forms = (int)has[0] + (int)has[1] + (int)has[2];
  b->launches += 2 + forms + t.n_host;  // table and depth copies, allocation, one
                                        // integration per form
  return TSDF_OK;
}

}  // namespace

extern "C" {

int tsdf_batch_create(int32_t capacity, int32_t tables, void* stream, tsdf_batch** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (capacity < 1 || capacity > kMaxBatch || tables < 1 || tables > 4096 ||
      (long long)capacity * tables > kMaxSlots)
    return TSDF_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  TSDF_CUDA(cudaGetDevice(&dev));
  TSDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  tsdf_batch* b = (tsdf_batch*)calloc(1, sizeof(tsdf_batch));
  if (!b) return TSDF_ERR_OUT_OF_MEMORY;
  b->capacity = capacity;
  b->n_tables = tables;
  b->stream = (cudaStream_t)stream;
  b->device = dev;
  b->sm_count = sms;
  b->cfg.integrate_kernel = kBatchKernelStaged;
  b->cfg.integrate_threads = 512;
  b->cfg.integrate_ctas_per_sm = 1;
  b->cfg.alloc_tile = kAllocTile16x16;
  b->cfg.pipelined = 0;
  b->tables = (Table*)calloc(tables, sizeof(Table));
  if (!b->tables) {
    free(b);
    return TSDF_ERR_OUT_OF_MEMORY;
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < tables && e == cudaSuccess; ++i) {
    Table& t = b->tables[i];
    t.host = (HostDepth*)calloc(capacity, sizeof(HostDepth));
    if (!t.host) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMallocHost((void**)&t.h, sizeof(SlotDesc) * capacity);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t.d, sizeof(SlotDesc) * capacity);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.copied, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&b->ev_alloc[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_integ[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_tables(b);
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
  if (b->aux) cudaStreamSynchronize(b->aux);
  b->timer.end();
  free_tables(b);
  free(b);
  return TSDF_OK;
}

int tsdf_batch_set_config(tsdf_batch* b, const tsdf_batch_config* c) {
  if (!b || !c || !valid_config(*c)) return TSDF_ERR_INVALID_ARG;
  // a pipelined launch's table is read by its integration while the next
  // launch copies its own: at least two tables
  if (c->pipelined && b->n_tables < 2) return TSDF_ERR_INVALID_ARG;
  b->cfg = *c;
  return TSDF_OK;
}

int tsdf_batch_join(tsdf_batch* b) {
  if (!b) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  if (b->pipe_k > 0) {
    TSDF_CUDA(cudaStreamWaitEvent(b->stream, b->ev_integ[(b->pipe_k - 1) & 1], 0));
    b->pipe_k = 0;
  }
  return TSDF_OK;
}

int tsdf_batch_get_config(const tsdf_batch* b, tsdf_batch_config* c) {
  if (!b || !c) return TSDF_ERR_INVALID_ARG;
  *c = b->cfg;
  return TSDF_OK;
}

int tsdf_batch_cursor(const tsdf_batch* b, int32_t* cursor) {
  if (!b || !cursor) return TSDF_ERR_INVALID_ARG;
  *cursor = b->cursor;
  return TSDF_OK;
}

int tsdf_batch_set_cursor(tsdf_batch* b, int32_t cursor) {
  if (!b || cursor < 0 || cursor >= b->n_tables) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TSDF_CUDA(cudaStreamIsCapturing(b->stream, &cap));
  if (cap == cudaStreamCaptureStatusNone) {
    // every table may be rewritten from here on, also inside a capture
    for (int i = 0; i < b->n_tables; ++i) {
      Table& t = b->tables[i];
      if (t.copy_pending) {
        TSDF_CUDA(cudaEventSynchronize(t.copied));
        t.copy_pending = false;
      }
    }
  }
  b->cursor = cursor;
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
    if (!f.scene || !f.depth || (f.depth_on_host != 0 && f.depth_on_host != 1))
      return TSDF_ERR_INVALID_ARG;
    if (f.scene->device != b->device) return TSDF_ERR_INVALID_ARG;
    if (f.scene->sv.rgbw) return TSDF_ERR_INVALID_ARG;  // colour scenes fuse one by one
    if (f.scene->swap) return TSDF_ERR_INVALID_ARG;    // so do swapping scenes
    int rc = validate_intr(&f.intr);
    if (rc) return rc;
    if (f.pitch_elems < f.intr.width ||
        f.pitch_elems * (int64_t)f.intr.height >= (int64_t)1 << 31)
      return TSDF_ERR_INVALID_ARG;
  }
  Table& t = b->tables[b->cursor];
  // the table's previous contents must have reached the device; a wait is
  // not allowed while the stream is being captured
  if (t.copy_pending) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TSDF_CUDA(cudaStreamIsCapturing(b->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) return TSDF_ERR_INVALID_ARG;
    TSDF_CUDA(cudaEventSynchronize(t.copied));
    t.copy_pending = false;
  }
  t.n = 0;
  t.n_host = 0;
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    const tsdf_frame& f = frames[i];
    tsdf_scene* s = f.scene;
    int rc = ensure_depth_work(s, f.intr.width, f.intr.height);
    if (rc) return rc;
    const float* dptr = f.depth;
    long long pitch = f.pitch_elems;
    if (f.depth_on_host) {
      // the launch copies the frame into the scene's staging buffer
      if ((rc = ensure_depth_stage(s, (size_t)f.intr.width * f.intr.height))) return rc;
      HostDepth& c = t.host[t.n_host++];
      c.src = f.depth;
      c.pitch = f.pitch_elems;
      c.width = f.intr.width;
      c.height = f.intr.height;
      c.dst = s->depth_stage;
      dptr = s->depth_stage;
      pitch = f.intr.width;
    }
    s->stream = b->stream;  // the scene's later calls order after the batch
    SlotDesc& d = t.h[i];
    memset(&d, 0, sizeof(d));
    d.sv = s->sv;
    rc = make_frame_const(s, dptr, pitch, &f.intr, f.world_to_cam, &d.fc);
    if (rc) return rc;
    s->frame_seq += 1;  // the prepared frame is the scene's next one
    d.tile_begin = tiles;
    tiles += d.fc.ctiles_x * d.fc.ctiles_y;
  }
  t.n = n;
  return TSDF_OK;
}

int tsdf_batch_launch(tsdf_batch* b) {
  if (!b) return TSDF_ERR_INVALID_ARG;
  Table& t = b->tables[b->cursor];
  if (t.n < 1) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TSDF_CUDA(cudaStreamIsCapturing(b->stream, &cap));
  const int rc = launch_table(b, t, cap != cudaStreamCaptureStatusNone, b->cfg.pipelined != 0);
  if (rc) return rc;
  t.n = -t.n;  // launched: keeps its size for a replay, must be prepared again
  b->cursor = (b->cursor + 1) % b->n_tables;
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

int tsdf_batch_timing_begin(tsdf_batch* b, int32_t max_launches, int32_t integration_only) {
  if (!b) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  return b->timer.begin(max_launches, integration_only);
}

int tsdf_batch_timing_read(tsdf_batch* b, float* ms, int64_t capacity, int64_t* n_launches) {
  if (!b || !n_launches) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  long long n = 0;
  const int rc = b->timer.read(b->stream, ms, capacity, &n);
  *n_launches = n;
  return rc;
}

int tsdf_batch_timing_end(tsdf_batch* b) {
  if (!b) return TSDF_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  if (b->aux) cudaStreamSynchronize(b->aux);
  b->timer.end();
  return TSDF_OK;
}

int tsdf_batch_autotune(tsdf_batch* b, int32_t steps, tsdf_batch_config* best, float* best_ms) {
  if (!b || steps < 1) return TSDF_ERR_INVALID_ARG;
  Table& t = b->tables[b->cursor];
  if (t.n < 1) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(b->device));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TSDF_CUDA(cudaStreamIsCapturing(b->stream, &cap));
  if (cap != cudaStreamCaptureStatusNone) return TSDF_ERR_INVALID_ARG;
  cudaEvent_t e0, e1;
  TSDF_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce);
  }
  // the candidates re-launch the same frames (same sets): never pipelined
  if (int jrc = tsdf_batch_join(b)) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return jrc;
  }
  // candidates: the staged kernel at 512 and 256 threads, the general one
  // at 1, 2, 3 and as many CTAs per SM as fit (8), each with every
  // allocation tile
  std::vector<tsdf_batch_config> cands;
  for (int tile = kAllocTile16x16; tile <= kAllocTile32x8; ++tile) {
    for (int nt : {512, 256}) {
      tsdf_batch_config c = {};
      c.integrate_kernel = kBatchKernelStaged;
      c.integrate_threads = nt;
      c.integrate_ctas_per_sm = 1;
      c.alloc_tile = tile;
      cands.push_back(c);
    }
    for (int ctas : {1, 2, 3, 8}) {
      tsdf_batch_config c = {};
      c.integrate_kernel = kBatchKernelGeneral;
      c.integrate_threads = 256;
      c.integrate_ctas_per_sm = ctas;
      c.alloc_tile = tile;
      cands.push_back(c);
    }
  }
  const tsdf_batch_config saved = b->cfg;
  tsdf_batch_config winner = saved;
  float winner_ms = 1e30f;
  int rc = TSDF_OK;
  for (size_t ci = 0; ci < cands.size() && rc == TSDF_OK; ++ci) {
    tsdf_batch_config c = cands[ci];
    c.pipelined = saved.pipelined;
    b->cfg = c;
    if ((rc = launch_table(b, t, false, false))) break;  // warm-up
    cudaEventRecord(e0, b->stream);
    for (int k = 0; k < steps && rc == TSDF_OK; ++k) rc = launch_table(b, t, false, false);
    cudaEventRecord(e1, b->stream);
    if (rc) break;
    ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce);
      break;
    }
    t.copy_pending = false;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= steps;
    if (ms < winner_ms) {
      winner_ms = ms;
      winner = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cfg = rc ? saved : winner;
  if (rc == TSDF_OK) {
    if (best) *best = winner;
    if (best_ms) *best_ms = winner_ms;
  }
  return rc;
}

}  // extern "C"
