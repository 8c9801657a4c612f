// scene.cu -- C ABI of libtsdf: scene lifetime, per-frame host preparation
// (FP64 pose handling, the only FP64 in the library) and the launch sequence
// of one fusion step. See include/tsdf.h for the contract of every call.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "scene_impl.h"

using namespace tsdf;

namespace {

constexpr int kTileCap = 1 << 16;  // 16x16 depth tiles: images up to 4096 x 4096

int next_pow2(long long v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

__global__ void reset_kernel(SceneView sv, size_t n_entries) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (size_t i = tid; i < n_entries; i += stride) {
    sv.entries[i].key = kKeyEmpty;
    sv.entries[i].ptr = kPtrUnallocated;
    sv.entries[i].next = kLinkNone;
  }
  for (size_t i = tid; i < (size_t)sv.pool; i += stride) {
    sv.key_of_ptr[i] = kKeyEmpty;
  }
  for (size_t i = tid; i <= (size_t)sv.ov_set_mask; i += stride) sv.ov_set[i] = kKeyEmpty;
  for (size_t i = tid; i < 4 * (size_t)sv.tile_cap; i += stride) sv.tile_max[i] = 0u;
  if (tid == 0) {
    SceneCounters c{};
    c.free_top = sv.pool;
    *sv.sc = c;
    FrameCounters f{};
    *sv.fc = f;
  }
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

int validate_desc(const tsdf_scene_desc* d) {
  if (!d) return TSDF_ERR_INVALID_ARG;
  if (!finite_pos(d->voxel_size) || !finite_pos(d->mu)) return TSDF_ERR_INVALID_ARG;
  if (d->max_weight < 1 || d->max_weight > 255) return TSDF_ERR_INVALID_ARG;
  if (d->hash_buckets_log2 < 1 || d->hash_buckets_log2 > 26) return TSDF_ERR_INVALID_ARG;
  if (d->entries_per_bucket < 1 || d->entries_per_bucket > 8) return TSDF_ERR_INVALID_ARG;
  if (d->excess_entries < 1 || d->excess_entries > (1 << 26)) return TSDF_ERR_INVALID_ARG;
  if (d->pool_blocks < 1 || d->pool_blocks > (1 << 24)) return TSDF_ERR_INVALID_ARG;
  if (d->storage < TSDF_STORAGE_F32 || d->storage > TSDF_STORAGE_F16) return TSDF_ERR_INVALID_ARG;
  return TSDF_OK;
}

template <typename T>
int dev_alloc(T** p, size_t count) {
  *p = nullptr;
  TSDF_CUDA(cudaMalloc((void**)p, count * sizeof(T)));
  return TSDF_OK;
}

// Element counts of a scene's device buffers (tsdf_scene_create allocates
// exactly these; tsdf_scene_device_bytes adds them up).
struct SceneSizes {
  size_t entries, pool, voxels, new_cap, ov_size, tiles;
};

SceneSizes scene_sizes(const tsdf_scene_desc& d) {
  SceneSizes z;
  z.entries = ((size_t)1 << d.hash_buckets_log2) * d.entries_per_bucket + (size_t)d.excess_entries;
  z.pool = (size_t)d.pool_blocks;
  z.voxels = z.pool * kBlockVoxels;
  z.new_cap = (size_t)next_pow2(std::max(d.pool_blocks, 1024));
  z.ov_size = (size_t)next_pow2(std::max(2LL * d.excess_entries, 1024LL));
  z.tiles = 4 * (size_t)kTileCap;  // two pyramids (frame parity) of 2 kTileCap
  return z;
}

size_t scene_bytes(const tsdf_scene_desc& d) {
  const SceneSizes z = scene_sizes(d);
  return z.entries * sizeof(HashEntry) + z.pool * sizeof(unsigned long long) +
         z.voxels * (storage_bytes(d.storage) + 1) + z.new_cap * sizeof(NewRec) +
         z.ov_size * (sizeof(OverflowRec) + sizeof(unsigned long long)) +
         z.tiles * sizeof(unsigned) + sizeof(Counters);
}

void free_scene_buffers(tsdf_scene* s) {
  for (int k = 0; k < 2; ++k) {
    if (s->ev_alloc[k]) cudaEventDestroy(s->ev_alloc[k]);
    if (s->ev_integ[k]) cudaEventDestroy(s->ev_integ[k]);
  }
  if (s->ev_start) cudaEventDestroy(s->ev_start);
  if (s->aux) cudaStreamDestroy(s->aux);
  for (int k = 0; k < 2; ++k)
    if (s->ev_copy[k]) cudaEventDestroy(s->ev_copy[k]);
  if (s->copy) cudaStreamDestroy(s->copy);
  cudaFree(s->seq_stage);
  cudaFree(s->sv.entries);
  cudaFree(s->sv.key_of_ptr);
  cudaFree(s->sv.sdf);
  cudaFree(s->sv.w);
  cudaFree(s->sv.new_list);
  cudaFree(s->sv.ov_list);
  cudaFree(s->sv.ov_set);
  cudaFree(s->sv.tile_max);
  cudaFree(s->counters);
  cudaFree(s->depth_stage);
  cudaFree(s->sv.depth_san);
  cudaFree(s->sv.rgbw);
  free_ray_work(s);
  free_swap_work(s);
}

int enqueue_reset(tsdf_scene* s) {
  reset_kernel<<<s->sm_count * 4, 256, 0, s->stream>>>(s->sv, s->n_entries);
  TSDF_CUDA(cudaGetLastError());
  // voxel colours start at 0 (blocks handed out by integration clear theirs;
  // blocks loaded by tsdf_load_blocks keep these zeros)
  if (s->sv.rgbw)
    TSDF_CUDA(cudaMemsetAsync(s->sv.rgbw, 0, (size_t)s->sv.pool * kBlockVoxels * sizeof(unsigned),
                              s->stream));
  s->launches += 1;
  return swap_reset(s);
}

// 3x3 inverse by the adjugate; returns false if singular
bool invert3(const double m[9], double out[9]) {
  const double c00 = m[4] * m[8] - m[5] * m[7];
  const double c01 = m[5] * m[6] - m[3] * m[8];
  const double c02 = m[3] * m[7] - m[4] * m[6];
  const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  if (!(std::fabs(det) > 1e-300) || !std::isfinite(det)) return false;
  const double id = 1.0 / det;
  out[0] = c00 * id;
  out[1] = (m[2] * m[7] - m[1] * m[8]) * id;
  out[2] = (m[1] * m[5] - m[2] * m[4]) * id;
  out[3] = c01 * id;
  out[4] = (m[0] * m[8] - m[2] * m[6]) * id;
  out[5] = (m[2] * m[3] - m[0] * m[5]) * id;
  out[6] = c02 * id;
  out[7] = (m[1] * m[6] - m[0] * m[7]) * id;
  out[8] = (m[0] * m[4] - m[1] * m[3]) * id;
  return true;
}

void split(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// Per-frame constants from the FP64 pose (the only FP64 arithmetic):
//   voxel v (integer) -> camera: c = (s R) v + t        (A = s R as hi + lo)
//   camera point q -> world in block units: (R^-1 q - R^-1 t) / (8 s)

int make_frame_const_impl(const tsdf_scene* s, const float* depth, long long pitch,
                     const tsdf_intrinsics* in, const double* M, FrameConst* fc) {
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(M[i])) return TSDF_ERR_INVALID_ARG;
  if (M[12] != 0.0 || M[13] != 0.0 || M[14] != 0.0 || M[15] != 1.0) return TSDF_ERR_INVALID_ARG;
  const double R[9] = {M[0], M[1], M[2], M[4], M[5], M[6], M[8], M[9], M[10]};
  const double t[3] = {M[3], M[7], M[11]};
  double Ri[9];
  if (!invert3(R, Ri)) return TSDF_ERR_INVALID_ARG;
  const double vs = (double)s->desc.voxel_size;
  const double bs = 8.0 * vs;
  for (int i = 0; i < 9; ++i) {
    split(vs * R[i], fc->A_hi[i], fc->A_lo[i]);
    fc->G[i] = (float)(Ri[i] / bs);
  }
  for (int r = 0; r < 3; ++r) {
    split(t[r], fc->t_hi[r], fc->t_lo[r]);
    const double ct = Ri[3 * r] * t[0] + Ri[3 * r + 1] * t[1] + Ri[3 * r + 2] * t[2];
    fc->g[r] = (float)(-ct / bs);
  }
  fc->fx = in->fx;
  fc->fy = in->fy;
  fc->cx = in->cx;
  fc->cy = in->cy;
  fc->inv_fx = (float)(1.0 / (double)in->fx);
  fc->inv_fy = (float)(1.0 / (double)in->fy);
  fc->mu = s->desc.mu;
  fc->inv_mu = (float)(1.0 / (double)s->desc.mu);
  fc->xmax = (float)(in->width - 2);
  fc->ymax = (float)(in->height - 2);
  fc->width = in->width;
  fc->height = in->height;
  fc->pitch = (int)pitch;
  fc->tiles_x = (in->width + 15) / 16;
  fc->tiles_y = (in->height + 15) / 16;
  fc->alloc_tile = kAllocTile16x16;
  fc->ctiles_x = (in->width + alloc_tile_w(fc->alloc_tile) - 1) / alloc_tile_w(fc->alloc_tile);
  fc->ctiles_y = (in->height + alloc_tile_h(fc->alloc_tile) - 1) / alloc_tile_h(fc->alloc_tile);
  {
    int wl = 0, hl = 0;
    const int total = pyramid_level(fc->tiles_x, fc->tiles_y, kPyramidLevels, wl, hl);
    fc->use_tiles = ((long long)fc->tiles_x * fc->tiles_y <= s->sv.tile_cap &&
                     total <= 2 * s->sv.tile_cap) ? 1 : 0;
  }
  fc->max_weight = s->desc.max_weight;
  fc->voxel_size = s->desc.voxel_size;
  fc->depth = depth;
  fc->set = (int)(s->frame_seq & 1);
  fc->rgb = nullptr;
  return TSDF_OK;
}

int validate_intr_impl(const tsdf_intrinsics* in) {
  if (!in) return TSDF_ERR_INVALID_ARG;
  if (in->width < 3 || in->height < 3 || in->width > (1 << 16) || in->height > (1 << 16))
    return TSDF_ERR_INVALID_ARG;
  if (!std::isfinite(in->fx) || !std::isfinite(in->fy) || in->fx == 0.0f || in->fy == 0.0f ||
      !std::isfinite(in->cx) || !std::isfinite(in->cy))
    return TSDF_ERR_INVALID_ARG;
  return TSDF_OK;
}

// The scene counters as the stats report them.
int read_counters(tsdf_scene* s, SceneCounters* c) {
  Counters both;
  TSDF_CUDA(cudaMemcpyAsync(&both, s->counters, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
  TSDF_CUDA(cudaStreamSynchronize(s->stream));
  fold_counters(both, c);
  return TSDF_OK;
}

// synchronise, fetch counters, return and clear the recorded device status
int sync_and_status(tsdf_scene* s, SceneCounters* c) {
  int rc = read_counters(s, c);
  if (rc) return rc;
  if (c->status) {
    TSDF_CUDA(cudaMemsetAsync(&s->sv.sc->status, 0, sizeof(unsigned), s->stream));
    TSDF_CUDA(cudaStreamSynchronize(s->stream));
  }
  return status_code(c->status);
}

unsigned long long host_pack(int x, int y, int z) {
  return (unsigned long long)(unsigned short)x | ((unsigned long long)(unsigned short)y << 16) |
         ((unsigned long long)(unsigned short)z << 32);
}

}  // namespace

namespace tsdf {

// Scene counters as the host reports them (every frame's counts are folded
// into them by the frame's integration kernel).
void fold_counters(const Counters& both, SceneCounters* c) { *c = both.sc; }

int status_code(unsigned st) {
  if (st & kStInternal) return TSDF_ERR_INTERNAL;
  if (st & kStTimeout) return TSDF_ERR_TIMEOUT;
  if (st & kStExcess) return TSDF_ERR_EXCESS_EXHAUSTED;
  if (st & kStPool) return TSDF_ERR_POOL_EXHAUSTED;
  if (st & kStKeyRange) return TSDF_ERR_KEY_RANGE;
  return TSDF_OK;
}

int cuda_fail(cudaError_t e) {
  if (getenv("TSDF_DEBUG")) fprintf(stderr, "libtsdf: CUDA error %s\n", cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TSDF_ERR_OUT_OF_MEMORY : TSDF_ERR_CUDA;
}

int validate_intr(const tsdf_intrinsics* in) { return validate_intr_impl(in); }

int make_frame_const(const tsdf_scene* s, const float* depth, long long pitch,
                     const tsdf_intrinsics* in, const double* M, FrameConst* fc) {
  return make_frame_const_impl(s, depth, pitch, in, M, fc);
}

// The allocation kernel writes a sanitised copy of the depth for the
// integration kernel, one buffer per frame set; the buffers grow with the
// largest image seen (a larger image than any before allocates, so run one
// frame of each size before capturing frames into a CUDA graph).
int ensure_depth_work(tsdf_scene* s, int width, int height) {
  const size_t need = (size_t)width * height;
  if (s->depth_san_elems < need) {
    cudaFree(s->sv.depth_san);
    s->sv.depth_san = nullptr;
    s->depth_san_elems = 0;
    s->sv.depth_san_stride = 0;
    TSDF_CUDA(cudaMalloc((void**)&s->sv.depth_san, 2 * need * sizeof(float)));
    s->depth_san_elems = need;
    s->sv.depth_san_stride = (long long)need;
  }
  return TSDF_OK;
}


// The scene's staging buffer for one host depth frame (tsdf_integrate and
// batches), grown to `elems` floats (cudaFree waits for the work that may
// still read the old one).
int ensure_depth_stage(tsdf_scene* s, size_t elems) {
  if (s->depth_stage_elems >= elems) return TSDF_OK;
  cudaFree(s->depth_stage);
  s->depth_stage = nullptr;
  s->depth_stage_elems = 0;
  TSDF_CUDA(cudaMalloc((void**)&s->depth_stage, elems * sizeof(float)));
  s->depth_stage_elems = elems;
  return TSDF_OK;
}

}  // namespace tsdf

namespace tsdf {

int StageTimer::begin(int max_launches, int only_integration) {
  if (max_launches < 1 || max_launches > (1 << 20)) return TSDF_ERR_INVALID_ARG;
  end();
  events = (cudaEvent_t*)calloc((size_t)max_launches * kEvents, sizeof(cudaEvent_t));
  if (!events) return TSDF_ERR_OUT_OF_MEMORY;
  cap = max_launches;
  for (int i = 0; i < max_launches * kEvents; ++i) {
    const cudaError_t e = cudaEventCreate(&events[i]);
    if (e != cudaSuccess) {
      end();
      return cuda_fail(e);
    }
  }
  cursor = 0;
  integrate_only = only_integration ? 1 : 0;
  return TSDF_OK;
}

void StageTimer::end() {
  if (events) {
    for (int i = 0; i < cap * kEvents; ++i)
      if (events[i]) cudaEventDestroy(events[i]);
    free(events);
  }
  events = nullptr;
  cap = 0;
  cursor = 0;
}

cudaEvent_t* StageTimer::next(cudaStream_t st, bool* capturing) {
  *capturing = false;
  if (!events || cursor >= cap) return nullptr;
  cudaStreamCaptureStatus c = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &c) != cudaSuccess) return nullptr;
  *capturing = c == cudaStreamCaptureStatusActive;
  return events + (size_t)kEvents * cursor++;
}

cudaError_t StageTimer::mark(cudaEvent_t* ev, int i, cudaStream_t st, bool capturing) const {
  if (!ev || (integrate_only && i < kEvents - 2)) return cudaSuccess;  // keep the last stage
  // Under stream capture the record must be "external" to become an event
  // node that every graph replay executes (a plain record would only order
  // the capture); outside capture it is a plain record.
  if (capturing) return cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
  return cudaEventRecord(ev[i], st);
}

int StageTimer::read(cudaStream_t st, float* ms, long long capacity, long long* n) const {
  *n = events ? cursor : 0;
  if (!events || cursor == 0) return TSDF_OK;
  if (capacity < cursor || !ms) return TSDF_ERR_CAPACITY;
  TSDF_CUDA(cudaStreamSynchronize(st));
  const int first = integrate_only ? kEvents - 2 : 0;
  const cudaEvent_t ref = events[first];
  for (int f = 0; f < cursor; ++f) {
    const cudaEvent_t* ev = events + (size_t)kEvents * f;
    for (int b = 0; b < kEvents; ++b) {
      float t = NAN;
      if (!integrate_only || b >= kEvents - 2) TSDF_CUDA(cudaEventElapsedTime(&t, ref, ev[b]));
      ms[(size_t)f * kEvents + b] = t;
    }
  }
  return TSDF_OK;
}

}  // namespace tsdf

extern "C" {

int tsdf_scene_create(const tsdf_scene_desc* desc, void* stream, tsdf_scene** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = validate_desc(desc);
  if (rc) return rc;
  int dev = 0;
  TSDF_CUDA(cudaGetDevice(&dev));
  int sms = 0;
  TSDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  tsdf_scene* s = (tsdf_scene*)calloc(1, sizeof(tsdf_scene));
  if (!s) return TSDF_ERR_OUT_OF_MEMORY;
  s->desc = *desc;
  s->stream = (cudaStream_t)stream;
  s->device = dev;
  s->sm_count = sms;
  SceneView& sv = s->sv;
  const int nb = 1 << desc->hash_buckets_log2;
  sv.bucket_mask = nb - 1;
  sv.entries_per_bucket = desc->entries_per_bucket;
  sv.n_bucket_entries = nb * desc->entries_per_bucket;
  sv.excess_cap = desc->excess_entries;
  sv.pool = desc->pool_blocks;
  sv.storage = desc->storage;
  const SceneSizes z = scene_sizes(*desc);
  sv.new_cap = (int)z.new_cap;
  sv.ov_set_mask = (int)z.ov_size - 1;
  sv.tile_cap = kTileCap;
  s->n_entries = z.entries;
  if ((rc = dev_alloc(&sv.entries, z.entries)) || (rc = dev_alloc(&sv.key_of_ptr, z.pool)) ||
      (rc = dev_alloc((unsigned char**)&sv.sdf, z.voxels * storage_bytes(desc->storage))) ||
      (rc = dev_alloc(&sv.w, z.voxels)) || (rc = dev_alloc(&sv.new_list, z.new_cap)) ||
      (rc = dev_alloc(&sv.ov_list, z.ov_size)) || (rc = dev_alloc(&sv.ov_set, z.ov_size)) ||
      (rc = dev_alloc(&sv.tile_max, z.tiles)) ||
      (rc = dev_alloc(&s->counters, 1))) {
    free_scene_buffers(s);
    free(s);
    return rc;
  }
  sv.sc = &s->counters->sc;
  sv.fc = &s->counters->fc;
  // the integration stream and events of pipelined sequences
  {
    cudaError_t e = cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&s->ev_alloc[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_integ[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      free_scene_buffers(s);
      free(s);
      return cuda_fail(e);
    }
  }
  if ((rc = enqueue_reset(s))) {
    free_scene_buffers(s);
    free(s);
    return rc;
  }
  *out = s;
  return TSDF_OK;
}

int tsdf_scene_device_bytes(const tsdf_scene_desc* desc, int32_t width, int32_t height,
                            int64_t* bytes) {
  if (!bytes) return TSDF_ERR_INVALID_ARG;
  *bytes = 0;
  const int rc = validate_desc(desc);
  if (rc) return rc;
  if (width < 0 || height < 0) return TSDF_ERR_INVALID_ARG;
  *bytes = (int64_t)scene_bytes(*desc) + 2 * (int64_t)width * height * (int64_t)sizeof(float);
  return TSDF_OK;
}

int tsdf_scene_destroy(tsdf_scene* s) {
  if (!s) return TSDF_OK;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  s->timer.end();
  free_scene_buffers(s);
  free(s);
  return TSDF_OK;
}

int tsdf_scene_reset(tsdf_scene* s) {
  if (!s) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  s->frame_seq = 0;
  return enqueue_reset(s);
}

int tsdf_scene_device(const tsdf_scene* s, int32_t* device) {
  if (!s || !device) return TSDF_ERR_INVALID_ARG;
  *device = s->device;
  return TSDF_OK;
}

int tsdf_scene_set_stream(tsdf_scene* s, void* stream) {
  if (!s) return TSDF_ERR_INVALID_ARG;
  s->stream = (cudaStream_t)stream;
  return TSDF_OK;
}

namespace {
int integrate_one(tsdf_scene* s, const float* depth, int64_t pitch_elems, int depth_on_host,
                  const uint8_t* rgb, const tsdf_intrinsics* intr, const double world_to_cam[16]) {
  if (!s || !depth || !world_to_cam) return TSDF_ERR_INVALID_ARG;
  int rc = validate_intr(intr);
  if (rc) return rc;
  if (pitch_elems < intr->width) return TSDF_ERR_INVALID_ARG;
  if (pitch_elems * (int64_t)intr->height >= (int64_t)1 << 31) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  const float* dptr = depth;
  long long pitch = pitch_elems;
  if (depth_on_host) {
    if ((rc = ensure_depth_stage(s, (size_t)intr->width * intr->height))) return rc;
    TSDF_CUDA(cudaMemcpy2DAsync(s->depth_stage, intr->width * sizeof(float), depth,
                                (size_t)pitch_elems * sizeof(float), intr->width * sizeof(float),
                                intr->height, cudaMemcpyHostToDevice, s->stream));
    dptr = s->depth_stage;
    pitch = intr->width;
  }
  if ((rc = ensure_depth_work(s, intr->width, intr->height))) return rc;
  FrameConst fc;
  rc = make_frame_const(s, dptr, pitch, intr, world_to_cam, &fc);
  if (rc) return rc;
  fc.rgb = reinterpret_cast<const uchar4*>(rgb);
  bool capturing = false;
  cudaEvent_t* ev = s->timer.next(s->stream, &capturing);
  auto mark = [&](int i) { return s->timer.mark(ev, i, s->stream, capturing); };
  // The allocation set this frame writes is clear (the scene reset, the
  // resume path and the previous frame's integration kernel leave it so);
  // this frame's allocation kernel folds and zeroes the previous frame's
  // visible and integration counts.
  TSDF_CUDA(mark(0));
  TSDF_CUDA(launch_alloc(fc, s->sv, s->stream));  // band allocation + commit
  TSDF_CUDA(mark(1));
  TSDF_CUDA(launch_integrate(fc, s->sv, s->sm_count, s->stream));  // selection + rule U
  TSDF_CUDA(mark(2));
  s->launches += 2;
  s->frame_seq += 1;
  return TSDF_OK;
}
}  // namespace

int tsdf_integrate(tsdf_scene* s, const float* depth, int64_t pitch_elems, int depth_on_host,
                   const tsdf_intrinsics* intr, const double world_to_cam[16]) {
  return integrate_one(s, depth, pitch_elems, depth_on_host, nullptr, intr, world_to_cam);
}

int tsdf_scene_enable_colour(tsdf_scene* s) {
  if (!s) return TSDF_ERR_INVALID_ARG;
  if (s->sv.rgbw) return TSDF_OK;
  if (s->swap) return TSDF_ERR_INVALID_ARG;  // the host block layout is fixed
  TSDF_CUDA(cudaSetDevice(s->device));
  const size_t bytes = (size_t)s->sv.pool * kBlockVoxels * sizeof(unsigned);
  TSDF_CUDA(cudaMalloc((void**)&s->sv.rgbw, bytes));
  const cudaError_t e = cudaMemsetAsync(s->sv.rgbw, 0, bytes, s->stream);
  if (e != cudaSuccess) {
    cudaFree(s->sv.rgbw);
    s->sv.rgbw = nullptr;
    return cuda_fail(e);
  }
  return TSDF_OK;
}

int tsdf_integrate_rgb(tsdf_scene* s, const float* depth, int64_t pitch_elems, int depth_on_host,
                       const uint8_t* rgb, const tsdf_intrinsics* intr,
                       const double world_to_cam[16]) {
  if (!s || !rgb || !s->sv.rgbw) return TSDF_ERR_INVALID_ARG;
  if ((uintptr_t)rgb & 3) return TSDF_ERR_INVALID_ARG;
  return integrate_one(s, depth, pitch_elems, depth_on_host, rgb, intr, world_to_cam);
}

int tsdf_read_colour(tsdf_scene* s, uint8_t* rgbw, int64_t capacity, int64_t* n_written) {
  if (!s || !n_written || !s->sv.rgbw) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  SceneCounters c;
  const int status = sync_and_status(s, &c);
  if (status == TSDF_ERR_CUDA) return status;
  const int n = s->sv.pool - c.free_top;
  *n_written = n;
  if (capacity < n || (n > 0 && !rgbw)) return TSDF_ERR_CAPACITY;
  if (n == 0) return status;
  const int n2 = next_pow2(n);
  const int chunk = std::min(n, 16384);
  unsigned long long* sk = nullptr;
  int* sp = nullptr;
  unsigned* buf = nullptr;
  cudaError_t e = cudaMalloc((void**)&sk, n2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sp, n2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&buf, (size_t)chunk * kBlockVoxels * sizeof(unsigned));
  if (e == cudaSuccess) e = launch_sort_allocated(s->sv, n, sk, sp, n2, s->stream);
  for (int b0 = 0; e == cudaSuccess && b0 < n; b0 += chunk) {
    const int m = std::min(chunk, n - b0);
    e = launch_gather_colour(s->sv, sp + b0, m, buf, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rgbw + (size_t)b0 * kBlockVoxels * 4, buf,
                          (size_t)m * kBlockVoxels * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  const int rc = e != cudaSuccess ? cuda_fail(e) : TSDF_OK;
  cudaStreamSynchronize(s->stream);
  cudaFree(sk);
  cudaFree(sp);
  cudaFree(buf);
  return rc ? rc : status;
}

// The copy stream, its events and the two staging buffers of host-depth
// sequences, created or grown to `elems` floats each (waits for the scene's
// stream before freeing smaller buffers).
static int ensure_seq_stage(tsdf_scene* s, size_t elems) {
  if (!s->copy) {
    TSDF_CUDA(cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k)
      TSDF_CUDA(cudaEventCreateWithFlags(&s->ev_copy[k], cudaEventDisableTiming));
  }
  if (s->seq_stage_elems >= elems) return TSDF_OK;
  TSDF_CUDA(cudaStreamSynchronize(s->stream));
  TSDF_CUDA(cudaStreamSynchronize(s->copy));
  cudaFree(s->seq_stage);
  s->seq_stage = nullptr;
  s->seq_stage_elems = 0;
  TSDF_CUDA(cudaMalloc((void**)&s->seq_stage, 2 * elems * sizeof(float)));
  s->seq_stage_elems = elems;
  return TSDF_OK;
}

// Integration CTAs per SM in a pipelined sequence: room is left on every SM
// for the next frame's allocation CTAs, which run at the same time.
constexpr int kSequenceIntegCtasPerSm = 2;

int tsdf_integrate_frames(tsdf_scene* s, const tsdf_frame* frames, int32_t n) {
  if (!s || n < 0 || (n > 0 && !frames)) return TSDF_ERR_INVALID_ARG;
  if (n == 0) return TSDF_OK;
  int max_w = 0, max_h = 0;
  bool any_host = false;
  for (int i = 0; i < n; ++i) {
    const tsdf_frame& f = frames[i];
    if ((f.scene && f.scene != s) || !f.depth) return TSDF_ERR_INVALID_ARG;
    if (f.depth_on_host != 0 && f.depth_on_host != 1) return TSDF_ERR_INVALID_ARG;
    any_host = any_host || f.depth_on_host;
    int rc = validate_intr(&f.intr);
    if (rc) return rc;
    if (f.pitch_elems < f.intr.width || f.pitch_elems * (int64_t)f.intr.height >= (int64_t)1 << 31)
      return TSDF_ERR_INVALID_ARG;
    max_w = std::max(max_w, (int)f.intr.width);
    max_h = std::max(max_h, (int)f.intr.height);
  }
  TSDF_CUDA(cudaSetDevice(s->device));
  int rc = ensure_depth_work(s, max_w, max_h);
  if (rc) return rc;
  if (any_host && (rc = ensure_seq_stage(s, (size_t)max_w * max_h))) return rc;
  // Frame t: allocation on the scene's stream after frame t - 2's
  // integration (the previous user of its set), integration on the second
  // stream after frame t's allocation and frame t - 1's integration. So
  // frame t + 1's allocation overlaps frame t's integration. A host frame's
  // copy into staging buffer t & 1 runs on the copy stream after frame t -
  // 2's allocation (the buffer's previous reader).
  TSDF_CUDA(cudaEventRecord(s->ev_start, s->stream));
  TSDF_CUDA(cudaStreamWaitEvent(s->aux, s->ev_start, 0));
  if (any_host) TSDF_CUDA(cudaStreamWaitEvent(s->copy, s->ev_start, 0));
  for (int t = 0; t < n; ++t) {
    const tsdf_frame& f = frames[t];
    const float* dptr = f.depth;
    long long pitch = f.pitch_elems;
    if (f.depth_on_host) {
      float* stage = s->seq_stage + (size_t)(t & 1) * s->seq_stage_elems;
      if (t >= 2) TSDF_CUDA(cudaStreamWaitEvent(s->copy, s->ev_alloc[t & 1], 0));
      TSDF_CUDA(cudaMemcpy2DAsync(stage, f.intr.width * sizeof(float), f.depth,
                                  (size_t)f.pitch_elems * sizeof(float),
                                  f.intr.width * sizeof(float), f.intr.height,
                                  cudaMemcpyHostToDevice, s->copy));
      TSDF_CUDA(cudaEventRecord(s->ev_copy[t & 1], s->copy));
      TSDF_CUDA(cudaStreamWaitEvent(s->stream, s->ev_copy[t & 1], 0));
      dptr = stage;
      pitch = f.intr.width;
    }
    FrameConst fc;
    rc = make_frame_const(s, dptr, pitch, &f.intr, f.world_to_cam, &fc);
    if (rc) return rc;  // (frames already enqueued stay; the streams are joined below)
    if (t >= 2) TSDF_CUDA(cudaStreamWaitEvent(s->stream, s->ev_integ[t & 1], 0));
    TSDF_CUDA(launch_alloc(fc, s->sv, s->stream));
    TSDF_CUDA(cudaEventRecord(s->ev_alloc[t & 1], s->stream));
    TSDF_CUDA(cudaStreamWaitEvent(s->aux, s->ev_alloc[t & 1], 0));
    TSDF_CUDA(launch_integrate(fc, s->sv, s->sm_count, s->aux, kSequenceIntegCtasPerSm));
    TSDF_CUDA(cudaEventRecord(s->ev_integ[t & 1], s->aux));
    s->launches += 2;
    s->frame_seq += 1;
  }
  // join: later work on the scene's stream sees every frame
  TSDF_CUDA(cudaStreamWaitEvent(s->stream, s->ev_integ[(n - 1) & 1], 0));
  return TSDF_OK;
}

int tsdf_sync(tsdf_scene* s) {
  if (!s) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  SceneCounters c;
  return sync_and_status(s, &c);
}

int tsdf_get_stats(tsdf_scene* s, tsdf_stats* out) {
  if (!s || !out) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  SceneCounters c;
  const int rc = sync_and_status(s, &c);
  if (rc == TSDF_ERR_CUDA || rc == TSDF_ERR_OUT_OF_MEMORY) return rc;
  out->frames = (int64_t)c.frames;
  out->allocated_blocks = (int64_t)(s->sv.pool - c.free_top);
  out->last_new_blocks = (int64_t)c.last_new;
  out->last_visible_blocks = (int64_t)c.last_visible;
  out->last_updated_voxels = (int64_t)c.last_updated;
  out->total_updated_voxels = (int64_t)c.total_updated;
  out->total_visible_blocks = (int64_t)c.total_visible;
  out->excess_used = std::min<int64_t>(c.excess_top, s->sv.excess_cap);
  out->kernel_launches = s->launches;
  return rc;
}

int tsdf_num_blocks(tsdf_scene* s, int64_t* n) {
  if (!s || !n) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  SceneCounters c;
  const int rc = sync_and_status(s, &c);
  *n = (int64_t)(s->sv.pool - c.free_top);
  return rc;
}

int tsdf_read_blocks(tsdf_scene* s, int16_t* keys, void* sdf, uint8_t* w, int64_t capacity,
                     int64_t* n_written) {
  if (!s || !n_written) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  SceneCounters c;
  const int status = sync_and_status(s, &c);
  if (status == TSDF_ERR_CUDA) return status;
  const int n = s->sv.pool - c.free_top;
  *n_written = n;
  if (capacity < n) return TSDF_ERR_CAPACITY;
  if (n == 0) return status;
  const int n2 = next_pow2(n);
  unsigned long long* sk = nullptr;
  int* sp = nullptr;
  short* kbuf = nullptr;
  unsigned char* sbuf = nullptr;
  unsigned char* wbuf = nullptr;
  const int chunk = std::min(n, 16384);
  const size_t sb = storage_bytes(s->desc.storage);
  int rc = TSDF_OK;
  cudaError_t e = cudaMalloc((void**)&sk, n2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sp, n2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&kbuf, (size_t)chunk * 3 * sizeof(short));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sbuf, (size_t)chunk * kBlockVoxels * sb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&wbuf, (size_t)chunk * kBlockVoxels);
  if (e == cudaSuccess) e = launch_sort_allocated(s->sv, n, sk, sp, n2, s->stream);
  for (int b0 = 0; e == cudaSuccess && b0 < n; b0 += chunk) {
    const int m = std::min(chunk, n - b0);
    e = launch_gather_blocks(s->sv, sp + b0, m, kbuf, sdf ? sbuf : nullptr, w ? wbuf : nullptr,
                             s->stream);
    if (e == cudaSuccess && keys)
      e = cudaMemcpyAsync(keys + 3 * (size_t)b0, kbuf, (size_t)m * 3 * sizeof(short),
                          cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && sdf)
      e = cudaMemcpyAsync((unsigned char*)sdf + (size_t)b0 * kBlockVoxels * sb, sbuf,
                          (size_t)m * kBlockVoxels * sb, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && w)
      e = cudaMemcpyAsync(w + (size_t)b0 * kBlockVoxels, wbuf, (size_t)m * kBlockVoxels,
                          cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  if (e != cudaSuccess) rc = cuda_fail(e);
  cudaStreamSynchronize(s->stream);
  cudaFree(sk);
  cudaFree(sp);
  cudaFree(kbuf);
  cudaFree(sbuf);
  cudaFree(wbuf);
  return rc ? rc : status;
}

int tsdf_load_blocks(tsdf_scene* s, const int16_t* keys, const void* sdf, const uint8_t* w,
                     int64_t n) {
  if (!s || n < 0 || (n > 0 && (!keys || !sdf || !w))) return TSDF_ERR_INVALID_ARG;
  if (n == 0) return TSDF_OK;
  if (n > (1 << 26)) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  std::vector<unsigned long long> packed((size_t)n);
  for (int64_t i = 0; i < n; ++i) packed[i] = host_pack(keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]);
  {
    std::vector<unsigned long long> sorted(packed);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return TSDF_ERR_INVALID_ARG;
  }
  // weights above the scene's cap cannot come out of integration (and the
  // integration kernel relies on w <= maxW)
  for (int64_t i = 0; i < n * kBlockVoxels; ++i)
    if (w[i] > s->desc.max_weight) return TSDF_ERR_INVALID_ARG;
  SceneCounters before;
  const int prior = sync_and_status(s, &before);
  if (prior == TSDF_ERR_CUDA) return prior;
  {
    // a loaded key must not shadow a host copy of the same block
    long long on_host = 0;
    const int rc = swap_host_blocks(s, &on_host);
    if (rc) return rc;
    if (on_host > 0) return TSDF_ERR_INVALID_ARG;
  }
  const size_t sb = storage_bytes(s->desc.storage);
  unsigned long long* dk = nullptr;
  unsigned char* ds = nullptr;
  unsigned char* dw = nullptr;
  cudaError_t e = cudaMalloc((void**)&dk, (size_t)n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ds, (size_t)n * kBlockVoxels * sb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw, (size_t)n * kBlockVoxels);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dk, packed.data(), (size_t)n * sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ds, sdf, (size_t)n * kBlockVoxels * sb, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dw, w, (size_t)n * kBlockVoxels, cudaMemcpyHostToDevice, s->stream);
  // the allocation stages run in the set of the next frame (clear, and
  // cleared again afterwards)
  const int set = (int)(s->frame_seq & 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(&s->sv.fc->a[set], 0, sizeof(AllocCounters), s->stream);
  if (e == cudaSuccess) e = launch_insert_keys(dk, (int)n, s->sv, set, s->stream);
  if (e == cudaSuccess) e = launch_commit(s->sv, set, s->stream);
  if (e == cudaSuccess) e = launch_assign(s->sv, set, s->sm_count, s->stream);
  if (e == cudaSuccess) e = launch_scatter_blocks(s->sv, dk, (int)n, ds, dw, s->stream);
  if (e == cudaSuccess) e = launch_finish_frame(s->sv, set, s->stream);  // clear the set
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(dk);
  cudaFree(ds);
  cudaFree(dw);
  if (e != cudaSuccess) return cuda_fail(e);
  SceneCounters c;
  const int rc = sync_and_status(s, &c);
  return rc ? rc : prior;
}

int tsdf_lookup_blocks(tsdf_scene* s, const int16_t* keys, int64_t n, int32_t* ptr_out) {
  if (!s || n < 0 || (n > 0 && (!keys || !ptr_out))) return TSDF_ERR_INVALID_ARG;
  if (n == 0) return TSDF_OK;
  if (n > (1 << 28)) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  std::vector<unsigned long long> packed((size_t)n);
  for (int64_t i = 0; i < n; ++i) packed[i] = host_pack(keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]);
  unsigned long long* dk = nullptr;
  int* dp = nullptr;
  cudaError_t e = cudaMalloc((void**)&dk, (size_t)n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dp, (size_t)n * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dk, packed.data(), (size_t)n * sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = launch_lookup(dk, (int)n, dp, s->sv, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ptr_out, dp, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(dk);
  cudaFree(dp);
  if (e != cudaSuccess) return cuda_fail(e);
  return TSDF_OK;
}

int tsdf_timing_begin(tsdf_scene* s, int32_t max_frames, int32_t integration_only) {
  if (!s) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  return s->timer.begin(max_frames, integration_only);
}

int tsdf_timing_read(tsdf_scene* s, float* ms, int64_t capacity, int64_t* n_frames) {
  if (!s || !n_frames) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  long long n = 0;
  const int rc = s->timer.read(s->stream, ms, capacity, &n);
  *n_frames = n;
  return rc;
}

int tsdf_timing_end(tsdf_scene* s) {
  if (!s) return TSDF_ERR_INVALID_ARG;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  s->timer.end();
  return TSDF_OK;
}

const char* tsdf_status_string(int status) {
  switch (status) {
    case TSDF_OK: return "ok";
    case TSDF_ERR_INVALID_ARG: return "invalid argument";
    case TSDF_ERR_OUT_OF_MEMORY: return "out of device memory";
    case TSDF_ERR_POOL_EXHAUSTED: return "voxel block pool exhausted";
    case TSDF_ERR_EXCESS_EXHAUSTED: return "hash excess list exhausted";
    case TSDF_ERR_CUDA: return "CUDA runtime error";
    case TSDF_ERR_TIMEOUT: return "bounded device loop gave up";
    case TSDF_ERR_CAPACITY: return "caller buffer too small";
    case TSDF_ERR_KEY_RANGE: return "block coordinate outside int16 range";
    case TSDF_ERR_INTERNAL: return "device consistency check failed (access skipped)";
    default: return "unknown status";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Canonical readback into caller device buffers without any allocation.
//
// tsdf_read_blocks sorts the allocated keys in cudaMalloc'ed scratch. Some
// callers cannot allocate device memory at the moment they want a readback:
// code that is being captured into a CUDA graph, a real-time loop that must
// not take the allocator's locks or its implicit synchronisation, or a host
// framework whose own memory pool owns the whole device. For them the sort
// scratch below is a fixed array in the library's device image: it exists on
// every GPU that loads the library, from load until process exit, and is
// shared by every call.

namespace {

constexpr int kNoAllocMaxBlocks = TSDF_READ_NOALLOC_MAX_BLOCKS;
constexpr int kMaxDevices = 64;

// sort keys (u64) for kNoAllocMaxBlocks entries, then their pool indices (i32)
static __device__ __align__(256) unsigned char
    g_readback_scratch[(size_t)kNoAllocMaxBlocks * (sizeof(unsigned long long) + sizeof(int))];

std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on `device` (which must be current). The
// symbol's host-side name is only a stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress and cached.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_readback_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" int tsdf_read_blocks_device_noalloc(tsdf_scene* s, int16_t* keys_dev, void* sdf_dev,
                                               uint8_t* w_dev, int64_t capacity,
                                               int64_t* n_written) {
  if (!s || !n_written) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(s->device));
  void* scratch = nullptr;
  TSDF_CUDA(scratch_address(s->device, &scratch));
  SceneCounters c;
  const int status = sync_and_status(s, &c);
  if (status == TSDF_ERR_CUDA) return status;
  const int n = s->sv.pool - c.free_top;
  *n_written = n;
  if (n > kNoAllocMaxBlocks || capacity < n) return TSDF_ERR_CAPACITY;
  if (n == 0) return status;
  const int n2 = next_pow2(n);
  unsigned long long* sk = static_cast<unsigned long long*>(scratch);
  int* sp = reinterpret_cast<int*>(static_cast<unsigned char*>(scratch) +
                                   (size_t)kNoAllocMaxBlocks * sizeof(unsigned long long));
  // every call rewrites [0, n2) of both arrays before reading them, so no
  // clearing is needed between calls
  TSDF_CUDA(launch_sort_allocated(s->sv, n, sk, sp, n2, s->stream));
  TSDF_CUDA(launch_gather_blocks(s->sv, sp, n, reinterpret_cast<short*>(keys_dev), sdf_dev, w_dev,
                                 s->stream));
  TSDF_CUDA(cudaStreamSynchronize(s->stream));
  return status;
}
