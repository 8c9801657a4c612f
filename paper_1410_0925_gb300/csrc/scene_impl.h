// scene_impl.h -- host-side definition of a scene, shared by the single-scene
// C ABI (scene.cu) and the batched step (batch.cu).
#pragma once

#include "tsdf_internal.cuh"

namespace tsdf {

struct SwapWork;  // swapping state (swap.cu)

// Stage timing: three CUDA events per timed launch (before stage 0, before
// stage 1, after stage 1). Records are stream operations; under stream capture they
// are external records, so that every graph replay executes them. Plain
// data, zero-initialised by its owner (scenes and batches are calloc'ed).
struct StageTimer {
  static constexpr int kEvents = 3;
  cudaEvent_t* events;
  int cap;
  int cursor;
  int integrate_only;

  int begin(int max_launches, int only_integration);
  void end();
  // the next launch's events (nullptr once `cap` launches were timed or when
  // timing is off); `capturing` tells how to record on `st`
  cudaEvent_t* next(cudaStream_t st, bool* capturing);
  cudaError_t mark(cudaEvent_t* ev, int i, cudaStream_t st, bool capturing) const;
  int read(cudaStream_t st, float* ms, long long capacity, long long* n) const;
};

}  // namespace tsdf

struct tsdf_scene {
  tsdf_scene_desc desc;
  cudaStream_t stream;
  int device;
  int sm_count;
  tsdf::SceneView sv;
  tsdf::Counters* counters;  // sv.sc and sv.fc point into it
  size_t n_entries;
  float* depth_stage;
  size_t depth_stage_elems;
  size_t depth_san_elems;      // per buffer (two buffers: frame set)
  long long launches;
  tsdf::StageTimer timer;  // tsdf_timing_*
  long long frame_seq;     // frames enqueued since creation / reset: the next
                           // frame uses set frame_seq & 1
  // pipelined sequences (tsdf_integrate_frames): integration stream and
  // events (created on first use)
  cudaStream_t aux;
  cudaEvent_t ev_alloc[2], ev_integ[2], ev_start;
  // host-depth sequences: copy stream, its events and a ring of two dense
  // depth staging buffers of seq_stage_elems floats each (created on first use)
  cudaStream_t copy;
  cudaEvent_t ev_copy[2];
  float* seq_stage;
  size_t seq_stage_elems;
  // raycast work buffers (tsdf_raycast; allocated on first use)
  tsdf::RayWork ray;
  // swapping (tsdf_scene_enable_swapping) or null
  tsdf::SwapWork* swap;
};

namespace tsdf {

// CUDA error -> status (prints the CUDA error when TSDF_DEBUG is set)
int cuda_fail(cudaError_t e);
// host view of a copy of a scene's counters
void fold_counters(const Counters& both, SceneCounters* c);
// device status bits -> TSDF_ERR_* (most severe first)
int status_code(unsigned st);
int validate_intr(const tsdf_intrinsics* in);
// release the raycast work buffers
void free_ray_work(tsdf_scene* s);
// swapping: release its buffers; clear its state (enqueued); read the number
// of blocks with a host copy (synchronises); all no-ops without swapping
void free_swap_work(tsdf_scene* s);
int swap_reset(tsdf_scene* s);
int swap_host_blocks(tsdf_scene* s, long long* n);
// grow the scene's per-frame depth work buffer to width x height
int ensure_depth_work(tsdf_scene* s, int width, int height);
// grow the scene's staging buffer for one host depth frame to `elems` floats
int ensure_depth_stage(tsdf_scene* s, size_t elems);
// per-frame constants from the FP64 pose (see scene.cu)
int make_frame_const(const tsdf_scene* s, const float* depth, long long pitch,
                     const tsdf_intrinsics* in, const double* M, FrameConst* fc);

}  // namespace tsdf

#define TSDF_CUDA(call)                                          \
  do {                                                           \
    cudaError_t err_ = (call);                                   \
    if (err_ != cudaSuccess) return ::tsdf::cuda_fail(err_);     \
  } while (0)
