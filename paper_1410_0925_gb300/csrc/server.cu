// server.cu -- the serving loop: fusion sessions admitted by device memory,
// continuous batching of their frames over the batched step, per-frame
// completion times. Host code only; the device work is the batch's. See
// include/tsdf.h (tsdf_admission_*, tsdf_server_*).
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "scene_impl.h"

using namespace tsdf;

// ---------------------------------------------------------------------------
// admission controller: FIFO queue of sessions, each with a byte cost;
// admits from the head while the active sessions' bytes stay within the
// budget and their count within max_active (the head waits for room: no
// later session overtakes it, so none starves)

struct tsdf_admission {
  int64_t budget;
  int32_t max_active;
  int64_t active_bytes;
  std::deque<std::pair<int64_t, int64_t>> queue;  // (id, bytes)
  std::unordered_map<int64_t, int64_t> active;    // id -> bytes
  std::unordered_map<int64_t, int64_t> queued;    // id -> bytes
};

extern "C" {

int tsdf_admission_create(int64_t budget_bytes, int32_t max_active, tsdf_admission** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (budget_bytes <= 0 || max_active < 1) return TSDF_ERR_INVALID_ARG;
  tsdf_admission* a = new (std::nothrow) tsdf_admission();
  if (!a) return TSDF_ERR_OUT_OF_MEMORY;
  a->budget = budget_bytes;
  a->max_active = max_active;
  a->active_bytes = 0;
  *out = a;
  return TSDF_OK;
}

int tsdf_admission_destroy(tsdf_admission* a) {
  delete a;
  return TSDF_OK;
}

int tsdf_admission_enqueue(tsdf_admission* a, int64_t id, int64_t bytes) {
  if (!a || bytes < 0 || bytes > a->budget) return TSDF_ERR_INVALID_ARG;
  if (a->active.count(id) || a->queued.count(id)) return TSDF_ERR_INVALID_ARG;
  a->queue.emplace_back(id, bytes);
  a->queued[id] = bytes;
  return TSDF_OK;
}

int tsdf_admission_cancel(tsdf_admission* a, int64_t id) {
  if (!a || !a->queued.count(id)) return TSDF_ERR_INVALID_ARG;
  a->queued.erase(id);
  for (auto it = a->queue.begin(); it != a->queue.end(); ++it)
    if (it->first == id) {
      a->queue.erase(it);
      break;
    }
  return TSDF_OK;
}

int tsdf_admission_admit(tsdf_admission* a, int64_t* ids, int32_t capacity, int32_t* n) {
  if (!a || !n || capacity < 0 || (capacity > 0 && !ids)) return TSDF_ERR_INVALID_ARG;
  *n = 0;
  while (!a->queue.empty() && *n < capacity && (int32_t)a->active.size() < a->max_active) {
    const auto [id, bytes] = a->queue.front();
    if (a->active_bytes + bytes > a->budget) break;
    a->queue.pop_front();
    a->queued.erase(id);
    a->active[id] = bytes;
    a->active_bytes += bytes;
    ids[(*n)++] = id;
  }
  return TSDF_OK;
}

int tsdf_admission_release(tsdf_admission* a, int64_t id) {
  if (!a) return TSDF_ERR_INVALID_ARG;
  auto it = a->active.find(id);
  if (it == a->active.end()) return TSDF_ERR_INVALID_ARG;
  a->active_bytes -= it->second;
  a->active.erase(it);
  return TSDF_OK;
}

int tsdf_admission_stats(const tsdf_admission* a, int64_t* active_bytes, int32_t* n_active,
                         int32_t* n_queued) {
  if (!a) return TSDF_ERR_INVALID_ARG;
  if (active_bytes) *active_bytes = a->active_bytes;
  if (n_active) *n_active = (int32_t)a->active.size();
  if (n_queued) *n_queued = (int32_t)a->queue.size();
  return TSDF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// server

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct PendingFrame {
  int64_t ticket;
  const float* depth;
  int64_t pitch;
  tsdf_intrinsics intr;
  double pose[16];
  double submit_ms;
};

struct Session {
  int64_t id;
  int slot;            // pinned counter slot while admitted, else -1
  bool final_enqueued; // final counter copy enqueued
  int64_t updated, allocated;
  int32_t device_status;
  tsdf_scene_desc desc;
  int32_t width, height;
  int64_t bytes;
  int32_t state;  // TSDF_SESSION_*
  int32_t status;
  bool closed;
  tsdf_scene* scene;
  std::deque<PendingFrame> queue;  // submitted, not yet launched
  int64_t submitted, launched, done;
  double open_ms, admit_ms, finish_ms;
};

struct InFlight {
  cudaEvent_t done;
  std::vector<std::tuple<int64_t, int64_t, double>> frames;  // (ticket, session, submit_ms)
  std::vector<int64_t> finals;  // sessions whose final counters this step copies
};

// scenes of released sessions, reusable by sessions of the same buffer sizes
// (hash, excess list, pool, storage form and image size)
using SizeKey = std::tuple<int32_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t>;
SizeKey size_key(const tsdf_scene_desc& d, int32_t width, int32_t height) {
  return {d.hash_buckets_log2, d.entries_per_bucket, d.excess_entries, d.pool_blocks, d.storage,
          width, height};
}

}  // namespace

struct tsdf_server {
  tsdf_server_config cfg;
  cudaStream_t stream;
  int device;
  tsdf_admission* adm;
  tsdf_batch* batch;
  std::unordered_map<int64_t, std::unique_ptr<Session>> sessions;
  std::vector<int64_t> active;  // admission order
  std::multimap<SizeKey, std::pair<tsdf_scene*, int64_t>> cache;  // key -> (scene, bytes)
  int64_t cached_bytes;
  std::deque<InFlight> inflight;
  std::vector<cudaEvent_t> spare_events;
  std::vector<tsdf_frame_done> completed;  // not yet polled
  cudaEvent_t ref;
  double ref_ms;
  int64_t next_session, next_ticket;
  int64_t steps, frames_launched, resets;
  std::vector<tsdf_frame> frames;    // step scratch
  std::vector<int64_t> admit_ids;    // step scratch
  Counters* slots;                   // pinned, one per admitted session
  std::vector<int> free_slots;
};

namespace {

void destroy_cached(tsdf_server* sv) {
  for (auto& kv : sv->cache) tsdf_scene_destroy(kv.second.first);
  sv->cache.clear();
  sv->cached_bytes = 0;
}

// Device time of an event on the host clock: the reference event was
// observed complete at ref_ms.
double event_ms(const tsdf_server* sv, cudaEvent_t e) {
  float dt = 0.0f;
  if (cudaEventElapsedTime(&dt, sv->ref, e) != cudaSuccess) return now_ms();
  return sv->ref_ms + dt;
}

// Retire the oldest in-flight step (its event has completed).
void retire_front(tsdf_server* sv) {
  InFlight& f = sv->inflight.front();
  const double t = event_ms(sv, f.done);
  for (const auto& [ticket, sid, submit] : f.frames) {
    tsdf_frame_done d;
    d.ticket = ticket;
    d.session = sid;
    d.submit_ms = submit;
    d.done_ms = t;
    sv->completed.push_back(d);
    auto it = sv->sessions.find(sid);
    if (it != sv->sessions.end()) it->second->done += 1;
  }
  for (int64_t sid : f.finals) {
    auto it = sv->sessions.find(sid);
    if (it == sv->sessions.end()) continue;
    Session& s = *it->second;
    SceneCounters c;
    fold_counters(sv->slots[s.slot], &c);
    s.updated = (int64_t)c.total_updated;
    s.allocated = (int64_t)(s.scene->sv.pool - c.free_top);
    s.device_status = status_code(c.status);
    s.state = TSDF_SESSION_FINISHED;
    s.finish_ms = t;
  }
  sv->spare_events.push_back(f.done);
  sv->inflight.pop_front();
}

int retire_ready(tsdf_server* sv, bool block_oldest) {
  if (block_oldest && !sv->inflight.empty()) {
    TSDF_CUDA(cudaEventSynchronize(sv->inflight.front().done));
    retire_front(sv);
  }
  while (!sv->inflight.empty()) {
    const cudaError_t e = cudaEventQuery(sv->inflight.front().done);
    if (e == cudaErrorNotReady) break;
    if (e != cudaSuccess) return cuda_fail(e);
    retire_front(sv);
  }
  return TSDF_OK;
}

// A device scene for an admitted session: a cached scene of the same sizes
// (re-parameterised and reset on the server stream), else a new one after
// evicting cached scenes until everything held fits the budget.
int bind_scene(tsdf_server* sv, Session& s) {
  auto it = sv->cache.find(size_key(s.desc, s.width, s.height));
  if (it != sv->cache.end()) {
    tsdf_scene* sc = it->second.first;
    sv->cached_bytes -= it->second.second;
    sv->cache.erase(it);
    sc->desc = s.desc;  // same buffer sizes; voxel size, mu and cap may differ
    sc->stream = sv->stream;
    const int rc = tsdf_scene_reset(sc);
    if (rc) {
      tsdf_scene_destroy(sc);
      return rc;
    }
    s.scene = sc;
    sv->resets += 1;
    return TSDF_OK;
  }
  int64_t active_bytes = 0;
  tsdf_admission_stats(sv->adm, &active_bytes, nullptr, nullptr);
  while (!sv->cache.empty() && active_bytes + sv->cached_bytes > sv->cfg.pool_budget_bytes) {
    auto victim = sv->cache.begin();
    tsdf_scene_destroy(victim->second.first);
    sv->cached_bytes -= victim->second.second;
    sv->cache.erase(victim);
  }
  int rc = tsdf_scene_create(&s.desc, sv->stream, &s.scene);
  if (rc) return rc;
  sv->resets += 1;  // creation enqueues one initialisation kernel
  rc = ensure_depth_work(s.scene, s.width, s.height);
  if (rc) {
    tsdf_scene_destroy(s.scene);
    s.scene = nullptr;
  }
  return rc;
}

// Enqueue the final counter copies of `rec.finals` and the record's event
// behind everything launched so far, and keep the record in flight.
int push_record(tsdf_server* sv, InFlight& rec) {
  for (int64_t id : rec.finals) {
    Session& s = *sv->sessions[id];
    TSDF_CUDA(cudaMemcpyAsync(&sv->slots[s.slot], s.scene->counters, sizeof(Counters),
                              cudaMemcpyDeviceToHost, sv->stream));
    s.final_enqueued = true;
  }
  if (sv->spare_events.empty()) {
    cudaEvent_t e;
    TSDF_CUDA(cudaEventCreate(&e));
    sv->spare_events.push_back(e);
  }
  rec.done = sv->spare_events.back();
  sv->spare_events.pop_back();
  TSDF_CUDA(cudaEventRecord(rec.done, sv->stream));
  sv->inflight.push_back(std::move(rec));
  return TSDF_OK;
}

}  // namespace

extern "C" {

int tsdf_server_create(const tsdf_server_config* cfg, void* stream, tsdf_server** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->pool_budget_bytes <= 0 || cfg->max_active < 1 || cfg->max_active > kMaxBatch ||
      cfg->max_queued_frames < 1 || cfg->max_inflight_steps < 1 || cfg->max_inflight_steps > 8)
    return TSDF_ERR_INVALID_ARG;
  std::unique_ptr<tsdf_server> sv(new (std::nothrow) tsdf_server());
  if (!sv) return TSDF_ERR_OUT_OF_MEMORY;
  sv->cfg = *cfg;
  sv->stream = (cudaStream_t)stream;
  TSDF_CUDA(cudaGetDevice(&sv->device));
  int rc = tsdf_admission_create(cfg->pool_budget_bytes, cfg->max_active, &sv->adm);
  if (rc) return rc;
  // one table per step in flight plus the one being prepared
  rc = tsdf_batch_create(cfg->max_active, cfg->max_inflight_steps + 1, stream, &sv->batch);
  if (rc) {
    tsdf_admission_destroy(sv->adm);
    return rc;
  }
  cudaError_t e = cudaEventCreate(&sv->ref);
  if (e == cudaSuccess) e = cudaEventRecord(sv->ref, sv->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(sv->ref);
  if (e != cudaSuccess) {
    tsdf_batch_destroy(sv->batch);
    tsdf_admission_destroy(sv->adm);
    return cuda_fail(e);
  }
  e = cudaMallocHost((void**)&sv->slots, sizeof(Counters) * cfg->max_active);
  if (e != cudaSuccess) {
    cudaEventDestroy(sv->ref);
    tsdf_batch_destroy(sv->batch);
    tsdf_admission_destroy(sv->adm);
    return cuda_fail(e);
  }
  for (int i = cfg->max_active - 1; i >= 0; --i) sv->free_slots.push_back(i);
  sv->ref_ms = now_ms();
  sv->next_session = 1;
  sv->next_ticket = 1;
  sv->frames.resize(cfg->max_active);
  sv->admit_ids.resize(cfg->max_active);
  *out = sv.release();
  return TSDF_OK;
}

int tsdf_server_destroy(tsdf_server* sv) {
  if (!sv) return TSDF_OK;
  cudaSetDevice(sv->device);
  cudaStreamSynchronize(sv->stream);
  for (auto& kv : sv->sessions)
    if (kv.second->scene) tsdf_scene_destroy(kv.second->scene);
  destroy_cached(sv);
  for (auto& f : sv->inflight) cudaEventDestroy(f.done);
  for (auto e : sv->spare_events) cudaEventDestroy(e);
  cudaEventDestroy(sv->ref);
  cudaFreeHost(sv->slots);
  tsdf_batch_destroy(sv->batch);
  tsdf_admission_destroy(sv->adm);
  delete sv;
  return TSDF_OK;
}

int tsdf_server_open(tsdf_server* sv, const tsdf_scene_desc* desc, int32_t width, int32_t height,
                     int64_t* session) {
  if (!sv || !desc || !session || width < 3 || height < 3) return TSDF_ERR_INVALID_ARG;
  int64_t bytes = 0;
  int rc = tsdf_scene_device_bytes(desc, width, height, &bytes);
  if (rc) return rc;
  if (bytes > sv->cfg.pool_budget_bytes) return TSDF_ERR_INVALID_ARG;
  auto s = std::make_unique<Session>();
  s->id = sv->next_session++;
  s->desc = *desc;
  s->width = width;
  s->height = height;
  s->bytes = bytes;
  s->state = TSDF_SESSION_QUEUED;
  s->slot = -1;
  s->open_ms = now_ms();
  rc = tsdf_admission_enqueue(sv->adm, s->id, bytes);
  if (rc) return rc;
  *session = s->id;
  sv->sessions[s->id] = std::move(s);
  return TSDF_OK;
}

int tsdf_server_submit(tsdf_server* sv, int64_t session, const float* depth, int64_t pitch_elems,
                       const tsdf_intrinsics* intr, const double world_to_cam[16],
                       int64_t* ticket) {
  if (!sv || !depth || !intr || !world_to_cam) return TSDF_ERR_INVALID_ARG;
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return TSDF_ERR_INVALID_ARG;
  Session& s = *it->second;
  if (s.closed || s.state == TSDF_SESSION_FAILED) return TSDF_ERR_INVALID_ARG;
  int rc = validate_intr(intr);
  if (rc) return rc;
  if (intr->width > s.width || intr->height > s.height) return TSDF_ERR_INVALID_ARG;
  if (pitch_elems < intr->width || pitch_elems * (int64_t)intr->height >= (int64_t)1 << 31)
    return TSDF_ERR_INVALID_ARG;
  if ((int32_t)s.queue.size() >= sv->cfg.max_queued_frames) return TSDF_ERR_CAPACITY;
  PendingFrame f;
  f.ticket = sv->next_ticket++;
  f.depth = depth;
  f.pitch = pitch_elems;
  f.intr = *intr;
  memcpy(f.pose, world_to_cam, sizeof(f.pose));
  f.submit_ms = now_ms();
  s.queue.push_back(f);
  s.submitted += 1;
  if (ticket) *ticket = f.ticket;
  return TSDF_OK;
}

int tsdf_server_close(tsdf_server* sv, int64_t session) {
  if (!sv) return TSDF_ERR_INVALID_ARG;
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return TSDF_ERR_INVALID_ARG;
  Session& s = *it->second;
  s.closed = true;
  // every frame launched already: copy the final counters now; otherwise
  // the step that launches the last frame does (FINISHED when it retires)
  if (s.state == TSDF_SESSION_ACTIVE && !s.final_enqueued && s.queue.empty() &&
      s.launched == s.submitted) {
    TSDF_CUDA(cudaSetDevice(sv->device));
    InFlight rec;
    rec.finals.push_back(s.id);
    return push_record(sv, rec);
  }
  return TSDF_OK;
}

int tsdf_server_step(tsdf_server* sv, tsdf_server_step_info* info) {
  if (!sv) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(sv->device));
  tsdf_server_step_info si;
  memset(&si, 0, sizeof(si));
  int rc = retire_ready(sv, false);
  if (rc) return rc;
  // admit while memory and slots allow
  int32_t n_adm = 0;
  rc = tsdf_admission_admit(sv->adm, sv->admit_ids.data(), (int32_t)sv->admit_ids.size(), &n_adm);
  if (rc) return rc;
  for (int i = 0; i < n_adm; ++i) {
    Session& s = *sv->sessions[sv->admit_ids[i]];
    const int brc = bind_scene(sv, s);
    if (brc) {
      // the session cannot run: give its budget back and report it
      s.state = TSDF_SESSION_FAILED;
      s.status = brc;
      tsdf_admission_release(sv->adm, s.id);
      continue;
    }
    s.state = TSDF_SESSION_ACTIVE;
    s.admit_ms = now_ms();
    s.slot = sv->free_slots.back();  // admitted sessions <= max_active slots
    sv->free_slots.pop_back();
    sv->active.push_back(s.id);
    si.admitted += 1;
  }
  // one frame of every active session that has one queued
  int n = 0;
  InFlight rec;
  for (int64_t id : sv->active) {
    Session& s = *sv->sessions[id];
    if (s.state != TSDF_SESSION_ACTIVE || s.queue.empty()) continue;
    const PendingFrame& f = s.queue.front();
    tsdf_frame& fr = sv->frames[n++];
    fr.scene = s.scene;
    fr.depth = f.depth;
    fr.pitch_elems = f.pitch;
    fr.intr = f.intr;
    memcpy(fr.world_to_cam, f.pose, sizeof(fr.world_to_cam));
    rec.frames.emplace_back(f.ticket, s.id, f.submit_ms);
  }
  // closed sessions whose every frame is launched: copy their counters
  // behind their last frame
  for (int64_t id : sv->active) {
    Session& s = *sv->sessions[id];
    if (s.state != TSDF_SESSION_ACTIVE || !s.closed || s.final_enqueued) continue;
    const bool last_now = s.queue.size() == 1 && s.launched + 1 == s.submitted;
    const bool all_launched = s.queue.empty() && s.launched == s.submitted;
    if (last_now || all_launched) rec.finals.push_back(id);
  }
  if (n > 0 || !rec.finals.empty()) {
    // bounded number of steps in flight (their tables stay untouched)
    while ((int)sv->inflight.size() >= sv->cfg.max_inflight_steps)
      if ((rc = retire_ready(sv, true))) return rc;
    if (n > 0) {
      rc = tsdf_batch_prepare(sv->batch, sv->frames.data(), n);
      if (rc) return rc;
      rc = tsdf_batch_launch(sv->batch);
      if (rc) return rc;
    }
    for (int64_t id : sv->active) {
      Session& s = *sv->sessions[id];
      if (s.state != TSDF_SESSION_ACTIVE || s.queue.empty()) continue;
      s.queue.pop_front();
      s.launched += 1;
    }
    if ((rc = push_record(sv, rec))) return rc;
    if (n > 0) {
      sv->steps += 1;
      sv->frames_launched += n;
    }
  }
  si.launched_frames = n;
  tsdf_admission_stats(sv->adm, &si.active_bytes, &si.active_sessions, &si.queued_sessions);
  si.cached_bytes = sv->cached_bytes;
  int64_t batch_launches = 0;
  tsdf_batch_kernel_launches(sv->batch, &batch_launches);
  si.launches = batch_launches + sv->resets;
  si.steps = sv->steps;
  si.inflight_steps = (int32_t)sv->inflight.size();
  if (info) *info = si;
  return TSDF_OK;
}

int tsdf_server_poll(tsdf_server* sv, int32_t wait_all, tsdf_frame_done* done, int32_t capacity,
                     int32_t* n) {
  if (!sv || !n || capacity < 0 || (capacity > 0 && !done)) return TSDF_ERR_INVALID_ARG;
  *n = 0;
  TSDF_CUDA(cudaSetDevice(sv->device));
  int rc = TSDF_OK;
  if (wait_all) {
    while (!sv->inflight.empty() && rc == TSDF_OK) rc = retire_ready(sv, true);
  } else {
    rc = retire_ready(sv, false);
  }
  if (rc) return rc;
  const int32_t m = (int32_t)std::min<size_t>(sv->completed.size(), (size_t)capacity);
  if (m > 0) {
    memcpy(done, sv->completed.data(), sizeof(tsdf_frame_done) * m);
    sv->completed.erase(sv->completed.begin(), sv->completed.begin() + m);
  }
  *n = m;
  return TSDF_OK;
}

int tsdf_server_session_info(const tsdf_server* sv, int64_t session, tsdf_session_info* info) {
  if (!sv || !info) return TSDF_ERR_INVALID_ARG;
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return TSDF_ERR_INVALID_ARG;
  const Session& s = *it->second;
  info->state = s.state;
  info->status = s.status;
  info->device_bytes = s.bytes;
  info->frames_submitted = s.submitted;
  info->frames_launched = s.launched;
  info->frames_done = s.done;
  info->open_ms = s.open_ms;
  info->admit_ms = s.admit_ms;
  info->finish_ms = s.finish_ms;
  info->updated_voxels = s.updated;
  info->allocated_blocks = s.allocated;
  info->device_status = s.device_status;
  info->reserved = 0;
  return TSDF_OK;
}

int tsdf_server_scene(tsdf_server* sv, int64_t session, tsdf_scene** scene) {
  if (!sv || !scene) return TSDF_ERR_INVALID_ARG;
  *scene = nullptr;
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end() || !it->second->scene) return TSDF_ERR_INVALID_ARG;
  *scene = it->second->scene;
  return TSDF_OK;
}

int tsdf_server_release(tsdf_server* sv, int64_t session) {
  if (!sv) return TSDF_ERR_INVALID_ARG;
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return TSDF_ERR_INVALID_ARG;
  Session& s = *it->second;
  if (s.state == TSDF_SESSION_QUEUED) {
    tsdf_admission_cancel(sv->adm, s.id);
  } else if (s.state == TSDF_SESSION_FINISHED) {
    tsdf_admission_release(sv->adm, s.id);
    sv->free_slots.push_back(s.slot);
    s.slot = -1;
    for (size_t i = 0; i < sv->active.size(); ++i)
      if (sv->active[i] == s.id) {
        sv->active.erase(sv->active.begin() + i);
        break;
      }
    // keep the scene for a later session of the same sizes (its memory
    // stays within the budget: bind_scene evicts cached scenes first)
    sv->cache.emplace(size_key(s.desc, s.width, s.height), std::make_pair(s.scene, s.bytes));
    sv->cached_bytes += s.bytes;
    s.scene = nullptr;
  } else if (s.state != TSDF_SESSION_FAILED) {
    return TSDF_ERR_INVALID_ARG;  // still fusing: close it and wait for FINISHED
  }
  sv->sessions.erase(it);
  return TSDF_OK;
}

int tsdf_server_trim(tsdf_server* sv) {
  if (!sv) return TSDF_ERR_INVALID_ARG;
  cudaSetDevice(sv->device);
  cudaStreamSynchronize(sv->stream);
  destroy_cached(sv);
  return TSDF_OK;
}

}  // extern "C"
