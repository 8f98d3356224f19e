// Serving runtime of the FUSE-Flow fusion path: several rigs resident on one GPU, frames
// from host memory, continuous batching over per-rig frame slots held under an HBM budget
// (declared in include/fuseflow.h).  Host code only; the per-frame work is the slot's
// recorded fuse call (a CUDA graph over its staging buffer) plus the copy-out kernel.
//
// Memory: a slot is one frame's working set (a context with its tables and outputs, and a
// staging buffer for the frame's images).  A rig keeps at least one slot while it is
// resident (its camera constants and hash tables stay on the device) and may ask for more;
// slots are allocated only at the administrative calls (adding a rig, reserving, removing
// a rig, whose memory goes round-robin to the rigs below their request), never while
// frames are served, because an allocation synchronizes the whole device.  A frame that
// finds every slot of its rig busy waits; when the rig holds fewer slots than it asked for,
// the budget is why, and the frame is counted as deferred by the budget.
#include <algorithm>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "ff_internal.h"

using namespace ffl;

namespace {

struct Request {
  int64_t id = 0;
  std::vector<const void*> depth;
  std::vector<const float*> conf;
  std::vector<const uint8_t*> rgb;
  fuseflow_host_cloud out{};
  bool deferred = false;                // counted once as deferred by the budget
};

struct Slot {
  fuseflow_ctx* ctx = nullptr;
  fuseflow_graph* graph = nullptr;      // the fuse call on d_in, recorded once
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* d_in = nullptr;                 // input staging: per camera depth | conf | rgb
  fuseflow_stats* h_stats = nullptr;    // pinned, written by the copy-out kernel
  bool busy = false;
  int fail = FUSEFLOW_OK;               // status of a start that failed after queuing copies
  int64_t request = 0;
  int64_t capacity = 0;
  int64_t bytes = 0;                    // device bytes of the slot (context + staging)
};

struct Rig {
  int n_cams = 0;
  size_t depth_bytes = 2;
  std::vector<size_t> px;               // pixels per camera
  size_t in_bytes = 0;
  std::vector<fuseflow_intrinsics> intr;
  std::vector<fuseflow_extrinsics> extr;
  fuseflow_params params{};
  int max_slots = 1;
  bool removed = false;
  bool tuned = false;                   // launch geometry chosen by fuseflow_server_autotune
  fuseflow_tuning tuning{};
  int64_t slot_bytes = 0;               // bytes of one slot (known once one exists)
  std::vector<Slot> slots;
  std::deque<Request> waiting;
};

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

void release_slot(Slot& s) {
  if (s.stream) cudaStreamSynchronize(s.stream);
  if (s.graph) fuseflow_graph_destroy(s.graph);
  if (s.ctx) fuseflow_destroy(s.ctx);
  if (s.d_in) cudaFree(s.d_in);
  if (s.h_stats) cudaFreeHost(s.h_stats);
  if (s.done) cudaEventDestroy(s.done);
  if (s.stream) cudaStreamDestroy(s.stream);
  s = Slot{};
}

}  // namespace

struct fuseflow_server {
  int device = 0;
  int64_t budget = 0;
  int64_t used = 0;
  int64_t next_id = 1;
  int64_t pending = 0;
  int32_t max_inflight = 0;             // frames on the device at once, 0 = every free slot
  int32_t inflight = 0;
  std::vector<Rig> rigs;
  std::deque<fuseflow_completion> ready;   // completions reported without a slot event
  fuseflow_server_stats st{};
  int inject_n = 0;                     // testing hook: failing frame starts still to make
  int inject_status = FUSEFLOW_OK;
  bool inject_after_copies = false;
};

namespace {

// Host-mapped addresses of the caller's pinned output arrays.
int map_outputs(const fuseflow_host_cloud& o, fuseflow_stats* h_stats, HostOutDev* d) {
  auto dev = [](void* p, void** q) {
    *q = nullptr;
    if (!p) return true;
    return cudaHostGetDevicePointer(q, p, 0) == cudaSuccess;
  };
  void *a, *b, *c, *e, *f, *g, *h;
  if (!dev(o.pos, &a) || !dev(o.rgb, &b) || !dev(o.weight, &c) || !dev(o.count, &e) ||
      !dev(o.rep, &f) || !dev(o.key, &g) || !dev(h_stats, &h)) {
    cudaGetLastError();
    return FUSEFLOW_ERR_INVALID_ARG;        // not pinned host memory
  }
  d->pos = static_cast<float*>(a);
  d->rgb = static_cast<float*>(b);
  d->weight = static_cast<float*>(c);
  d->count = static_cast<uint32_t*>(e);
  d->rep = static_cast<uint32_t*>(f);
  d->key = static_cast<unsigned long long*>(g);
  d->capacity = o.capacity;
  d->stats = static_cast<fuseflow_stats*>(h);
  return FUSEFLOW_OK;
}

// Device copies of one frame's images in slot s's staging buffer.
struct Staged {
  std::vector<const void*> depth;
  std::vector<const float*> conf;
  std::vector<const uint8_t*> rgb;
};

// Per camera depth | conf | rgb in slot s's staging buffer.
Staged staging(const Rig& g, const Slot& s) {
  Staged out;
  size_t o = 0;
  for (int i = 0; i < g.n_cams; ++i) {
    const size_t px = g.px[i];
    out.depth.push_back(s.d_in + o); o += round256(px * g.depth_bytes);
    out.conf.push_back(reinterpret_cast<const float*>(s.d_in + o)); o += round256(px * 4);
    out.rgb.push_back(reinterpret_cast<const uint8_t*>(s.d_in + o)); o += round256(px * 3);
  }
  return out;
}

// Enqueues the host-to-device copies of a frame's images (host pointers per camera) into
// slot s's staging buffer on its stream.
int stage(const Rig& g, const Slot& s, const void* const* depth, const float* const* conf,
          const uint8_t* const* rgb) {
  const Staged in = staging(g, s);
  for (int i = 0; i < g.n_cams; ++i) {
    const size_t px = g.px[i];
    if (cudaMemcpyAsync(const_cast<void*>(in.depth[i]), depth[i], px * g.depth_bytes, cudaMemcpyHostToDevice,
                        s.stream) != cudaSuccess ||
        cudaMemcpyAsync(const_cast<float*>(in.conf[i]), conf[i], px * 4, cudaMemcpyHostToDevice, s.stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(const_cast<uint8_t*>(in.rgb[i]), rgb[i], px * 3, cudaMemcpyHostToDevice, s.stream) !=
            cudaSuccess)
      return FUSEFLOW_ERR_CUDA;
  }
  return FUSEFLOW_OK;
}

// (Re-)records slot s's fuse call on its staging buffer as a graph (after any change of the
// context's launch geometry, so that the replay uses the current one).
int record(const Rig& g, Slot& s) {
  if (s.graph) fuseflow_graph_destroy(s.graph);
  s.graph = nullptr;
  const Staged in = staging(g, s);
  return fuseflow_graph_create(s.ctx, in.depth.data(), in.conf.data(), in.rgb.data(), &s.graph);
}

// Launch geometry of the rig's slots: the autotuned one if any, and with several slots
// plain stream order (overlapping slots fill the kernel boundaries, and blocks waiting for
// an earlier kernel would only hold back the other slots' work).
void apply_tuning(const Rig& g, Slot& s) {
  fuseflow_tuning tu{};
  if (g.tuned) tu = g.tuning;
  else fuseflow_get_tuning(s.ctx, &tu);
  if (g.max_slots > 1) tu.programmatic = 0;
  fuseflow_set_tuning(s.ctx, &tu);
}

// A new slot for rig g within the budget: CAPACITY (nothing allocated) if it does not fit.
int make_slot(fuseflow_server* srv, Rig& g, Slot* out) {
  if (g.slot_bytes > 0 && srv->used + g.slot_bytes > srv->budget) return FUSEFLOW_ERR_CAPACITY;
  Slot s;
  int st = fuseflow_create(g.intr.data(), g.extr.data(), g.n_cams, &g.params, &s.ctx);
  if (st != FUSEFLOW_OK) return st;
  s.bytes = fuseflow_device_bytes(s.ctx) + (int64_t)g.in_bytes;
  if (srv->used + s.bytes > srv->budget) {
    fuseflow_destroy(s.ctx);
    g.slot_bytes = s.bytes;
    return FUSEFLOW_ERR_CAPACITY;
  }
  if (cudaMalloc(&s.d_in, g.in_bytes) != cudaSuccess) {
    s.d_in = nullptr;
    cudaGetLastError();
    release_slot(s);
    return FUSEFLOW_ERR_OUT_OF_MEMORY;
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&s.h_stats), sizeof(fuseflow_stats), cudaHostAllocMapped) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    release_slot(s);
    return FUSEFLOW_ERR_CUDA;
  }
  apply_tuning(g, s);
  if ((st = record(g, s)) != FUSEFLOW_OK) {
    release_slot(s);
    return st;
  }
  g.slot_bytes = s.bytes;
  srv->used += s.bytes;
  *out = s;
  return FUSEFLOW_OK;
}

// Gives slots, one per rig in turn, to the rigs that hold fewer than they asked for, while
// they fit in the budget (after a removal freed memory).
void top_up(fuseflow_server* srv) {
  for (bool grew = true; grew;) {
    grew = false;
    for (Rig& g : srv->rigs) {
      if (g.removed || (int)g.slots.size() >= g.max_slots) continue;
      Slot s;
      if (make_slot(srv, g, &s) != FUSEFLOW_OK) {
        cudaGetLastError();
        continue;
      }
      g.slots.push_back(s);
      ++srv->st.slots_grown;
      grew = true;
    }
  }
}

// A completion reported without a slot event (a frame that never reached the device, or a
// frame of a removed rig).
void report(fuseflow_server* srv, int64_t request, int32_t rig, int status, const fuseflow_stats* st) {
  fuseflow_completion c{};
  c.request = request;
  c.rig = rig;
  c.status = status;
  if (st) c.stats = *st;
  srv->ready.push_back(c);
}

// Enqueues request r on free slot s of rig g: host-to-device copies of the images, the
// fusion kernels, the copy-out into the caller's host arrays, then the slot's event.  A
// start that fails after copies were queued still records the event, so that the frame is
// reported (with the error) only once the copies from the caller's buffers are done.
// Returns the status of a failure that queued nothing (the frame is then reported at once).
int start(fuseflow_server* srv, Rig& g, Slot& s, const Request& r) {
  int injected = FUSEFLOW_OK;
  if (srv->inject_n > 0) {                  // testing hook (fuseflow_server_inject_start_failure)
    --srv->inject_n;
    if (!srv->inject_after_copies) return srv->inject_status;
    injected = srv->inject_status;
  }
  HostOutDev hd{};
  int st = map_outputs(r.out, s.h_stats, &hd);
  if (st != FUSEFLOW_OK) return st;
  std::memset(s.h_stats, 0, sizeof(fuseflow_stats));
  st = stage(g, s, r.depth.data(), r.conf.data(), r.rgb.data());
  if (st == FUSEFLOW_OK) st = injected;
  fuseflow_cloud cl;
  if (st == FUSEFLOW_OK) st = fuseflow_graph_launch(s.graph, &cl, s.stream);
  if (st == FUSEFLOW_OK && launch_copyout(cl, hd, s.stream) != cudaSuccess) st = FUSEFLOW_ERR_CUDA;
  if (cudaEventRecord(s.done, s.stream) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s.stream);       // the copies are finished (or failed) after this
    return st != FUSEFLOW_OK ? st : FUSEFLOW_ERR_CUDA;
  }
  if (st != FUSEFLOW_OK) cudaGetLastError();
  s.busy = true;
  s.fail = st;
  s.request = r.id;
  s.capacity = r.out.capacity;
  return FUSEFLOW_OK;
}

// Starts waiting frames while the cap allows: each time the oldest waiting frame (lowest
// request id, i.e. submission order across rigs) among the rigs that have a free slot.  A
// rig without one keeps its frames waiting while other rigs' frames start; when it holds
// fewer slots than it asked for, its first waiting frame is counted as deferred by the
// budget (once per frame).
void fill_slots(fuseflow_server* srv) {
  while (srv->max_inflight == 0 || srv->inflight < srv->max_inflight) {
    Rig* best = nullptr;
    int best_slot = -1;
    for (size_t gi = 0; gi < srv->rigs.size(); ++gi) {
      Rig& g = srv->rigs[gi];
      if (g.removed || g.waiting.empty()) continue;
      if (best && g.waiting.front().id > best->waiting.front().id) continue;
      int free_slot = -1;
      for (size_t k = 0; k < g.slots.size(); ++k)
        if (!g.slots[k].busy) { free_slot = (int)k; break; }
      if (free_slot < 0) {
        if ((int)g.slots.size() < g.max_slots && !g.waiting.front().deferred) {
          g.waiting.front().deferred = true;
          ++srv->st.deferred_by_budget;
        }
        continue;
      }
      best = &g;
      best_slot = free_slot;
    }
    if (!best) break;
    const int32_t gi = (int32_t)(best - srv->rigs.data());
    Request r = std::move(best->waiting.front());
    best->waiting.pop_front();
    const int st = start(srv, *best, best->slots[best_slot], r);
    if (st == FUSEFLOW_OK) {
      ++srv->inflight;
    } else {
      ++srv->st.frames_failed;
      report(srv, r.id, gi, st, nullptr);    // nothing was queued: reported at the next poll
    }
  }
}

int status_of(const fuseflow_stats& st, int64_t capacity) {
  const int s = status_of_error((unsigned)st.error);
  if (s != FUSEFLOW_OK) return s;
  return st.n_cells > capacity ? FUSEFLOW_ERR_CAPACITY : FUSEFLOW_OK;
}

bool valid_rig(const fuseflow_server* srv, int32_t rig) {
  return srv && rig >= 0 && rig < (int32_t)srv->rigs.size() && !srv->rigs[rig].removed;
}

}  // namespace

extern "C" {

int fuseflow_server_create(int64_t hbm_budget_bytes, fuseflow_server** out) {
  if (!out || hbm_budget_bytes <= 0) return FUSEFLOW_ERR_INVALID_ARG;
  *out = nullptr;
  fuseflow_server* srv = new (std::nothrow) fuseflow_server();
  if (!srv) return FUSEFLOW_ERR_OUT_OF_MEMORY;
  if (cudaGetDevice(&srv->device) != cudaSuccess) { delete srv; return FUSEFLOW_ERR_CUDA; }
  srv->budget = hbm_budget_bytes;
  *out = srv;
  return FUSEFLOW_OK;
}

int fuseflow_server_add_rig(fuseflow_server* srv, const fuseflow_intrinsics* intr,
                            const fuseflow_extrinsics* extr, int32_t n_cams,
                            const fuseflow_params* params, int32_t n_slots, int32_t* rig_id) {
  if (!srv || !intr || !extr || !params || !rig_id || n_slots < 1 || n_cams < 1)
    return FUSEFLOW_ERR_INVALID_ARG;
  Rig g;
  g.n_cams = n_cams;
  g.depth_bytes = params->depth_format == FUSEFLOW_DEPTH_F32 ? 4 : 2;
  for (int i = 0; i < n_cams; ++i) {
    if (intr[i].width <= 0 || intr[i].height <= 0) return FUSEFLOW_ERR_INVALID_ARG;
    const size_t px = (size_t)intr[i].width * intr[i].height;
    g.px.push_back(px);
    g.in_bytes += round256(px * g.depth_bytes) + round256(px * 4) + round256(px * 3);
  }
  g.intr.assign(intr, intr + n_cams);
  g.extr.assign(extr, extr + n_cams);
  g.params = *params;
  g.max_slots = n_slots;
  Slot s;
  const int st = make_slot(srv, g, &s);
  if (st != FUSEFLOW_OK) return st;
  g.slots.push_back(s);
  srv->rigs.push_back(std::move(g));
  *rig_id = (int32_t)srv->rigs.size() - 1;
  ++srv->st.slots_grown;
  return FUSEFLOW_OK;
}

int fuseflow_server_reserve(fuseflow_server* srv, int32_t rig, int32_t n_slots, int32_t* n_held) {
  if (!valid_rig(srv, rig) || n_slots < 1) return FUSEFLOW_ERR_INVALID_ARG;
  Rig& g = srv->rigs[rig];
  int st = FUSEFLOW_OK;
  while ((int)g.slots.size() < std::min(n_slots, g.max_slots)) {
    Slot s;
    if ((st = make_slot(srv, g, &s)) != FUSEFLOW_OK) break;
    g.slots.push_back(s);
    ++srv->st.slots_grown;
  }
  if (n_held) *n_held = (int32_t)g.slots.size();
  return st == FUSEFLOW_ERR_CAPACITY ? FUSEFLOW_OK : st;
}

int fuseflow_server_remove_rig(fuseflow_server* srv, int32_t rig) {
  if (!valid_rig(srv, rig)) return FUSEFLOW_ERR_INVALID_ARG;
  Rig& g = srv->rigs[rig];
  for (Slot& s : g.slots) {
    if (s.busy) {                           // finish the frame and report it normally
      const cudaError_t q = cudaEventSynchronize(s.done);
      const int st = q == cudaSuccess ? (s.fail != FUSEFLOW_OK ? s.fail : status_of(*s.h_stats, s.capacity))
                                      : FUSEFLOW_ERR_CUDA;
      if (q != cudaSuccess) cudaGetLastError();
      report(srv, s.request, rig, st, s.h_stats);
      s.busy = false;
      --srv->inflight;
      ++srv->st.frames_completed;
    }
    srv->used -= s.bytes;
    release_slot(s);
  }
  g.slots.clear();
  for (const Request& r : g.waiting) {      // never started: reported as cancelled
    report(srv, r.id, rig, FUSEFLOW_ERR_CANCELLED, nullptr);
    ++srv->st.frames_cancelled;
  }
  g.waiting.clear();
  g.removed = true;
  top_up(srv);                              // the freed memory goes to rigs below their request
  fill_slots(srv);
  return FUSEFLOW_OK;
}

int fuseflow_server_submit(fuseflow_server* srv, int32_t rig, const void* const* depth,
                           const float* const* conf, const uint8_t* const* rgb,
                           const fuseflow_host_cloud* out, int64_t* request) {
  if (!valid_rig(srv, rig) || !depth || !conf || !rgb || !out || !request || out->capacity < 0)
    return FUSEFLOW_ERR_INVALID_ARG;
  Rig& g = srv->rigs[rig];
  Request r;
  for (int i = 0; i < g.n_cams; ++i) {
    if (!depth[i] || !conf[i] || !rgb[i]) return FUSEFLOW_ERR_INVALID_ARG;
    r.depth.push_back(depth[i]);
    r.conf.push_back(conf[i]);
    r.rgb.push_back(rgb[i]);
  }
  r.id = srv->next_id++;
  r.out = *out;
  *request = r.id;
  // the frame queues behind every frame submitted before it and starts at once if a slot
  // of its rig is free (or fits in the budget) and the cap allows
  g.waiting.push_back(std::move(r));
  ++srv->pending;
  ++srv->st.frames_submitted;
  fill_slots(srv);
  return FUSEFLOW_OK;
}

int fuseflow_server_set_max_inflight(fuseflow_server* srv, int32_t max_inflight) {
  if (!srv || max_inflight < 0) return FUSEFLOW_ERR_INVALID_ARG;
  srv->max_inflight = max_inflight;
  fill_slots(srv);
  return FUSEFLOW_OK;
}

int fuseflow_server_poll(fuseflow_server* srv, fuseflow_completion* done, int32_t max_done,
                         int32_t* n_done) {
  if (!srv || !n_done || (max_done > 0 && !done)) return FUSEFLOW_ERR_INVALID_ARG;
  *n_done = 0;
  while (!srv->ready.empty() && *n_done < max_done) {
    done[(*n_done)++] = srv->ready.front();
    srv->ready.pop_front();
    --srv->pending;
  }
  for (int32_t gi = 0; gi < (int32_t)srv->rigs.size(); ++gi) {
    Rig& g = srv->rigs[gi];
    for (Slot& s : g.slots) {
      if (!s.busy || *n_done >= max_done) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      fuseflow_completion& c = done[(*n_done)++];
      c.request = s.request;
      c.rig = gi;
      c.stats = *s.h_stats;
      c.status = q != cudaSuccess ? FUSEFLOW_ERR_CUDA
               : s.fail != FUSEFLOW_OK ? s.fail : status_of(c.stats, s.capacity);
      if (q != cudaSuccess) cudaGetLastError();
      if (s.fail != FUSEFLOW_OK) ++srv->st.frames_failed;
      else ++srv->st.frames_completed;
      s.busy = false;
      s.fail = FUSEFLOW_OK;
      --srv->pending;
      --srv->inflight;
    }
  }
  // continuous batching: freed slots take the oldest waiting frames at once
  fill_slots(srv);
  return FUSEFLOW_OK;
}

int fuseflow_server_autotune(fuseflow_server* srv, int32_t rig, const void* const* depth,
                             const float* const* conf, const uint8_t* const* rgb, int32_t reps,
                             fuseflow_tuning* chosen, double* frame_us) {
  if (!valid_rig(srv, rig) || !depth || !conf || !rgb) return FUSEFLOW_ERR_INVALID_ARG;
  Rig& g = srv->rigs[rig];
  if (!g.waiting.empty() || g.slots.empty()) return FUSEFLOW_ERR_INVALID_ARG;
  for (const Slot& s : g.slots)
    if (s.busy) return FUSEFLOW_ERR_INVALID_ARG;
  for (int i = 0; i < g.n_cams; ++i)
    if (!depth[i] || !conf[i] || !rgb[i]) return FUSEFLOW_ERR_INVALID_ARG;
  Slot& s = g.slots[0];
  int st = stage(g, s, depth, conf, rgb);
  if (st != FUSEFLOW_OK) return st;
  const Staged in = staging(g, s);
  fuseflow_tuning tu{};
  st = fuseflow_autotune(s.ctx, in.depth.data(), in.conf.data(), in.rgb.data(), reps, &tu, frame_us,
                         s.stream);
  if (st != FUSEFLOW_OK) return st;
  g.tuned = true;
  g.tuning = tu;
  for (Slot& o : g.slots) {
    apply_tuning(g, o);
    if ((st = record(g, o)) != FUSEFLOW_OK) return st;
  }
  if (chosen) fuseflow_get_tuning(s.ctx, chosen);
  return FUSEFLOW_OK;
}

int fuseflow_server_get_stats(const fuseflow_server* srv, fuseflow_server_stats* out) {
  if (!srv || !out) return FUSEFLOW_ERR_INVALID_ARG;
  *out = srv->st;
  out->budget_bytes = srv->budget;
  out->used_bytes = srv->used;
  out->inflight = srv->inflight;
  out->rigs = 0;
  out->slots = 0;
  out->waiting = 0;
  for (const Rig& g : srv->rigs) {
    if (g.removed) continue;
    ++out->rigs;
    out->slots += (int32_t)g.slots.size();
    out->waiting += (int32_t)g.waiting.size();
  }
  return FUSEFLOW_OK;
}

int fuseflow_server_inject_start_failure(fuseflow_server* srv, int32_t n, int32_t status,
                                         int32_t after_copies) {
  if (!srv || n < 0 || (n > 0 && status == FUSEFLOW_OK)) return FUSEFLOW_ERR_INVALID_ARG;
  srv->inject_n = n;
  srv->inject_status = status;
  srv->inject_after_copies = after_copies != 0;
  return FUSEFLOW_OK;
}

int64_t fuseflow_server_pending(const fuseflow_server* srv) { return srv ? srv->pending : 0; }

int64_t fuseflow_server_device_bytes(const fuseflow_server* srv) { return srv ? srv->used : 0; }

void fuseflow_server_destroy(fuseflow_server* srv) {
  if (!srv) return;
  for (Rig& g : srv->rigs)
    for (Slot& s : g.slots) release_slot(s);
  delete srv;
}

}  // extern "C"
