// Serving runtime of the FUSE-Flow fusion path: several rigs resident on one GPU, frames
// from host memory, continuous batching over per-rig frame slots (declared in
// include/fuseflow.h).  Host code only; the per-frame work is the slot's recorded fuse
// call (a CUDA graph over its staging buffer) plus the copy-out kernel.
#include <algorithm>
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
};

struct Slot {
  fuseflow_ctx* ctx = nullptr;
  fuseflow_graph* graph = nullptr;      // the fuse call on d_in, recorded once
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* d_in = nullptr;                 // input staging: per camera depth | conf | rgb
  fuseflow_stats* h_stats = nullptr;    // pinned, written by the copy-out kernel
  bool busy = false;
  int64_t request = 0;
  int64_t capacity = 0;
};

struct Rig {
  int n_cams = 0;
  size_t depth_bytes = 2;
  std::vector<size_t> px;               // pixels per camera
  size_t in_bytes = 0;
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

// Enqueues request r on free slot s of rig g: host-to-device copies of the images, the
// fusion kernels, the copy-out into the caller's host arrays, then the slot's event.
int start(Rig& g, Slot& s, const Request& r) {
  HostOutDev hd{};
  int st = map_outputs(r.out, s.h_stats, &hd);
  if (st != FUSEFLOW_OK) return st;
  st = stage(g, s, r.depth.data(), r.conf.data(), r.rgb.data());
  if (st != FUSEFLOW_OK) return st;
  fuseflow_cloud cl;
  st = fuseflow_graph_launch(s.graph, &cl, s.stream);
  if (st != FUSEFLOW_OK) return st;
  if (launch_copyout(cl, hd, s.stream) != cudaSuccess ||
      cudaEventRecord(s.done, s.stream) != cudaSuccess)
    return FUSEFLOW_ERR_CUDA;
  s.busy = true;
  s.request = r.id;
  s.capacity = r.out.capacity;
  return FUSEFLOW_OK;
}

// Starts waiting frames while the cap allows: each time the oldest waiting frame (lowest
// request id, i.e. submission order across rigs) among the rigs with a free slot.
// Returns the first error of a start that failed (the frame is dropped).
int fill_slots(fuseflow_server* srv) {
  int status = FUSEFLOW_OK;
  while (srv->max_inflight == 0 || srv->inflight < srv->max_inflight) {
    Rig* best = nullptr;
    Slot* free_slot = nullptr;
    for (Rig& g : srv->rigs) {
      if (g.waiting.empty() || (best && g.waiting.front().id > best->waiting.front().id)) continue;
      for (Slot& sl : g.slots)
        if (!sl.busy) {
          best = &g;
          free_slot = &sl;
          break;
        }
    }
    if (!best) break;
    Request r = std::move(best->waiting.front());
    best->waiting.pop_front();
    const int st = start(*best, *free_slot, r);
    if (st == FUSEFLOW_OK) {
      ++srv->inflight;
    } else {
      if (status == FUSEFLOW_OK) status = st;
      --srv->pending;                      // dropped: reported through the return value
    }
  }
  return status;
}

int status_of(const fuseflow_stats& st, int64_t capacity) {
  const int s = status_of_error((unsigned)st.error);
  if (s != FUSEFLOW_OK) return s;
  return st.n_cells > capacity ? FUSEFLOW_ERR_CAPACITY : FUSEFLOW_OK;
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
  int64_t added = 0;
  int st = FUSEFLOW_OK;
  for (int k = 0; k < n_slots && st == FUSEFLOW_OK; ++k) {
    Slot s;
    st = fuseflow_create(intr, extr, n_cams, params, &s.ctx);
    if (st != FUSEFLOW_OK) break;
    const int64_t bytes = fuseflow_device_bytes(s.ctx) + (int64_t)g.in_bytes;
    if (srv->used + added + bytes > srv->budget) {
      fuseflow_destroy(s.ctx);
      st = FUSEFLOW_ERR_CAPACITY;
      break;
    }
    if (cudaMalloc(&s.d_in, g.in_bytes) != cudaSuccess) {
      s.d_in = nullptr;
      release_slot(s);
      st = FUSEFLOW_ERR_OUT_OF_MEMORY;
      break;
    }
    if (cudaHostAlloc(reinterpret_cast<void**>(&s.h_stats), sizeof(fuseflow_stats), cudaHostAllocMapped) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      release_slot(s);
      st = FUSEFLOW_ERR_CUDA;
      break;
    }
    if (n_slots > 1) {                     // overlapping slots fill the kernel boundaries
      fuseflow_tuning tu{};
      fuseflow_get_tuning(s.ctx, &tu);
      tu.programmatic = 0;
      fuseflow_set_tuning(s.ctx, &tu);
    }
    if ((st = record(g, s)) != FUSEFLOW_OK) {
      release_slot(s);
      break;
    }
    added += bytes;
    g.slots.push_back(s);
  }
  if (st != FUSEFLOW_OK) {
    for (Slot& s : g.slots) release_slot(s);
    return st;
  }
  srv->used += added;
  srv->rigs.push_back(std::move(g));
  *rig_id = (int32_t)srv->rigs.size() - 1;
  return FUSEFLOW_OK;
}

int fuseflow_server_submit(fuseflow_server* srv, int32_t rig, const void* const* depth,
                           const float* const* conf, const uint8_t* const* rgb,
                           const fuseflow_host_cloud* out, int64_t* request) {
  if (!srv || rig < 0 || rig >= (int32_t)srv->rigs.size() || !depth || !conf || !rgb || !out ||
      !request || out->capacity < 0)
    return FUSEFLOW_ERR_INVALID_ARG;
  Rig& g = srv->rigs[rig];
  Request r;
  r.id = srv->next_id++;
  for (int i = 0; i < g.n_cams; ++i) {
    if (!depth[i] || !conf[i] || !rgb[i]) return FUSEFLOW_ERR_INVALID_ARG;
    r.depth.push_back(depth[i]);
    r.conf.push_back(conf[i]);
    r.rgb.push_back(rgb[i]);
  }
  r.out = *out;
  *request = r.id;
  // the frame queues behind every frame submitted before it and starts at once if a slot
  // of its rig is free and the cap allows
  g.waiting.push_back(std::move(r));
  ++srv->pending;
  return fill_slots(srv);
}

int fuseflow_server_set_max_inflight(fuseflow_server* srv, int32_t max_inflight) {
  if (!srv || max_inflight < 0) return FUSEFLOW_ERR_INVALID_ARG;
  srv->max_inflight = max_inflight;
  return fill_slots(srv);
}

int fuseflow_server_poll(fuseflow_server* srv, fuseflow_completion* done, int32_t max_done,
                         int32_t* n_done) {
  if (!srv || !n_done || (max_done > 0 && !done)) return FUSEFLOW_ERR_INVALID_ARG;
  *n_done = 0;
  int status = FUSEFLOW_OK;
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
      c.status = q == cudaSuccess ? status_of(c.stats, s.capacity) : FUSEFLOW_ERR_CUDA;
      if (q != cudaSuccess) cudaGetLastError();
      s.busy = false;
      --srv->pending;
      --srv->inflight;
    }
  }
  // continuous batching: freed slots take the oldest waiting frames at once
  const int st = fill_slots(srv);
  return status != FUSEFLOW_OK ? status : st;
}

int fuseflow_server_autotune(fuseflow_server* srv, int32_t rig, const void* const* depth,
                             const float* const* conf, const uint8_t* const* rgb, int32_t reps,
                             fuseflow_tuning* chosen, double* frame_us) {
  if (!srv || rig < 0 || rig >= (int32_t)srv->rigs.size() || !depth || !conf || !rgb)
    return FUSEFLOW_ERR_INVALID_ARG;
  Rig& g = srv->rigs[rig];
  if (!g.waiting.empty()) return FUSEFLOW_ERR_INVALID_ARG;
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
  if (g.slots.size() > 1) tu.programmatic = 0;   // see fuseflow_server_add_rig
  for (Slot& o : g.slots) {
    fuseflow_set_tuning(o.ctx, &tu);
    if ((st = record(g, o)) != FUSEFLOW_OK) return st;
  }
  if (chosen) *chosen = tu;
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
