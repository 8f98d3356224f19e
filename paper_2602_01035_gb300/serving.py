"""Serving driver over the C ABI's server (``fuseflow_server_*``) and the plain path.

A seeded Poisson arrival trace (one stream of frames per rig) is replayed in wall-clock
time.  The served path submits each frame to the server as it arrives (continuous
batching over per-rig slots, frames from pinned host memory); the plain path fuses one
frame at a time in arrival order through ``fuseflow_fuse_frame_host``.  Latency is the
time from a frame's arrival to the host seeing its result.  All fusion work runs in
``libfuseflow.so``; this module only marshals buffers and keeps time.
"""
from __future__ import annotations

import ctypes as C
import gc
import time
from collections import deque
from contextlib import contextmanager

import numpy as np

from . import fuseflow as F


def poisson_trace(rates_fps, duration_s: float, seed: int):
    """Sorted (arrival time s, rig index) events: independent Poisson streams."""
    rng = np.random.default_rng(seed)
    ev = []
    for r, lam in enumerate(rates_fps):
        t = rng.exponential(1.0 / lam)
        while t < duration_s:
            ev.append((t, r))
            t += rng.exponential(1.0 / lam)
    ev.sort()
    return ev


def pinned_frame(frame):
    """Pinned host copies of a frame's images (torch tensors) and their pointers."""
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    d = [pin(x) for x in frame.depth]
    c = [pin(x) for x in frame.conf]
    r = [pin(x) for x in frame.rgb]
    return {"keep": (d, c, r), "depth": [t.data_ptr() for t in d],
            "conf": [t.data_ptr() for t in c], "rgb": [t.data_ptr() for t in r],
            "bytes": sum(t.numel() * t.element_size() for t in d + c + r)}


class HostCloud:
    """Pinned host output arrays of one frame (the layout of fuseflow_cloud)."""

    def __init__(self, capacity: int):
        import torch
        self.capacity = capacity
        self.pos = torch.empty((capacity, 3), dtype=torch.float32).pin_memory()
        self.rgb = torch.empty((capacity, 3), dtype=torch.float32).pin_memory()
        self.weight = torch.empty(capacity, dtype=torch.float32).pin_memory()
        self.count = torch.empty(capacity, dtype=torch.int32).pin_memory()
        self.rep = torch.empty(capacity, dtype=torch.int32).pin_memory()
        self.key = torch.empty(capacity, dtype=torch.int64).pin_memory()
        self.c = F.fuseflow_host_cloud(self.pos.data_ptr(), self.rgb.data_ptr(),
                                       self.weight.data_ptr(), self.count.data_ptr(),
                                       self.rep.data_ptr(), self.key.data_ptr(), capacity)

    def cells(self, n: int) -> dict:
        return {"pos": self.pos[:n].numpy().copy(), "rgb": self.rgb[:n].numpy().copy(),
                "weight": self.weight[:n].numpy().copy(),
                "count": self.count[:n].numpy().view(np.uint32).copy(),
                "rep": self.rep[:n].numpy().view(np.uint32).copy(),
                "key": self.key[:n].numpy().view(np.uint64).copy()}


class Server:
    """Several rigs resident on the current GPU under an HBM budget."""

    def __init__(self, hbm_budget_bytes: int):
        self.srv = F.fuseflow_server_create(hbm_budget_bytes)
        self.rigs = []
        self._done = (F.fuseflow_completion * 256)()

    def add_rig(self, rig, n_slots: int, **params) -> int:
        fmt = F.FUSEFLOW_DEPTH_F32 if rig.depth_format == "f32" else F.FUSEFLOW_DEPTH_U16
        p = F.fuseflow_default_params(depth_format=fmt, depth_scale=float(rig.depth_scale))
        for k, v in params.items():
            setattr(p, k, v)
        intr, extr = F.rig_arrays(rig)
        status, rid = F.fuseflow_server_add_rig(self.srv, intr, extr, len(rig.cameras), p, n_slots)
        if status != F.FUSEFLOW_OK:
            raise F.FuseFlowError(status, "fuseflow_server_add_rig")
        cap = p.max_cells if p.max_cells > 0 else max(65536, rig.n_pixels // 8)
        self.rigs.append({"rig": rig, "slots": n_slots, "capacity": cap, "params": p})
        return rid

    def submit(self, rid: int, frame: dict, out: HostCloud) -> int:
        return F.fuseflow_server_submit(self.srv, rid, frame["depth"], frame["conf"],
                                        frame["rgb"], out.c)

    def autotune(self, rid: int, frame: dict, reps: int = 9):
        """Launch geometry of an idle rig tuned on one pinned frame: (tuning, us before, after)."""
        return F.fuseflow_server_autotune(self.srv, rid, frame["depth"], frame["conf"],
                                          frame["rgb"], reps)

    def poll(self):
        n = F.fuseflow_server_poll(self.srv, self._done, len(self._done))
        return [(self._done[i].request, self._done[i].rig, self._done[i].status,
                 self._done[i].stats.as_dict()) for i in range(n)]

    def reserve(self, rid: int, n_slots: int) -> int:
        """Allocates up to n_slots slots of the rig now (as the budget allows); returns the
        number it holds."""
        return F.fuseflow_server_reserve(self.srv, rid, n_slots)

    def remove_rig(self, rid: int) -> None:
        F.fuseflow_server_remove_rig(self.srv, rid)

    def stats(self) -> dict:
        return F.fuseflow_server_get_stats(self.srv)

    def set_max_inflight(self, n: int) -> None:
        """At most n frames on the device at once (0: every free slot)."""
        F.fuseflow_server_set_max_inflight(self.srv, n)

    def pending(self) -> int:
        return F.fuseflow_server_pending(self.srv)

    def device_bytes(self) -> int:
        return F.fuseflow_server_device_bytes(self.srv)

    def drain(self):
        out = []
        while self.pending():
            out += self.poll()
        return out

    def close(self):
        if self.srv:
            F.fuseflow_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@contextmanager
def _no_gc_pauses():
    """The cyclic garbage collector stays off while a trace is replayed: a full collection
    of a large process can stall the polling loop for tens of milliseconds, which would show
    up as frame latency (reference counting still frees everything the loop allocates)."""
    gc.collect()
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def _summary(lat_s, first_arrival, last_done, n, px_total, statuses):
    lat = np.sort(np.asarray(lat_s)) * 1e3
    span = max(last_done - first_arrival, 1e-9)
    return {"frames": n, "frames_per_s": round(n / span, 2), "px_per_s": round(px_total / span, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 3) if n else None,
            "p99_ms": round(float(np.percentile(lat, 99)), 3) if n else None,
            "max_ms": round(float(lat[-1]), 3) if n else None,
            "all_ok": all(s == F.FUSEFLOW_OK for s in statuses)}


def without_removed(trace, removals):
    """The trace without the arrivals of each removed rig from its removal time on."""
    cut = {r: t for t, r in removals}
    return [(t, r) for t, r in trace if r not in cut or t < cut[r]]


def replay_served(server: Server, rig_ids, frames, outputs, trace, px_per_rig, removals=()):
    """Replays `trace` in wall-clock time through the server.  frames[r] is rig r's pinned
    frame, outputs[r] a deque of HostCloud buffers (at least one per slot).  removals:
    (time s, rig index) events at which a rig is removed from the server (its later
    arrivals are not submitted; frames it still had waiting are reported cancelled)."""
    with _no_gc_pauses():
        return _replay_served(server, rig_ids, frames, outputs, trace, px_per_rig, removals)


def _replay_served(server, rig_ids, frames, outputs, trace, px_per_rig, removals):
    t0 = time.perf_counter()
    nxt, inflight, lat, statuses, px = 0, {}, [], [], 0
    last = t0
    first = trace[0][0] if trace else 0.0
    waiting = deque()
    removals = sorted(removals)
    cut = removals[0][0] if removals else None
    removed = set()
    n_cancelled = 0
    arrivals = []
    trace = without_removed(trace, removals)
    while nxt < len(trace) or inflight or waiting:
        now = time.perf_counter() - t0
        while removals and removals[0][0] <= now:
            _, r = removals.pop(0)
            server.remove_rig(rig_ids[r])
            removed.add(r)
            waiting = deque(w for w in waiting if w[1] != r)
        while nxt < len(trace) and trace[nxt][0] <= now:
            waiting.append(trace[nxt])
            nxt += 1
        # admit arrived frames whose rig has a free output buffer (the server queues them
        # on its slots; buffers bound the frames in flight per rig)
        for _ in range(len(waiting)):
            t_arr, r = waiting.popleft()
            if outputs[r]:
                buf = outputs[r].popleft()
                req = server.submit(rig_ids[r], frames[r], buf)
                inflight[req] = (t_arr, r, buf)
            else:
                waiting.append((t_arr, r))
        for req, _, status, st in server.poll():
            t_done = time.perf_counter() - t0
            t_arr, r, buf = inflight.pop(req)
            outputs[r].append(buf)
            if status == F.FUSEFLOW_ERR_CANCELLED:
                n_cancelled += 1
                continue
            lat.append(t_done - t_arr)
            arrivals.append(t_arr)
            statuses.append(status)
            px += px_per_rig[r]
            last = t_done
    out = _summary(lat, first, last, len(lat), px, statuses)
    out["cancelled"] = n_cancelled
    if cut is not None and lat:
        la, ar = np.asarray(lat) * 1e3, np.asarray(arrivals)
        for name, m in (("before_removal", ar < cut), ("after_removal", ar >= cut + 1.0)):
            if m.any():
                out[name] = {"frames": int(m.sum()), "p50_ms": round(float(np.percentile(la[m], 50)), 3),
                             "p99_ms": round(float(np.percentile(la[m], 99)), 3)}
        out["phases"] = "arrivals before the removal, and from 1 s after it"
    if lat:
        la, ar = np.asarray(lat) * 1e3, np.asarray(arrivals)
        w = 10.0
        out["p99_ms_per_10s"] = [round(float(np.percentile(la[(ar >= t) & (ar < t + w)], 99)), 2)
                                 for t in np.arange(0.0, float(ar.max()) + 1e-9, w)
                                 if ((ar >= t) & (ar < t + w)).any()]
    return out


def replay_plain(contexts, frames, outputs, trace, px_per_rig, stream: int = 0, removals=()):
    """The same trace through the plain path: one synchronous fuse_frame_host per frame,
    in arrival order (a frame waits for every earlier one); removed rigs' later arrivals
    are left out as in replay_served."""
    with _no_gc_pauses():
        return _replay_plain(contexts, frames, outputs, without_removed(trace, removals),
                             px_per_rig, stream)


def _replay_plain(contexts, frames, outputs, trace, px_per_rig, stream):
    t0 = time.perf_counter()
    lat, statuses, px = [], [], 0
    first = trace[0][0] if trace else 0.0
    last = 0.0
    for t_arr, r in trace:
        now = time.perf_counter() - t0
        if now < t_arr:
            time.sleep(max(0.0, t_arr - now - 2e-4))
            while time.perf_counter() - t0 < t_arr:
                pass
        fr, out = frames[r], outputs[r]
        status, _ = F.fuseflow_fuse_frame_host(
            contexts[r], fr["depth"], fr["conf"], fr["rgb"], out.c.pos, out.c.rgb, out.c.weight,
            out.c.count, out.c.rep, out.c.key, stream)
        t_done = time.perf_counter() - t0
        lat.append(t_done - t_arr)
        statuses.append(status)
        px += px_per_rig[r]
        last = t_done
    return _summary(lat, first, last, len(lat), px, statuses)
