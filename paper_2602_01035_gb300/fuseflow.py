"""Python binding of the C ABI in ``include/fuseflow.h`` (ctypes, argument marshalling only).

Every function here carries the name of the C entry point it calls.  Device memory and
streams come from PyTorch; all arithmetic of the fusion path runs in ``libfuseflow.so``.
There is no fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

FUSEFLOW_OK = 0
FUSEFLOW_ERR_INVALID_ARG = 1
FUSEFLOW_ERR_OUT_OF_MEMORY = 2
FUSEFLOW_ERR_CAPACITY = 3
FUSEFLOW_ERR_CUDA = 4
FUSEFLOW_ERR_TIMEOUT = 5
FUSEFLOW_ERR_INTERNAL = 6
FUSEFLOW_ERR_CANCELLED = 7
FUSEFLOW_DEPTH_U16 = 0
FUSEFLOW_DEPTH_F32 = 1
KEY_NONE = 0xFFFFFFFFFFFFFFFF


class fuseflow_intrinsics(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32)]


class fuseflow_extrinsics(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


class fuseflow_params(C.Structure):
    _fields_ = [("tau", C.c_float), ("k_views", C.c_int32), ("sigma_m", C.c_double),
                ("coarse_cell_m", C.c_double), ("max_level", C.c_int32), ("n_min", C.c_int32),
                ("depth_format", C.c_int32), ("use_conf", C.c_int32), ("depth_scale", C.c_double),
                ("use_consistency", C.c_int32), ("top_k", C.c_int32), ("max_cells", C.c_int64),
                ("screen_min_m", C.c_double), ("screen_max_m", C.c_double),
                ("screen_edge_rel", C.c_float), ("reserved1", C.c_int32)]


class fuseflow_stats(C.Structure):
    _fields_ = [("n_valid", C.c_int64), ("n_gated", C.c_int64), ("n_out_of_range", C.c_int64),
                ("n_cells", C.c_int64), ("bbox", C.c_float * 6), ("error", C.c_int32),
                ("n_coarse", C.c_int32)]

    def as_dict(self) -> dict:
        return {"n_valid": self.n_valid, "n_gated": self.n_gated,
                "n_out_of_range": self.n_out_of_range, "n_cells": self.n_cells,
                "bbox": list(self.bbox), "error": self.error, "n_coarse": self.n_coarse}


class fuseflow_cloud(C.Structure):
    _fields_ = [("stats", C.c_void_p), ("pos", C.c_void_p), ("rgb", C.c_void_p),
                ("weight", C.c_void_p), ("count", C.c_void_p), ("rep", C.c_void_p),
                ("key", C.c_void_p), ("capacity", C.c_int64)]


class fuseflow_trace(C.Structure):
    _fields_ = [("pw", C.c_void_p), ("omega", C.c_void_p), ("e", C.c_void_p),
                ("nview", C.c_void_p), ("key", C.c_void_p)]


class fuseflow_conf_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("delta", C.c_double)]


class fuseflow_host_cloud(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("rgb", C.c_void_p), ("weight", C.c_void_p),
                ("count", C.c_void_p), ("rep", C.c_void_p), ("key", C.c_void_p),
                ("capacity", C.c_int64)]


class fuseflow_tuning(C.Structure):
    _fields_ = [("count_chunks", C.c_int32), ("emit_blocks", C.c_int32),
                ("prefetch_tiles", C.c_int32), ("programmatic", C.c_int32), ("tile_h", C.c_int32)]

    def as_dict(self) -> dict:
        return {"count_chunks": self.count_chunks, "emit_blocks": self.emit_blocks,
                "prefetch_tiles": self.prefetch_tiles, "programmatic": self.programmatic,
                "tile_h": self.tile_h}


class fuseflow_server_stats(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("used_bytes", C.c_int64), ("rigs", C.c_int32),
                ("slots", C.c_int32), ("inflight", C.c_int32), ("waiting", C.c_int32),
                ("frames_submitted", C.c_int64), ("frames_completed", C.c_int64),
                ("frames_failed", C.c_int64), ("frames_cancelled", C.c_int64),
                ("deferred_by_budget", C.c_int64), ("slots_grown", C.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class fuseflow_completion(C.Structure):
    _fields_ = [("request", C.c_int64), ("rig", C.c_int32), ("status", C.c_int32),
                ("stats", fuseflow_stats)]


EXPORTS = {
    "fuseflow_default_params": (None, [C.POINTER(fuseflow_params)]),
    "fuseflow_create": (C.c_int, [C.POINTER(fuseflow_intrinsics), C.POINTER(fuseflow_extrinsics),
                                  C.c_int32, C.POINTER(fuseflow_params), C.POINTER(C.c_void_p)]),
    "fuseflow_destroy": (None, [C.c_void_p]),
    "fuseflow_fuse_frame": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.POINTER(fuseflow_cloud), C.c_void_p]),
    "fuseflow_graph_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "fuseflow_graph_launch": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_cloud), C.c_void_p]),
    "fuseflow_graph_destroy": (None, [C.c_void_p]),
    "fuseflow_get_cloud": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_cloud)]),
    "fuseflow_fuse_points": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                       C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_void_p]),
    "fuseflow_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "fuseflow_batch_fuse": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.c_void_p]),
    "fuseflow_batch_graph_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p),
                                              C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                              C.POINTER(C.c_void_p)]),
    "fuseflow_batch_destroy": (None, [C.c_void_p]),
    "fuseflow_read_stats": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_stats), C.c_void_p]),
    "fuseflow_fuse_frame_host": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                           C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.POINTER(fuseflow_stats), C.c_void_p]),
    "fuseflow_set_trace": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_trace)]),
    "fuseflow_get_neighbours": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "fuseflow_num_pixels": (C.c_int64, [C.c_void_p]),
    "fuseflow_capacity": (C.c_int64, [C.c_void_p]),
    "fuseflow_device_bytes": (C.c_int64, [C.c_void_p]),
    "fuseflow_status_string": (C.c_char_p, [C.c_int]),
    "fuseflow_enable_stage_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "fuseflow_read_stage_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "fuseflow_stage_name": (C.c_char_p, [C.c_int]),
    "fuseflow_fuse_frame_static": (C.c_int, [C.POINTER(fuseflow_intrinsics),
                                             C.POINTER(fuseflow_extrinsics), C.c_int32,
                                             C.POINTER(fuseflow_params), C.POINTER(C.c_void_p),
                                             C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fuseflow_screen_depth": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.c_void_p]),
    "fuseflow_default_conf_params": (None, [C.POINTER(fuseflow_conf_params)]),
    "fuseflow_confidence": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(fuseflow_conf_params), C.c_void_p]),
    "fuseflow_mc_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_void_p),
                                    C.c_double, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64), C.c_void_p]),
    "fuseflow_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_tuning)]),
    "fuseflow_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_tuning)]),
    "fuseflow_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_void_p), C.c_int32, C.POINTER(fuseflow_tuning),
                                    C.POINTER(C.c_double), C.c_void_p]),
    "fuseflow_server_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p),
                                           C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                           C.c_int32, C.POINTER(fuseflow_tuning),
                                           C.POINTER(C.c_double)]),
    "fuseflow_server_create": (C.c_int, [C.c_int64, C.POINTER(C.c_void_p)]),
    "fuseflow_server_add_rig": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_intrinsics),
                                          C.POINTER(fuseflow_extrinsics), C.c_int32,
                                          C.POINTER(fuseflow_params), C.c_int32,
                                          C.POINTER(C.c_int32)]),
    "fuseflow_server_submit": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p),
                                         C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                         C.POINTER(fuseflow_host_cloud), C.POINTER(C.c_int64)]),
    "fuseflow_server_poll": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_completion), C.c_int32,
                                       C.POINTER(C.c_int32)]),
    "fuseflow_server_set_max_inflight": (C.c_int, [C.c_void_p, C.c_int32]),
    "fuseflow_server_reserve": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "fuseflow_server_remove_rig": (C.c_int, [C.c_void_p, C.c_int32]),
    "fuseflow_server_inject_start_failure": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "fuseflow_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(fuseflow_server_stats)]),
    "fuseflow_server_pending": (C.c_int64, [C.c_void_p]),
    "fuseflow_server_device_bytes": (C.c_int64, [C.c_void_p]),
    "fuseflow_server_destroy": (None, [C.c_void_p]),
}
FUSEFLOW_N_STAGES = 6

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfuseflow.so (building it in-tree when stale); raises if it cannot."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libfuseflow.so not found at {_build.LIB}; run build()")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class FuseFlowError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().fuseflow_status_string(status).decode()
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


def _check(status: int, where: str):
    if status != FUSEFLOW_OK:
        raise FuseFlowError(status, where)


# --------------------------------------------------------------------------- marshalling
def fuseflow_default_params(**overrides) -> fuseflow_params:
    p = fuseflow_params()
    load().fuseflow_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def rig_arrays(rig):
    """(intrinsics[], extrinsics[]) ctypes arrays from a rig of pinhole cameras."""
    n = len(rig.cameras)
    intr = (fuseflow_intrinsics * n)()
    extr = (fuseflow_extrinsics * n)()
    for i, c in enumerate(rig.cameras):
        intr[i] = fuseflow_intrinsics(c.fx, c.fy, c.cx, c.cy, c.width, c.height)
        extr[i].R[:] = [float(v) for v in np.asarray(c.R, dtype=np.float64).ravel()]
        extr[i].t[:] = [float(v) for v in np.asarray(c.t, dtype=np.float64).ravel()]
    return intr, extr


def fuseflow_create(intr, extr, n_cams: int, params: fuseflow_params) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(load().fuseflow_create(intr, extr, n_cams, C.byref(params), C.byref(ctx)),
           "fuseflow_create")
    return ctx


def fuseflow_destroy(ctx) -> None:
    load().fuseflow_destroy(ctx)


def _ptr_array(ptrs: Sequence[int]):
    arr = (C.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p.value if isinstance(p, C.c_void_p) else int(p)
    return arr


def fuseflow_fuse_frame(ctx, depth_ptrs, conf_ptrs, rgb_ptrs, stream: int = 0) -> fuseflow_cloud:
    cloud = fuseflow_cloud()
    _check(load().fuseflow_fuse_frame(ctx, _ptr_array(depth_ptrs), _ptr_array(conf_ptrs),
                                      _ptr_array(rgb_ptrs), C.byref(cloud), C.c_void_p(stream)),
           "fuseflow_fuse_frame")
    return cloud


def fuseflow_graph_create(ctx, depth_ptrs, conf_ptrs, rgb_ptrs) -> C.c_void_p:
    g = C.c_void_p()
    _check(load().fuseflow_graph_create(ctx, _ptr_array(depth_ptrs), _ptr_array(conf_ptrs),
                                        _ptr_array(rgb_ptrs), C.byref(g)), "fuseflow_graph_create")
    return g


def fuseflow_graph_launch(graph, stream: int = 0) -> fuseflow_cloud:
    cloud = fuseflow_cloud()
    _check(load().fuseflow_graph_launch(graph, C.byref(cloud), C.c_void_p(stream)),
           "fuseflow_graph_launch")
    return cloud


def fuseflow_graph_destroy(graph) -> None:
    load().fuseflow_graph_destroy(graph)


FUSEFLOW_MAX_BATCH = 8


def fuseflow_get_cloud(ctx) -> fuseflow_cloud:
    cloud = fuseflow_cloud()
    _check(load().fuseflow_get_cloud(ctx, C.byref(cloud)), "fuseflow_get_cloud")
    return cloud


def fuseflow_fuse_points(ctx, depth_ptrs, conf_ptrs, rgb_ptrs, pos: int, weight: int, rgb_out: int,
                         stream: int = 0, counts: bool = True):
    """Point-wise fusion (Table II "No SA") into caller-owned device arrays; returns
    (n_valid, n_gated) when counts, else None (then asynchronous)."""
    nv, ng = C.c_int64(), C.c_int64()
    _check(load().fuseflow_fuse_points(ctx, _ptr_array(depth_ptrs), _ptr_array(conf_ptrs),
                                       _ptr_array(rgb_ptrs), C.c_void_p(pos), C.c_void_p(weight),
                                       C.c_void_p(rgb_out), C.byref(nv) if counts else None,
                                       C.byref(ng) if counts else None, C.c_void_p(stream)),
           "fuseflow_fuse_points")
    return (nv.value, ng.value) if counts else None


def fuseflow_batch_create(ctxs) -> C.c_void_p:
    b = C.c_void_p()
    _check(load().fuseflow_batch_create(_ptr_array(ctxs), len(ctxs), C.byref(b)), "fuseflow_batch_create")
    return b


def _nested(per_ctx):
    """array of per-context pointer arrays (kept alive with the outer array)"""
    inner = [_ptr_array(p) for p in per_ctx]
    outer = (C.c_void_p * len(inner))(*[C.cast(a, C.c_void_p) for a in inner])
    outer._keep = inner
    return outer


def fuseflow_batch_fuse(batch, depth_ptrs, conf_ptrs, rgb_ptrs, stream: int = 0) -> int:
    """depth_ptrs[i] etc.: context i's per-camera device pointers; returns the status."""
    return load().fuseflow_batch_fuse(batch, _nested(depth_ptrs), _nested(conf_ptrs),
                                      _nested(rgb_ptrs), C.c_void_p(stream))


def fuseflow_batch_graph_create(batch, depth_ptrs, conf_ptrs, rgb_ptrs) -> C.c_void_p:
    g = C.c_void_p()
    _check(load().fuseflow_batch_graph_create(batch, _nested(depth_ptrs), _nested(conf_ptrs),
                                              _nested(rgb_ptrs), C.byref(g)),
           "fuseflow_batch_graph_create")
    return g


def fuseflow_batch_destroy(batch) -> None:
    load().fuseflow_batch_destroy(batch)


def fuseflow_read_stats(ctx, stream: int = 0, check: bool = True):
    st = fuseflow_stats()
    status = load().fuseflow_read_stats(ctx, C.byref(st), C.c_void_p(stream))
    if check:
        _check(status, "fuseflow_read_stats")
    return status, st


def fuseflow_fuse_frame_host(ctx, depth_ptrs, conf_ptrs, rgb_ptrs, pos, rgb_out, weight, count,
                             rep, key, stream: int = 0):
    st = fuseflow_stats()
    status = load().fuseflow_fuse_frame_host(
        ctx, _ptr_array(depth_ptrs), _ptr_array(conf_ptrs), _ptr_array(rgb_ptrs),
        C.c_void_p(pos), C.c_void_p(rgb_out), C.c_void_p(weight), C.c_void_p(count),
        C.c_void_p(rep), C.c_void_p(key), C.byref(st), C.c_void_p(stream))
    return status, st


def fuseflow_set_trace(ctx, pw=0, omega=0, e=0, nview=0, key=0, clear: bool = False):
    if clear:
        _check(load().fuseflow_set_trace(ctx, None), "fuseflow_set_trace")
        return
    tr = fuseflow_trace(pw, omega, e, nview, key)
    _check(load().fuseflow_set_trace(ctx, C.byref(tr)), "fuseflow_set_trace")


def fuseflow_get_neighbours(ctx, n_cams: int) -> np.ndarray:
    k1 = C.c_int32()
    _check(load().fuseflow_get_neighbours(ctx, None, C.byref(k1)), "fuseflow_get_neighbours")
    out = np.zeros(max(n_cams * k1.value, 1), dtype=np.int32)
    _check(load().fuseflow_get_neighbours(ctx, out.ctypes.data_as(C.POINTER(C.c_int32)),
                                          C.byref(k1)), "fuseflow_get_neighbours")
    return out[:n_cams * k1.value].reshape(n_cams, k1.value)


def fuseflow_num_pixels(ctx) -> int:
    return int(load().fuseflow_num_pixels(ctx))


def fuseflow_capacity(ctx) -> int:
    return int(load().fuseflow_capacity(ctx))


def fuseflow_device_bytes(ctx) -> int:
    return int(load().fuseflow_device_bytes(ctx))


def fuseflow_fuse_frame_static(intr, extr, n_cams: int, params: fuseflow_params, depth_ptrs,
                               conf_ptrs, rgb_ptrs, pos, rgb_out, weight, count, rep, key, stats,
                               stream: int = 0) -> int:
    """Allocation-free fusion of one frame (device inputs and outputs); returns the status."""
    return load().fuseflow_fuse_frame_static(
        intr, extr, n_cams, C.byref(params), _ptr_array(depth_ptrs), _ptr_array(conf_ptrs),
        _ptr_array(rgb_ptrs), C.c_void_p(pos), C.c_void_p(rgb_out), C.c_void_p(weight),
        C.c_void_p(count), C.c_void_p(rep), C.c_void_p(key), C.c_void_p(stats),
        C.c_void_p(stream))


def fuseflow_enable_stage_timing(ctx, enable: bool) -> None:
    _check(load().fuseflow_enable_stage_timing(ctx, 1 if enable else 0),
           "fuseflow_enable_stage_timing")


def fuseflow_read_stage_times(ctx):
    """(dict stage name -> summed ms, number of frames) since timing was enabled."""
    ms = (C.c_double * FUSEFLOW_N_STAGES)()
    n = C.c_int64()
    _check(load().fuseflow_read_stage_times(ctx, ms, C.byref(n)), "fuseflow_read_stage_times")
    return {fuseflow_stage_name(k): ms[k] for k in range(FUSEFLOW_N_STAGES)}, n.value


def fuseflow_stage_name(stage: int) -> str:
    return load().fuseflow_stage_name(stage).decode()


def fuseflow_status_string(status: int) -> str:
    return load().fuseflow_status_string(status).decode()


def fuseflow_confidence(ctx, depth_ptrs, out_ptrs, stream: int = 0, **weights) -> None:
    """Eq. 3 confidence of every camera's depth image into float32 device buffers."""
    cp = fuseflow_conf_params()
    load().fuseflow_default_conf_params(C.byref(cp))
    for k, v in weights.items():
        setattr(cp, k, v)
    _check(load().fuseflow_confidence(ctx, _ptr_array(depth_ptrs), _ptr_array(out_ptrs),
                                      C.byref(cp), C.c_void_p(stream)), "fuseflow_confidence")


def fuseflow_screen_depth(ctx, in_ptrs, out_ptrs, stream: int = 0) -> None:
    """D^r of Eq. 8 (the context's screen parameters) of every camera into device buffers."""
    _check(load().fuseflow_screen_depth(ctx, _ptr_array(in_ptrs), _ptr_array(out_ptrs),
                                        C.c_void_p(stream)), "fuseflow_screen_depth")


MC_OCCLUSION_M = 0.05   # default occlusion margin of Eq. 12's visibility test, metres


def fuseflow_mc_error(ctx, pos_ptr: int, n_points: int, depth_ptrs, err_ptr: int = 0,
                      nvis_ptr: int = 0, stream: int = 0, occlusion_m: float = MC_OCCLUSION_M):
    """(E_MC in metres, points used): Eq. 12 on n_points device positions."""
    mc = C.c_double()
    used = C.c_int64()
    _check(load().fuseflow_mc_error(ctx, C.c_void_p(pos_ptr), n_points, _ptr_array(depth_ptrs),
                                    float(occlusion_m), C.c_void_p(err_ptr), C.c_void_p(nvis_ptr),
                                    C.byref(mc),
                                    C.byref(used), C.c_void_p(stream)), "fuseflow_mc_error")
    return mc.value, used.value


def fuseflow_get_tuning(ctx) -> fuseflow_tuning:
    tu = fuseflow_tuning()
    _check(load().fuseflow_get_tuning(ctx, C.byref(tu)), "fuseflow_get_tuning")
    return tu


def fuseflow_set_tuning(ctx, count_chunks: int, emit_blocks: int, prefetch_tiles: int,
                        programmatic: int = 0, tile_h: int = 0) -> int:
    """Status of replacing the context's launch geometry (INVALID_ARG leaves it unchanged;
    tile_h 0 keeps the current tile height)."""
    tu = fuseflow_tuning(count_chunks, emit_blocks, prefetch_tiles, programmatic, tile_h)
    return load().fuseflow_set_tuning(ctx, C.byref(tu))


def fuseflow_autotune(ctx, depth_ptrs, conf_ptrs, rgb_ptrs, reps: int = 9, stream: int = 0):
    """(chosen fuseflow_tuning, median frame us before, after) for one device frame."""
    tu = fuseflow_tuning()
    us = (C.c_double * 2)()
    _check(load().fuseflow_autotune(ctx, _ptr_array(depth_ptrs), _ptr_array(conf_ptrs),
                                    _ptr_array(rgb_ptrs), reps, C.byref(tu), us,
                                    C.c_void_p(stream)), "fuseflow_autotune")
    return tu, us[0], us[1]


def fuseflow_server_autotune(srv, rig: int, depth_ptrs, conf_ptrs, rgb_ptrs, reps: int = 9):
    """As fuseflow_autotune for all slots of an idle served rig (HOST frame pointers)."""
    tu = fuseflow_tuning()
    us = (C.c_double * 2)()
    _check(load().fuseflow_server_autotune(srv, rig, _ptr_array(depth_ptrs), _ptr_array(conf_ptrs),
                                           _ptr_array(rgb_ptrs), reps, C.byref(tu), us),
           "fuseflow_server_autotune")
    return tu, us[0], us[1]


def fuseflow_server_create(hbm_budget_bytes: int) -> C.c_void_p:
    srv = C.c_void_p()
    _check(load().fuseflow_server_create(int(hbm_budget_bytes), C.byref(srv)),
           "fuseflow_server_create")
    return srv


def fuseflow_server_add_rig(srv, intr, extr, n_cams: int, params: fuseflow_params,
                            n_slots: int):
    """(status, rig id); CAPACITY when the slots would exceed the budget."""
    rid = C.c_int32(-1)
    status = load().fuseflow_server_add_rig(srv, intr, extr, n_cams, C.byref(params), n_slots,
                                            C.byref(rid))
    return status, rid.value


def fuseflow_server_submit(srv, rig: int, depth_ptrs, conf_ptrs, rgb_ptrs,
                           out: fuseflow_host_cloud) -> int:
    req = C.c_int64()
    _check(load().fuseflow_server_submit(srv, rig, _ptr_array(depth_ptrs), _ptr_array(conf_ptrs),
                                         _ptr_array(rgb_ptrs), C.byref(out), C.byref(req)),
           "fuseflow_server_submit")
    return req.value


def fuseflow_server_poll(srv, buf, max_done: int):
    """Number of completions written into ``buf`` (a fuseflow_completion array)."""
    n = C.c_int32()
    _check(load().fuseflow_server_poll(srv, buf, max_done, C.byref(n)), "fuseflow_server_poll")
    return n.value


def fuseflow_server_set_max_inflight(srv, max_inflight: int) -> None:
    _check(load().fuseflow_server_set_max_inflight(srv, max_inflight),
           "fuseflow_server_set_max_inflight")


def fuseflow_server_reserve(srv, rig: int, n_slots: int) -> int:
    held = C.c_int32()
    _check(load().fuseflow_server_reserve(srv, rig, n_slots, C.byref(held)), "fuseflow_server_reserve")
    return held.value


def fuseflow_server_remove_rig(srv, rig: int) -> None:
    _check(load().fuseflow_server_remove_rig(srv, rig), "fuseflow_server_remove_rig")


def fuseflow_server_inject_start_failure(srv, n: int, status: int, after_copies: bool) -> None:
    _check(load().fuseflow_server_inject_start_failure(srv, n, status, int(after_copies)),
           "fuseflow_server_inject_start_failure")


def fuseflow_server_get_stats(srv) -> dict:
    st = fuseflow_server_stats()
    _check(load().fuseflow_server_get_stats(srv, C.byref(st)), "fuseflow_server_get_stats")
    return st.as_dict()


def fuseflow_server_pending(srv) -> int:
    return int(load().fuseflow_server_pending(srv))


def fuseflow_server_device_bytes(srv) -> int:
    return int(load().fuseflow_server_device_bytes(srv))


def fuseflow_server_destroy(srv) -> None:
    load().fuseflow_server_destroy(srv)


# --------------------------------------------------------------------------- torch helpers
class _CudaArray:
    """Zero-copy view of a context-owned device array (``__cuda_array_interface__``)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr: int, shape, typestr: str):
    import torch
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


class FuseFlow:
    """One context per rig: ``fuse(depth, conf, rgb)`` takes lists of CUDA tensors."""

    def __init__(self, rig, **params):
        self.rig = rig
        fmt = FUSEFLOW_DEPTH_F32 if rig.depth_format == "f32" else FUSEFLOW_DEPTH_U16
        p = fuseflow_default_params(depth_format=fmt, depth_scale=float(rig.depth_scale))
        for k, v in params.items():
            setattr(p, k, v)
        self.params = p
        self.intr, self.extr = rig_arrays(rig)
        self.ctx = fuseflow_create(self.intr, self.extr, len(rig.cameras), p)
        self.n_pixels = fuseflow_num_pixels(self.ctx)
        self.capacity = fuseflow_capacity(self.ctx)

    def close(self):
        if self.ctx:
            fuseflow_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def neighbours(self) -> np.ndarray:
        return fuseflow_get_neighbours(self.ctx, len(self.rig.cameras))

    def fuse_ptrs(self, depth_ptrs, conf_ptrs, rgb_ptrs, stream: Optional[int] = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        return fuseflow_fuse_frame(self.ctx, depth_ptrs, conf_ptrs, rgb_ptrs, stream)

    def fuse(self, depth, conf, rgb, stream: Optional[int] = None):
        for t in list(depth) + list(conf) + list(rgb):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("inputs must be contiguous CUDA tensors")
        return self.fuse_ptrs([t.data_ptr() for t in depth], [t.data_ptr() for t in conf],
                              [t.data_ptr() for t in rgb], stream)

    def stats(self, stream: Optional[int] = None, check: bool = True):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        return fuseflow_read_stats(self.ctx, stream, check)

    def cloud_tensors(self, cloud: fuseflow_cloud, n: int) -> dict:
        """Zero-copy torch views of the first ``n`` cells of a fused cloud (count, rep and key
        are exposed as signed integers of the same width; view them as unsigned)."""
        return {"pos": device_view(cloud.pos, (n, 3), "<f4"),
                "rgb": device_view(cloud.rgb, (n, 3), "<f4"),
                "weight": device_view(cloud.weight, (n,), "<f4"),
                "count": device_view(cloud.count, (n,), "<i4"),
                "rep": device_view(cloud.rep, (n,), "<i4"),
                "key": device_view(cloud.key, (n,), "<i8")}

    def autotune(self, depth, conf, rgb, reps: int = 9, stream: Optional[int] = None):
        """Tunes the launch geometry on one frame of CUDA tensors: (tuning, us before, after)."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        return fuseflow_autotune(self.ctx, [t.data_ptr() for t in depth],
                                 [t.data_ptr() for t in conf], [t.data_ptr() for t in rgb],
                                 reps, stream)

    def graph(self, depth, conf, rgb) -> "FrameGraph":
        """The fuse call on these CUDA tensors recorded once, for replay (the tensors are
        read at every launch; keep them alive while the graph is used)."""
        return FrameGraph(self, depth, conf, rgb)

    def tuning(self) -> dict:
        return fuseflow_get_tuning(self.ctx).as_dict()

    def set_tuning(self, count_chunks: int, emit_blocks: int, prefetch_tiles: int,
                   programmatic: int = 0, tile_h: int = 0):
        _check(fuseflow_set_tuning(self.ctx, count_chunks, emit_blocks, prefetch_tiles,
                                   programmatic, tile_h), "fuseflow_set_tuning")

    def set_trace(self, **arrays):
        fuseflow_set_trace(self.ctx, **{k: (v.data_ptr() if v is not None else 0)
                                        for k, v in arrays.items()})

    def clear_trace(self):
        fuseflow_set_trace(self.ctx, clear=True)


class FrameGraph:
    """A recorded fuse call of one context (fuseflow_graph_*)."""

    def __init__(self, ff: "FuseFlow", depth, conf, rgb):
        self.ff = ff
        self.inputs = (list(depth), list(conf), list(rgb))
        self.g = fuseflow_graph_create(ff.ctx, [t.data_ptr() for t in depth],
                                       [t.data_ptr() for t in conf], [t.data_ptr() for t in rgb])

    def launch(self, stream: Optional[int] = None) -> fuseflow_cloud:
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        return fuseflow_graph_launch(self.g, stream)

    def close(self):
        if self.g:
            fuseflow_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several contexts fused by one launch of each frame kernel (fuseflow_batch_*)."""

    def __init__(self, contexts: Sequence["FuseFlow"]):
        self.contexts = list(contexts)
        self.b = fuseflow_batch_create([c.ctx for c in self.contexts])

    def fuse(self, frames, stream: Optional[int] = None) -> int:
        """frames[i] = (depth, conf, rgb) lists of CUDA tensors of context i."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        return fuseflow_batch_fuse(self.b, *self._ptrs(frames), stream)

    def fuse_ptrs(self, depth_ptrs, conf_ptrs, rgb_ptrs, stream: int) -> int:
        return fuseflow_batch_fuse(self.b, depth_ptrs, conf_ptrs, rgb_ptrs, stream)

    @staticmethod
    def _ptrs(frames):
        return ([[t.data_ptr() for t in f[0]] for f in frames], [[t.data_ptr() for t in f[1]] for f in frames],
                [[t.data_ptr() for t in f[2]] for f in frames])

    def graph(self, frames) -> "BatchGraph":
        return BatchGraph(self, frames)

    def close(self):
        if self.b:
            fuseflow_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchGraph:
    """A recorded batch call on fixed input tensors (keep them alive while it is used)."""

    def __init__(self, batch: Batch, frames):
        self.batch = batch
        self.frames = frames
        self.g = fuseflow_batch_graph_create(batch.b, *Batch._ptrs(frames))

    def launch(self, stream: Optional[int] = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        return fuseflow_graph_launch(self.g, stream)

    def close(self):
        if self.g:
            fuseflow_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
