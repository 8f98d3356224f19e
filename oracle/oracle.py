"""ctypes wrapper of the FP64 CPU oracle (``fuseflow_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  It shares no code with the CUDA
path; it receives the same seeded input bytes from ``paper_2602_01035_gb300.scenes``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fuseflow_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEPTH_FORMATS = {"u16": 0, "f32": 1, "f64": 2}
CELL_BOUNDARY, CELL_AMBIGUOUS_LEVEL, CELL_TIE = 1, 2, 4
KEY_NONE = np.uint64(0xFFFFFFFFFFFFFFFF)


class _Camera(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("R", C.c_double * 9),
                ("t", C.c_double * 3)]


class _Params(C.Structure):
    _fields_ = [("tau", C.c_float), ("k_views", C.c_int32), ("sigma_m", C.c_double),
                ("coarse_cell_m", C.c_double), ("max_level", C.c_int32), ("n_min", C.c_int32),
                ("depth_format", C.c_int32), ("use_conf", C.c_int32), ("depth_scale", C.c_double),
                ("use_consistency", C.c_int32), ("row_step", C.c_int32), ("band_m", C.c_double),
                ("band_px", C.c_double), ("band_az", C.c_double), ("top_k", C.c_int32),
                ("screen_min_m", C.c_double), ("screen_max_m", C.c_double),
                ("screen_edge_rel", C.c_float)]


_P = C.c_void_p


class _Points(C.Structure):
    _fields_ = [(n, _P) for n in ("valid", "gated", "in_range", "pw", "e", "omega", "log_omega",
                                  "nview", "key", "level", "margin_cell_m", "margin_tie_px",
                                  "min_az")]


class _Cells(C.Structure):
    _fields_ = [(n, _P) for n in ("key", "count", "rep", "weight", "pos", "rgb", "flags")]


class _Stats(C.Structure):
    _fields_ = [("n_valid", C.c_int64), ("n_gated", C.c_int64), ("n_out_of_range", C.c_int64),
                ("n_cells", C.c_int64), ("bbox", C.c_double * 6),
                ("n_boundary_points", C.c_int64), ("n_tie_points", C.c_int64),
                ("n_ambiguous_coarse", C.c_int64), ("n_coarse", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fuseflow_oracle.h"))):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                                   "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        lib.orc_fuse_frame.restype = C.c_int
        lib.orc_fuse_frame.argtypes = [C.POINTER(_Camera), C.c_int32, C.POINTER(_Params),
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                       C.POINTER(C.c_void_p), C.POINTER(_Points),
                                       C.POINTER(_Cells), C.c_int64, C.POINTER(_Stats)]
        lib.orc_neighbours.restype = C.c_int
        lib.orc_neighbours.argtypes = [C.POINTER(_Camera), C.c_int32, C.c_int32,
                                       C.POINTER(C.c_int32)]
        lib.orc_mc_error.restype = C.c_int
        lib.orc_mc_error.argtypes = [C.POINTER(_Camera), C.c_int32, C.POINTER(_Params),
                                     C.POINTER(C.c_void_p), C.c_void_p, C.c_int64, C.c_double,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                     C.POINTER(C.c_int64)]
        lib.orc_confidence.restype = C.c_int
        lib.orc_confidence.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(_Params),
                                       C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p]
        lib.orc_screen_depth.restype = C.c_int
        lib.orc_screen_depth.argtypes = [C.POINTER(_Params), C.c_int32, C.c_int32, C.c_void_p,
                                         C.c_void_p]
        lib.orc_default_params.restype = None
        lib.orc_default_params.argtypes = [C.POINTER(_Params)]
        _lib = lib
    return _lib


def _cams(rig):
    arr = (_Camera * rig.n_cams)()
    for k, c in enumerate(rig.cameras):
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = c.fx, c.fy, c.cx, c.cy
        arr[k].width, arr[k].height = c.width, c.height
        arr[k].R[:] = [float(v) for v in np.asarray(c.R, dtype=np.float64).ravel()]
        arr[k].t[:] = [float(v) for v in np.asarray(c.t, dtype=np.float64).ravel()]
    return arr


def default_params() -> dict:
    p = _Params()
    _load().orc_default_params(C.byref(p))
    return {name: getattr(p, name) for name, _ in _Params._fields_}


def neighbours(rig, k_views: int = 4) -> np.ndarray:
    K = min(k_views, rig.n_cams)
    out = np.zeros((rig.n_cams, max(K - 1, 0)), dtype=np.int32)
    buf = np.zeros(max(out.size, 1), dtype=np.int32)
    rc = _load().orc_neighbours(_cams(rig), rig.n_cams, k_views,
                                buf.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise ValueError(f"orc_neighbours failed: {rc}")
    out[...] = buf[:out.size].reshape(out.shape)
    return out


def fuse_frame(rig, frame, params: dict | None = None, points: bool = True,
               depth_format: str | None = None, cell_capacity: int | None = None) -> dict:
    """Run the oracle on one frame; returns numpy arrays (per pixel and per cell) and stats."""
    lib = _load()
    prm = _Params()
    lib.orc_default_params(C.byref(prm))
    fmt = depth_format or rig.depth_format
    prm.depth_format = DEPTH_FORMATS[fmt]
    prm.depth_scale = rig.depth_scale
    for k, v in (params or {}).items():
        if k in ("max_cells", "autotune"):
            continue
        setattr(prm, k, v)
    n = rig.n_cams
    keep = []
    dep = (C.c_void_p * n)()
    cnf = (C.c_void_p * n)()
    col = (C.c_void_p * n)()
    want = {"u16": np.uint16, "f32": np.float32, "f64": np.float64}[fmt]
    for i in range(n):
        d = np.ascontiguousarray(frame.depth[i], dtype=want)
        c = np.ascontiguousarray(frame.conf[i], dtype=np.float32)
        r = np.ascontiguousarray(frame.rgb[i], dtype=np.uint8)
        keep += [d, c, r]
        dep[i], cnf[i], col[i] = d.ctypes.data, c.ctypes.data, r.ctypes.data
    npx = rig.n_pixels
    out = {}
    pts = _Points()
    if points:
        spec = {"valid": (np.uint8, ()), "gated": (np.uint8, ()), "in_range": (np.uint8, ()),
                "pw": (np.float64, (3,)), "e": (np.float64, ()), "omega": (np.float64, ()),
                "log_omega": (np.float64, ()), "nview": (np.int32, ()), "key": (np.uint64, ()),
                "level": (np.int32, ()), "margin_cell_m": (np.float64, ()),
                "margin_tie_px": (np.float64, ()), "min_az": (np.float64, ())}
        for name, (dt, tail) in spec.items():
            a = np.zeros((npx,) + tail, dtype=dt)
            if name == "pw" or name in ("e", "omega", "log_omega"):
                a[...] = np.nan
            out[name] = a
            setattr(pts, name, a.ctypes.data)
    cap = npx if cell_capacity is None else cell_capacity
    cap = max(cap, 1)
    cells_np = {"key": np.zeros(cap, np.uint64), "count": np.zeros(cap, np.uint32),
                "rep": np.zeros(cap, np.uint32), "weight": np.zeros(cap, np.float64),
                "pos": np.zeros((cap, 3), np.float64), "rgb": np.zeros((cap, 3), np.float64),
                "flags": np.zeros(cap, np.uint32)}
    cells = _Cells(*[cells_np[n].ctypes.data for n, _ in _Cells._fields_])
    st = _Stats()
    rc = lib.orc_fuse_frame(_cams(rig), n, C.byref(prm), dep, cnf, col,
                            C.byref(pts) if points else None, C.byref(cells), cap, C.byref(st))
    if rc != 0:
        raise RuntimeError(f"orc_fuse_frame failed with status {rc}")
    nc = st.n_cells
    out["cells"] = {k: v[:nc] for k, v in cells_np.items()}
    out["stats"] = {name: (list(getattr(st, name)) if name == "bbox" else int(getattr(st, name)))
                    for name, _ in _Stats._fields_}
    out["params"] = {name: getattr(prm, name) for name, _ in _Params._fields_}
    return out


MC_OCCLUSION_M = 0.05   # about three times the sensor noise at 3 m (0.0015 z^2)


def mc_error(rig, depth, points, occlusion_m: float = MC_OCCLUSION_M,
             depth_format: str | None = None) -> dict:
    """Eq. 12 on a point set (n x 3 metres) against the rig's depth maps (FP64 oracle):
    per-point error (metres), visible cameras, tie margin (px), the mean and its count."""
    lib = _load()
    prm = _Params()
    lib.orc_default_params(C.byref(prm))
    fmt = depth_format or rig.depth_format
    prm.depth_format = DEPTH_FORMATS[fmt]
    prm.depth_scale = rig.depth_scale
    want = {"u16": np.uint16, "f32": np.float32, "f64": np.float64}[fmt]
    keep = [np.ascontiguousarray(d, dtype=want) for d in depth]
    dep = (C.c_void_p * rig.n_cams)(*[d.ctypes.data for d in keep])
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    n = len(pts)
    err = np.zeros(max(n, 1), np.float64)
    nvis = np.zeros(max(n, 1), np.int32)
    tie = np.zeros(max(n, 1), np.float64)
    mc = C.c_double()
    used = C.c_int64()
    rc = lib.orc_mc_error(_cams(rig), rig.n_cams, C.byref(prm), dep, pts.ctypes.data, n,
                          float(occlusion_m), err.ctypes.data, nvis.ctypes.data, tie.ctypes.data, C.byref(mc),
                          C.byref(used))
    if rc != 0:
        raise RuntimeError(f"orc_mc_error failed with status {rc}")
    return {"err_m": err[:n], "nvis": nvis[:n], "tie_px": tie[:n], "mc_m": mc.value,
            "n_used": used.value}


PAPER_CONF = {"alpha": 0.5, "beta": 0.5, "gamma": 1.0, "delta": 1.0}   # Eq. 3's constants


def confidence(depth, depth_format: str, depth_scale: float, alpha=0.5, beta=0.5, gamma=1.0,
               delta=1.0) -> np.ndarray:
    """Eq. 3 confidence of one depth image (FP64 oracle)."""
    lib = _load()
    prm = _Params()
    lib.orc_default_params(C.byref(prm))
    prm.depth_format = DEPTH_FORMATS[depth_format]
    prm.depth_scale = depth_scale
    want = {"u16": np.uint16, "f32": np.float32, "f64": np.float64}[depth_format]
    d = np.ascontiguousarray(depth, dtype=want)
    h, w = d.shape
    out = np.zeros((h, w), np.float64)
    rc = lib.orc_confidence(d.ctypes.data, w, h, C.byref(prm), alpha, beta, gamma, delta,
                            out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"orc_confidence failed with status {rc}")
    return out


def screen_depth(depth, depth_format: str, depth_scale: float, screen_min_m: float = 0.0,
                 screen_max_m: float = 0.0, screen_edge_rel: float = 0.0) -> np.ndarray:
    """D^r of Eq. 8 of one depth image under the stated screen rule (oracle)."""
    lib = _load()
    prm = _Params()
    lib.orc_default_params(C.byref(prm))
    prm.depth_format = DEPTH_FORMATS[depth_format]
    prm.depth_scale = depth_scale
    prm.screen_min_m, prm.screen_max_m = screen_min_m, screen_max_m
    prm.screen_edge_rel = screen_edge_rel
    want = {"u16": np.uint16, "f32": np.float32, "f64": np.float64}[depth_format]
    d = np.ascontiguousarray(depth, dtype=want)
    h, w = d.shape
    out = np.empty_like(d)
    rc = lib.orc_screen_depth(C.byref(prm), w, h, d.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"orc_screen_depth failed with status {rc}")
    return out


def key_fields(key):
    """Split packed cell keys into (level, kx, ky, kz)."""
    key = np.asarray(key, dtype=np.uint64)
    m = np.uint64((1 << 20) - 1)
    lvl = (key >> np.uint64(60)).astype(np.int64)
    kx = ((key >> np.uint64(40)) & m).astype(np.int64) - (1 << 19)
    ky = ((key >> np.uint64(20)) & m).astype(np.int64) - (1 << 19)
    kz = (key & m).astype(np.int64) - (1 << 19)
    return lvl, kx, ky, kz
