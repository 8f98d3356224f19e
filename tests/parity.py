"""Comparison of the CUDA path with the FP64 oracle (test helper): GPU-side marshalling
here, the comparison itself in oracle/compare.py.

Tolerances (from the arithmetic; the targets are 1e-5 m and 1e-5 relative):
* integer outputs (counts, keys, representative, valid/gated counts): exact, except for
  the ambiguity sets the oracle reports: points within 1e-5 m of a cell boundary, coarse
  cells whose level could flip when such points move, and projections within 1e-6 px of
  a half-pixel tie (the latter only affect weights).
* joint weight omega and cell weight W: 1e-5 relative while the oracle value is a normal
  float32 number above 1e-30; below that float32 cannot carry 1e-5 relative precision
  and the difference must be below 1e-35.
* exponent e of Eq. 7 (float32 trace): |de| <= 1e-5 + 2^-23 e.
* positions: 1e-5 m + 1e-5 relative; colour: 6e-3 on the 0..255 scale (the mean of
  8-bit colours under weights with 1e-5 relative error moves by at most 2 * 1e-5 * 255).
"""
from __future__ import annotations

import numpy as np

from oracle.compare import W_ABS, W_FLOOR  # noqa: F401  (re-exported)


def run_gpu(ff, frame, torch, with_trace=True):
    """Fuse one frame through the C ABI; returns numpy outputs (+ per-pixel trace)."""
    dev = torch.device("cuda")
    depth = [torch.from_numpy(np.ascontiguousarray(d)).to(dev) for d in frame.depth]
    conf = [torch.from_numpy(np.ascontiguousarray(c)).to(dev) for c in frame.conf]
    rgb = [torch.from_numpy(np.ascontiguousarray(r)).to(dev) for r in frame.rgb]
    npx = ff.n_pixels
    tr = None
    if with_trace:
        tr = {"pw": torch.full((npx, 3), float("nan"), device=dev),
              "omega": torch.full((npx,), float("nan"), device=dev),
              "e": torch.full((npx,), float("nan"), device=dev),
              "nview": torch.full((npx,), -7, dtype=torch.int32, device=dev),
              "key": torch.zeros((npx,), dtype=torch.int64, device=dev)}
        ff.set_trace(**tr)
    cloud = ff.fuse(depth, conf, rgb)
    status, st = ff.stats(check=False)
    if with_trace:
        ff.clear_trace()
    n = int(st.n_cells)
    out = {k: v.cpu().numpy().copy() for k, v in ff.cloud_tensors(cloud, n).items()} if n else {
        "pos": np.zeros((0, 3), np.float32), "rgb": np.zeros((0, 3), np.float32),
        "weight": np.zeros(0, np.float32), "count": np.zeros(0, np.uint32),
        "rep": np.zeros(0, np.uint32), "key": np.zeros(0, np.uint64)}
    for k, dt in (("count", np.uint32), ("rep", np.uint32), ("key", np.uint64)):
        out[k] = out[k].view(dt)
    res = {"status": status, "stats": st.as_dict(), "cells": out}
    if with_trace:
        t = {k: v.cpu().numpy() for k, v in tr.items()}
        t["key"] = t["key"].view(np.uint64)
        res["trace"] = t
    return res


def compare(gpu, orc, oracle_mod=None):
    """Points and cells against the oracle (oracle.compare); returns the report."""
    from oracle import compare as OC
    return OC.compare(gpu, orc)
