"""Comparison of the CUDA path with the FP64 oracle (test helper).

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

W_FLOOR = 1e-30
W_ABS = 1e-35


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


def point_masks(orc, oracle_mod, band_m=1e-5, band_px=1e-6):
    """Per-pixel oracle flags: boundary, ambiguous level, tie."""
    g = orc["in_range"].astype(bool)
    boundary = g & (orc["margin_cell_m"] < band_m)
    tie = orc["gated"].astype(bool) & ((orc["margin_tie_px"] < band_px) | (orc["min_az"] < 1e-6))
    amb = np.zeros_like(g)
    cells = orc["cells"]
    bad = cells["key"][(cells["flags"] & oracle_mod.CELL_AMBIGUOUS_LEVEL) != 0]
    if bad.size:
        amb = g & np.isin(orc["key"], bad)
    return boundary, amb, tie


def compare_points(gpu, orc, oracle_mod, report):
    tr = gpu["trace"]
    gated = orc["gated"].astype(bool)
    boundary, amb, tie = point_masks(orc, oracle_mod)
    # gate (Eq. 9): exact (nview = -2: gated, weight computed per cell by the top-k variant)
    gpu_gated = (tr["nview"] >= 0) | (tr["nview"] == -2)
    assert np.array_equal(gpu_gated, gated), "gated set differs"
    weights_traced = not np.all(tr["nview"][gpu_gated] == -2)
    # Eq. 8 world points
    dp = np.abs(tr["pw"][gated].astype(np.float64) - orc["pw"][gated])
    tol = 1e-5 + 1e-6 * np.abs(orc["pw"][gated])
    assert np.all(dp <= tol), f"world point error {dp.max():.3g} m"
    report["max_pw_err_m"] = float(dp.max()) if dp.size else 0.0
    # Eq. 4-7: views and exponent
    ok = gated & ~tie
    if not weights_traced:
        ok = ok & False
    assert np.array_equal(tr["nview"][ok], orc["nview"][ok]), "valid-view counts differ"
    de = np.abs(tr["e"][ok].astype(np.float64) - orc["e"][ok])
    assert np.all(de <= 1e-5 + 2.0 ** -23 * orc["e"][ok]), f"exponent error {de.max():.3g}"
    # Eq. 10 joint weight
    wo = orc["omega"][ok]
    wg = tr["omega"][ok].astype(np.float64)
    big = wo >= W_FLOOR
    rel = np.abs(wg[big] - wo[big]) / wo[big]
    assert np.all(rel <= 1e-5), f"omega relative error {rel.max():.3g}"
    assert np.all(np.abs(wg[~big] - wo[~big]) <= W_ABS), "tiny omega differs"
    report["max_omega_rel_err"] = float(rel.max()) if rel.size else 0.0
    # Sec. II.5(1) keys: exact outside the ambiguity sets
    inr = orc["in_range"].astype(bool)
    cmp = inr & ~boundary & ~amb
    assert np.array_equal(tr["key"][cmp], orc["key"][cmp]), \
        f"{int(np.sum(tr['key'][cmp] != orc['key'][cmp]))} keys differ"
    report["n_points_compared"] = int(cmp.sum())
    report["n_boundary_points"] = int(boundary.sum())
    report["n_ambiguous_points"] = int(amb.sum())
    report["n_tie_points"] = int(tie.sum())
    report["n_key_mismatch_in_excluded"] = int(np.sum(tr["key"][inr & ~cmp] != orc["key"][inr & ~cmp]))
    return boundary | amb


def compare_cells(gpu, orc, oracle_mod, report, excluded_points=None):
    st_g, st_o = gpu["stats"], orc["stats"]
    for k in ("n_valid", "n_gated", "n_out_of_range"):
        assert st_g[k] == st_o[k], f"{k}: gpu {st_g[k]} oracle {st_o[k]}"
    if st_o["n_gated"]:
        bb_g = np.array(st_g["bbox"], dtype=np.float64)
        bb_o = np.array(st_o["bbox"], dtype=np.float64)
        assert np.all(np.abs(bb_g - bb_o) <= 1e-5 + 1e-6 * np.abs(bb_o)), "extent differs"
    gc, oc = gpu["cells"], orc["cells"]
    assert len(gc["key"]) == st_g["n_cells"]
    assert np.all(np.diff(gc["rep"].astype(np.int64)) > 0), "output not ordered by representative"
    gidx = {int(k): i for i, k in enumerate(gc["key"])}
    assert len(gidx) == len(gc["key"]), "duplicate keys"
    flags = oc["flags"]
    structural = (flags & (oracle_mod.CELL_BOUNDARY | oracle_mod.CELL_AMBIGUOUS_LEVEL)) == 0
    if excluded_points is not None and "trace" in gpu:
        # a boundary point may fall into the neighbouring cell on the GPU: exclude every
        # cell that an excluded point reaches on either side
        touched = np.union1d(gpu["trace"]["key"][excluded_points], orc["key"][excluded_points])
        structural &= ~np.isin(oc["key"], touched)
    valued = structural & ((flags & oracle_mod.CELL_TIE) == 0)
    n_match = 0
    worst = {"w": 0.0, "pos": 0.0, "rgb": 0.0}
    for i in np.flatnonzero(structural):
        k = int(oc["key"][i])
        assert k in gidx, f"cell {k:#x} missing on the GPU"
        j = gidx[k]
        assert gc["count"][j] == oc["count"][i], f"count differs in cell {k:#x}"
        assert gc["rep"][j] == oc["rep"][i], f"representative differs in cell {k:#x}"
        n_match += 1
        if not valued[i]:
            continue
        wo, wg = oc["weight"][i], float(gc["weight"][j])
        if wo >= W_FLOOR:
            r = abs(wg - wo) / wo
            assert r <= 1e-5, f"W relative error {r:.3g} in cell {k:#x}"
            worst["w"] = max(worst["w"], r)
        else:
            assert abs(wg - wo) <= W_ABS
        dp = np.abs(gc["pos"][j].astype(np.float64) - oc["pos"][i])
        assert np.all(dp <= 1e-5 + 1e-5 * np.abs(oc["pos"][i])), f"position error {dp.max():.3g}"
        worst["pos"] = max(worst["pos"], float(dp.max()))
        dc = np.abs(gc["rgb"][j].astype(np.float64) - oc["rgb"][i])
        assert np.all(dc <= 6e-3), f"colour error {dc.max():.3g}"
        worst["rgb"] = max(worst["rgb"], float(dc.max()))
    # every GPU cell without an oracle twin must be explained by excluded points
    okeys = set(int(k) for k in oc["key"])
    extra = [int(k) for k in gc["key"] if int(k) not in okeys]
    if extra and excluded_points is not None and "trace" in gpu:
        tk = gpu["trace"]["key"]
        for k in extra:
            members = tk == np.uint64(k)
            assert np.all(excluded_points[members]), f"unexplained GPU cell {k:#x}"
    report.update({"n_cells_gpu": int(st_g["n_cells"]), "n_cells_oracle": int(st_o["n_cells"]),
                   "n_cells_matched": n_match, "n_cells_excluded": int((~structural).sum()),
                   "n_cells_extra_gpu": len(extra), "max_w_rel_err": worst["w"],
                   "max_pos_err_m": worst["pos"], "max_rgb_err": worst["rgb"]})
    return report


def compare(gpu, orc, oracle_mod):
    report = {}
    excl = compare_points(gpu, orc, oracle_mod, report) if "trace" in gpu else None
    compare_cells(gpu, orc, oracle_mod, report, excl)
    return report
