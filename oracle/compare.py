"""Comparison of a fused frame from the CUDA path with the FP64 oracle.

TEST INFRASTRUCTURE ONLY (used by tests/ and by the oracle leg of bench.py); pure numpy on
the dictionaries returned by oracle.fuse_frame and by the GPU-side marshalling.

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

Excluded cells are bounded by the oracle's own prediction: the cells it flags (a member
within the boundary band, or an ambiguous coarse level) plus at most one more cell per
excluded point (the cell on the other side of the face the point may fall into).
"""
from __future__ import annotations

import numpy as np

W_FLOOR = 1e-30
W_ABS = 1e-35
CELL_BOUNDARY, CELL_AMBIGUOUS_LEVEL, CELL_TIE = 1, 2, 4


def point_masks(orc, band_m=1e-5, band_px=1e-6):
    """Per-pixel oracle flags: boundary, ambiguous level, tie."""
    g = orc["in_range"].astype(bool)
    boundary = g & (orc["margin_cell_m"] < band_m)
    tie = orc["gated"].astype(bool) & ((orc["margin_tie_px"] < band_px) | (orc["min_az"] < 1e-6))
    amb = np.zeros_like(g)
    cells = orc["cells"]
    bad = cells["key"][(cells["flags"] & CELL_AMBIGUOUS_LEVEL) != 0]
    if bad.size:
        amb = g & np.isin(orc["key"], bad)
    return boundary, amb, tie


def compare_points(tr, orc, report, rows=None):
    """Per-pixel checks of a GPU trace (pw, e, omega, nview, key) against the oracle;
    `rows` restricts them to a pixel mask.  Returns the excluded (boundary or ambiguous)
    points."""
    gated = orc["gated"].astype(bool)
    if rows is not None:
        gated = gated & rows
    boundary, amb, tie = point_masks(orc)
    # gate (Eq. 9): exact (nview = -2: gated, weight computed per cell by the top-k variant)
    gpu_gated = (tr["nview"] >= 0) | (tr["nview"] == -2)
    if rows is not None:
        gpu_gated = gpu_gated & rows
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
    if rows is not None:
        inr = inr & rows
    cmp = inr & ~boundary & ~amb
    assert np.array_equal(tr["key"][cmp], orc["key"][cmp]), \
        f"{int(np.sum(tr['key'][cmp] != orc['key'][cmp]))} keys differ"
    report["n_points_compared"] = int(cmp.sum())
    report["n_boundary_points"] = int((boundary & inr).sum())
    report["n_ambiguous_points"] = int((amb & inr).sum())
    report["n_tie_points"] = int((tie & gated).sum())
    report["n_key_mismatch_in_excluded"] = int(np.sum(tr["key"][inr & ~cmp] != orc["key"][inr & ~cmp]))
    return (boundary | amb) & inr


def compare_cells(gpu, orc, report, excluded_points=None, gpu_keys=None):
    """Every oracle cell outside the exclusion sets must exist on the GPU with the same
    count and representative, and (outside tie cells) W, position and colour within the
    tolerances.  gpu_keys: the GPU's per-pixel cell keys (trace), used to find the cells
    an excluded point reached on the GPU side."""
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
    order = np.argsort(gc["key"], kind="stable")
    gkeys = gc["key"][order]
    assert np.all(np.diff(gkeys.astype(np.uint64)) != 0) if len(gkeys) > 1 else True, "duplicate keys"
    flags = oc["flags"]
    flagged = (flags & (CELL_BOUNDARY | CELL_AMBIGUOUS_LEVEL)) != 0
    structural = ~flagged
    n_excl_pts = 0
    if excluded_points is not None:
        n_excl_pts = int(excluded_points.sum())
        if gpu_keys is not None:
            # a boundary point may fall into the neighbouring cell on the GPU: exclude every
            # cell that an excluded point reaches on either side
            touched = np.union1d(gpu_keys[excluded_points], orc["key"][excluded_points])
            structural &= ~np.isin(oc["key"], touched)
    valued = structural & ((flags & CELL_TIE) == 0)
    idx = np.flatnonzero(structural)
    k = oc["key"][idx]
    pos = np.searchsorted(gkeys, k)
    pos = np.minimum(pos, max(len(gkeys) - 1, 0))
    found = (len(gkeys) > 0) & (gkeys[pos] == k) if len(gkeys) else np.zeros(len(k), bool)
    assert np.all(found), f"{int((~found).sum())} oracle cells missing on the GPU, e.g. {int(k[~found][0]):#x}"
    j = order[pos]
    bad = gc["count"][j] != oc["count"][idx]
    assert not bad.any(), f"count differs in {int(bad.sum())} cells, e.g. {int(k[bad][0]):#x}"
    bad = gc["rep"][j] != oc["rep"][idx]
    assert not bad.any(), f"representative differs in {int(bad.sum())} cells, e.g. {int(k[bad][0]):#x}"
    v = valued[idx]
    jv, iv = j[v], idx[v]
    wo, wg = oc["weight"][iv], gc["weight"][jv].astype(np.float64)
    big = wo >= W_FLOOR
    rel = np.abs(wg[big] - wo[big]) / wo[big]
    assert np.all(rel <= 1e-5), f"W relative error {rel.max():.3g}"
    assert np.all(np.abs(wg[~big] - wo[~big]) <= W_ABS), "tiny W differs"
    dp = np.abs(gc["pos"][jv].astype(np.float64) - oc["pos"][iv])
    assert np.all(dp <= 1e-5 + 1e-5 * np.abs(oc["pos"][iv])), f"position error {dp.max():.3g}"
    dc = np.abs(gc["rgb"][jv].astype(np.float64) - oc["rgb"][iv])
    assert np.all(dc <= 6e-3), f"colour error {dc.max():.3g}"
    # every GPU cell without an oracle twin must be explained by excluded points
    okeys = np.sort(oc["key"])
    extra = gc["key"][~np.isin(gc["key"], okeys)]
    if extra.size and excluded_points is not None and gpu_keys is not None:
        members = np.isin(gpu_keys, extra)
        assert np.all(excluded_points[members]), "unexplained GPU cell"
    n_excluded = int((~structural).sum())
    n_flagged = int(flagged.sum())
    # the oracle's prediction bounds the exclusions: its flagged cells plus at most one
    # more cell per excluded point
    assert n_excluded <= n_flagged + n_excl_pts, (n_excluded, n_flagged, n_excl_pts)
    n_oracle = int(st_o["n_cells"])
    report.update({"n_cells_gpu": int(st_g["n_cells"]), "n_cells_oracle": n_oracle,
                   "n_cells_matched": int(len(idx)), "n_cells_valued": int(v.sum()),
                   "n_cells_excluded": n_excluded, "n_cells_flagged_by_oracle": n_flagged,
                   "n_cells_excluded_bound": n_flagged + n_excl_pts,
                   "excluded_fraction": round(n_excluded / max(n_oracle, 1), 5),
                   "n_cells_extra_gpu": int(extra.size),
                   "n_tie_cells": int(((flags & CELL_TIE) != 0).sum()),
                   "max_w_rel_err": float(rel.max()) if rel.size else 0.0,
                   "max_pos_err_m": float(dp.max()) if dp.size else 0.0,
                   "max_rgb_err": float(dc.max()) if dc.size else 0.0})
    assert report["n_cells_matched"] + n_excluded == n_oracle
    return report


def compare(gpu, orc):
    """Points (when the GPU result carries a trace) and cells; returns the report."""
    report = {}
    excl, keys = None, None
    if "trace" in gpu:
        excl = compare_points(gpu["trace"], orc, report)
        keys = gpu["trace"]["key"]
    compare_cells(gpu, orc, report, excl, keys)
    return report
