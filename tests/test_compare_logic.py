"""The oracle-vs-GPU comparison (oracle/compare.py) on CPU: a result built from the oracle's
own output in the GPU's layout (float32 values, cells ordered by representative, per-pixel
trace) passes, and planted differences in a count, a representative, a weight, a position
or a key fail."""
import copy

import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S


def _as_gpu(orc):
    cells = orc["cells"]
    order = np.argsort(cells["rep"], kind="stable")
    gc = {"pos": cells["pos"][order].astype(np.float32), "rgb": cells["rgb"][order].astype(np.float32),
          "weight": cells["weight"][order].astype(np.float32), "count": cells["count"][order],
          "rep": cells["rep"][order], "key": cells["key"][order]}
    st = dict(orc["stats"])
    st["bbox"] = [float(np.float32(v)) for v in st["bbox"]]
    g = orc["gated"].astype(bool)
    nview = np.where(g, orc["nview"], -1).astype(np.int32)
    tr = {"pw": np.where(g[:, None], orc["pw"], np.nan).astype(np.float32),
          "omega": np.where(g, orc["omega"], np.nan).astype(np.float32),
          "e": np.where(g, orc["e"], np.nan).astype(np.float32), "nview": nview,
          "key": orc["key"].copy()}
    return {"status": 0, "stats": st, "cells": gc, "trace": tr}


@pytest.fixture(scope="module")
def case(oracle_mod):
    rig, _, fr = S.config1()
    orc = oracle_mod.fuse_frame(rig, fr, {})
    return orc, _as_gpu(orc)


def test_identity_passes_and_reports(case):
    from oracle import compare as OC
    orc, gpu = case
    rep = OC.compare(copy.deepcopy(gpu), orc)
    assert rep["n_cells_matched"] + rep["n_cells_excluded"] == rep["n_cells_oracle"]
    assert rep["n_cells_excluded"] <= rep["n_cells_excluded_bound"]
    assert rep["n_cells_matched"] > 100 and rep["n_points_compared"] > 10000


@pytest.mark.parametrize("what", ["count", "rep", "weight", "pos", "key", "rgb"])
def test_planted_difference_fails(case, what):
    from oracle import compare as OC
    orc, gpu = case
    g = copy.deepcopy(gpu)
    flags = orc["cells"]["flags"]
    ok_keys = orc["cells"]["key"][flags == 0]
    j = int(np.flatnonzero(np.isin(g["cells"]["key"], ok_keys))[3])
    if what == "count":
        g["cells"]["count"][j] += 1
    elif what == "rep":
        members = np.flatnonzero(orc["key"] == g["cells"]["key"][j])
        other = [m for m in members if m != g["cells"]["rep"][j]]
        if not other:
            pytest.skip("single-member cell")
        g["cells"]["rep"][j] = other[0]
        order = np.argsort(g["cells"]["rep"], kind="stable")
        g["cells"] = {k: v[order] for k, v in g["cells"].items()}
    elif what == "weight":
        g["cells"]["weight"][j] *= 1.0 + 3e-5
    elif what == "pos":
        g["cells"]["pos"][j, 1] += 3e-5
    elif what == "rgb":
        g["cells"]["rgb"][j, 0] += 0.01
    elif what == "key":
        g["trace"]["key"] = g["trace"]["key"].copy()
        idx = np.flatnonzero(orc["key"] == g["cells"]["key"][j])[0]
        g["trace"]["key"][idx] ^= np.uint64(1)
    with pytest.raises(AssertionError):
        OC.compare(g, orc)
