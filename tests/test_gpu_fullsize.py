"""Parity at the largest sizes, in the launch configuration of the benchmark.

* Whole frames against the oracle, every pixel and every cell (the comparison of the other
  parity tests): the 16 and 32 x 1024^2 rig-scaling rigs (16.8 and 33.5 M pixels) and every
  one of the 12 serving rigs (up to 14 x 1920x1080, 29 M pixels).
* A fast variant on the same two largest rigs: per pixel on a sample of rows (every 48th;
  a pixel's Eq. 8-10 values depend only on that pixel and the other views' full depth
  maps), and on the whole frame, properties that hold at any size: every gated in-range
  point is in exactly one cell (the cells' counts are the histogram of the points' keys),
  each cell's representative is a member of largest confidence with the lowest index among
  equals, and the output is ordered by representative.
"""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import W_ABS, W_FLOOR, compare, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROW_STEP = 48
KEY_NONE = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module")
def ffmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _rig(name):
    if name == "32x1024x1024":
        rig, _, fr = S.config4(n_cams=32)
        return rig, fr
    rigs, _ = S.serving_rigs(12, 5999)
    i = max(range(len(rigs)), key=lambda k: rigs[k].n_pixels)
    return rigs[i], S.serving_frame(i)


def _sampled(rig):
    """Global pixel mask of the rows y % ROW_STEP == 0 of every camera."""
    parts = []
    for c in rig.cameras:
        m = np.zeros((c.height, c.width), bool)
        m[::ROW_STEP] = True
        parts.append(m.ravel())
    return np.concatenate(parts)


@pytest.mark.parametrize("name", ["32x1024x1024", "14x1920x1080"])
def test_full_size_rig(ffmod, oracle_mod, name):
    rig, fr = _rig(name)
    assert rig.n_pixels > 2.5e7
    ff = ffmod.FuseFlow(rig)
    try:
        gpu = run_gpu(ff, fr, torch, with_trace=True)
    finally:
        ff.close()
    assert gpu["status"] == ffmod.FUSEFLOW_OK, gpu["stats"]
    st, cells, tr = gpu["stats"], gpu["cells"], gpu["trace"]

    # --- per pixel on the sampled rows
    orc = oracle_mod.fuse_frame(rig, fr, {"row_step": ROW_STEP}, cell_capacity=1 << 21)
    rows = _sampled(rig)
    gated_o = orc["gated"].astype(bool) & rows
    gated_g = (tr["nview"] >= 0) & rows
    assert np.array_equal(gated_g, gated_o), "gated set differs on the sampled rows"
    assert gated_o.sum() > 100000
    dp = np.abs(tr["pw"][gated_o].astype(np.float64) - orc["pw"][gated_o])
    assert np.all(dp <= 1e-5 + 1e-6 * np.abs(orc["pw"][gated_o])), f"world point error {dp.max():.3g} m"
    ok = gated_o & (orc["margin_tie_px"] >= 1e-6) & (orc["min_az"] >= 1e-6)
    assert np.array_equal(tr["nview"][ok], orc["nview"][ok]), "valid-view counts differ"
    de = np.abs(tr["e"][ok].astype(np.float64) - orc["e"][ok])
    assert np.all(de <= 1e-5 + 2.0 ** -23 * orc["e"][ok]), f"exponent error {de.max():.3g}"
    wo, wg = orc["omega"][ok], tr["omega"][ok].astype(np.float64)
    big = wo >= W_FLOOR
    assert np.all(np.abs(wg[big] - wo[big]) <= 1e-5 * wo[big]), "omega differs"
    assert np.all(np.abs(wg[~big] - wo[~big]) <= W_ABS), "tiny omega differs"

    # --- whole frame: every point in exactly one cell, with the cells' counts
    n = int(st["n_cells"])
    assert n == len(cells["key"]) and n > 100000
    keyed = tr["key"] != KEY_NONE
    assert int(keyed.sum()) == st["n_gated"] - st["n_out_of_range"]
    ukeys, ucount = np.unique(tr["key"][keyed], return_counts=True)
    order = np.argsort(cells["key"])
    assert np.array_equal(ukeys, cells["key"][order]), "cell keys differ from the points' keys"
    assert np.array_equal(ucount, cells["count"][order].astype(np.int64)), "cell counts differ"
    assert int(cells["count"].sum()) == int(keyed.sum())

    # --- representatives: largest confidence in the cell, lowest index among equals
    rep = cells["rep"].astype(np.int64)
    assert np.all(np.diff(rep) > 0), "output not ordered by representative"
    assert np.array_equal(tr["key"][rep], cells["key"]), "a representative is not a member"
    conf = np.concatenate([c.ravel() for c in fr.conf]).astype(np.float32)
    g = np.flatnonzero(keyed)
    k = tr["key"][g]
    # members sorted by (key, confidence descending, index ascending): the first of each key
    o = np.lexsort((g, -conf[g], k))
    first = np.ones(len(o), bool)
    first[1:] = k[o][1:] != k[o][:-1]
    best = dict(zip(k[o][first].tolist(), g[o][first].tolist()))
    assert all(best[int(kk)] == int(r) for kk, r in zip(cells["key"], rep)), "representative differs"


def _whole_frame(ffmod, oracle_mod, rig, fr, parity_log, name):
    ff = ffmod.FuseFlow(rig)
    try:
        gpu = run_gpu(ff, fr, torch, with_trace=True)
    finally:
        ff.close()
    assert gpu["status"] == ffmod.FUSEFLOW_OK, gpu["stats"]
    orc = oracle_mod.fuse_frame(rig, fr, {}, cell_capacity=max(1 << 20, rig.n_pixels // 4))
    rep = compare(gpu, orc)
    rep["pixels"] = rig.n_pixels
    parity_log(name, rep)
    return rep


@pytest.mark.parametrize("n_cams", [16, 32])
def test_whole_frame_rig_scaling(ffmod, oracle_mod, parity_log, n_cams):
    rig, _, fr = S.config4(n_cams=n_cams)
    rep = _whole_frame(ffmod, oracle_mod, rig, fr, parity_log, f"cfg4_{n_cams}x1024x1024")
    assert rep["n_cells_oracle"] > 100000
    assert rep["excluded_fraction"] < 0.2


def test_whole_frame_every_serving_rig(ffmod, oracle_mod, parity_log):
    rigs, _ = S.serving_rigs(12, 5999)
    for i, rig in enumerate(rigs):
        c = rig.cameras[0]
        rep = _whole_frame(ffmod, oracle_mod, rig, S.serving_frame(i), parity_log,
                           f"serving_rig{i}_{rig.n_cams}x{c.width}x{c.height}")
        assert rep["n_cells_oracle"] > 1000
        assert rep["excluded_fraction"] < 0.2
