"""Launch-geometry tuning (fuseflow_get/set_tuning, fuseflow_autotune, and the server's
autotune): every admissible setting of the first four knobs gives bitwise the same cloud,
statistics and trace; the assign step's tile height (8, 16 or 32 rows) regroups each cell's
fixed-point partial sums, so it keeps every integer output, the statistics and the trace
bitwise and the fused values within the parity tolerances (and matches the oracle at every
height); out-of-range settings are refused without effect, and the autotuner keeps a
setting no slower than the one it started from."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import W_ABS, W_FLOOR, compare, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (count_chunks, emit_blocks, prefetch_tiles, programmatic): the extremes of each range and a
# few between, every level of programmatic launch
SETTINGS = [(1, 1, 0, 2), (64, 65536, 1, 0), (2, 152, 304, 1), (7, 999, 1 << 20, 2), (64, 3, 0, 1)]


@pytest.fixture(scope="module")
def ffmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _rows_differ(x, y):
    x, y = x.reshape(len(x), -1), y.reshape(len(y), -1)
    same = (x == y) | (np.isnan(x) & np.isnan(y)) if x.dtype.kind == "f" else x == y
    return np.flatnonzero(~np.all(same, axis=1))


def _same(a, b, with_trace=True):
    assert a["status"] == b["status"]
    assert a["stats"] == b["stats"]
    for k in ("pos", "rgb", "weight", "count", "rep", "key"):
        bad = _rows_differ(a["cells"][k], b["cells"][k])
        detail = [(int(i), a["cells"][k][i].tolist(), b["cells"][k][i].tolist(),
                   hex(int(a["cells"]["key"][i])), int(a["cells"]["count"][i])) for i in bad[:4]]
        assert len(bad) == 0, f"{k}: {len(bad)} rows differ, e.g. {detail}"
    if with_trace:
        for k in a["trace"]:
            assert np.array_equal(a["trace"][k], b["trace"][k], equal_nan=True), k


def _close(a, b, with_trace=True):
    """Integer outputs, statistics and trace bitwise; fused values within the parity
    tolerances (weights 1e-5 relative above W_FLOOR, positions 1e-5 m + 1e-5 relative,
    colour 6e-3)."""
    assert a["status"] == b["status"]
    assert a["stats"] == b["stats"]
    for k in ("count", "rep", "key"):
        assert np.array_equal(a["cells"][k], b["cells"][k]), k
    wa, wb = a["cells"]["weight"].astype(np.float64), b["cells"]["weight"].astype(np.float64)
    big = wa >= W_FLOOR
    assert np.all(np.abs(wb[big] - wa[big]) <= 1e-5 * wa[big]), "weights differ"
    assert np.all(np.abs(wb[~big] - wa[~big]) <= W_ABS), "tiny weights differ"
    pa, pb = a["cells"]["pos"].astype(np.float64), b["cells"]["pos"].astype(np.float64)
    assert np.all(np.abs(pb - pa) <= 1e-5 + 1e-5 * np.abs(pa)), "positions differ"
    ca, cb = a["cells"]["rgb"].astype(np.float64), b["cells"]["rgb"].astype(np.float64)
    assert np.all(np.abs(cb - ca) <= 6e-3), "colours differ"
    if with_trace:
        for k in a["trace"]:
            assert np.array_equal(a["trace"][k], b["trace"][k], equal_nan=True), k


def _cases():
    r1, _, f1 = S.config1()
    r2 = S.tiny_rig(n=3, width=97, height=61, spread_deg=25.0, fx=80.0, fy=78.0)
    f2 = S.random_frame(r2, seed=41, zero_frac=0.03, flying_frac=0.01)
    r3, _, f3 = S.config3(frame=2)
    return [("config1", r1, f1), ("ragged", r2, f2), ("8x1280x720", r3, f3)]


@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("top_k", [0, 3])
def test_every_setting_gives_the_same_result(ffmod, case, top_k):
    name, rig, fr = _cases()[case]
    ff = ffmod.FuseFlow(rig, top_k=top_k)
    try:
        trace = name != "8x1280x720"
        base = run_gpu(ff, fr, torch, with_trace=trace)
        assert base["stats"]["n_cells"] > 0
        for cc, eb, pf, pg in SETTINGS:
            ff.set_tuning(cc, eb, pf, pg)
            assert ff.tuning() == {"count_chunks": cc, "emit_blocks": eb, "prefetch_tiles": pf,
                                   "programmatic": pg, "tile_h": 16}
            _same(base, run_gpu(ff, fr, torch, with_trace=trace), with_trace=trace)
    finally:
        ff.close()


@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("top_k", [0, 3])
def test_tile_heights_keep_integers_and_tolerances(ffmod, case, top_k):
    name, rig, fr = _cases()[case]
    ff = ffmod.FuseFlow(rig, top_k=top_k)
    try:
        trace = name != "8x1280x720"
        base = run_gpu(ff, fr, torch, with_trace=trace)
        tu = ff.tuning()
        for th in (8, 32, 16):
            ff.set_tuning(tu["count_chunks"], tu["emit_blocks"], tu["prefetch_tiles"],
                          tu["programmatic"], th)
            assert ff.tuning()["tile_h"] == th
            got = run_gpu(ff, fr, torch, with_trace=trace)
            if th == 16:
                _same(base, got, with_trace=trace)
            else:
                _close(base, got, with_trace=trace)
    finally:
        ff.close()


@pytest.mark.parametrize("th", [8, 32])
def test_tile_heights_match_the_oracle(ffmod, oracle_mod, parity_log, th):
    rig, _, fr = S.config2(frame=0)
    ff = ffmod.FuseFlow(rig)
    try:
        tu = ff.tuning()
        ff.set_tuning(tu["count_chunks"], tu["emit_blocks"], tu["prefetch_tiles"], tu["programmatic"], th)
        gpu = run_gpu(ff, fr, torch, with_trace=True)
    finally:
        ff.close()
    assert gpu["status"] == ffmod.FUSEFLOW_OK
    orc = oracle_mod.fuse_frame(rig, fr, {})
    rep = compare(gpu, orc)
    parity_log(f"cfg2_4x640x480_tile_h{th}", rep)
    assert rep["excluded_fraction"] < 0.2


def test_a_batch_needs_one_tile_height(ffmod):
    rig, _, fr = S.config1()
    a, b = ffmod.FuseFlow(rig), ffmod.FuseFlow(rig)
    dev = torch.device("cuda")
    try:
        d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.depth]
        c = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.conf]
        r = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.rgb]
        tu = b.tuning()
        b.set_tuning(tu["count_chunks"], tu["emit_blocks"], tu["prefetch_tiles"], tu["programmatic"], 8)
        batch = ffmod.Batch([a, b])
        try:
            assert batch.fuse([(d, c, r), (d, c, r)]) == ffmod.FUSEFLOW_ERR_INVALID_ARG
            b.set_tuning(tu["count_chunks"], tu["emit_blocks"], tu["prefetch_tiles"], tu["programmatic"], 16)
            assert batch.fuse([(d, c, r), (d, c, r)]) == ffmod.FUSEFLOW_OK
            torch.cuda.synchronize()
            # at another common height the batch gives each context's own result bitwise
            for x in (a, b):
                x.set_tuning(tu["count_chunks"], tu["emit_blocks"], tu["prefetch_tiles"], tu["programmatic"], 32)
            alone = run_gpu(a, fr, torch, with_trace=False)
            assert batch.fuse([(d, c, r), (d, c, r)]) == ffmod.FUSEFLOW_OK
            torch.cuda.synchronize()
            for x in (a, b):
                status, st = x.stats(check=False)
                assert status == ffmod.FUSEFLOW_OK and st.as_dict() == alone["stats"]
                cloud = ffmod.fuseflow_get_cloud(x.ctx)
                got = {k: v.cpu().numpy() for k, v in x.cloud_tensors(cloud, int(st.n_cells)).items()}
                for k in ("pos", "rgb", "weight", "count", "rep", "key"):
                    assert np.array_equal(got[k].view(alone["cells"][k].dtype), alone["cells"][k]), k
        finally:
            batch.close()
    finally:
        a.close()
        b.close()


def test_out_of_range_settings_are_refused_without_effect(ffmod):
    rig, _, _ = S.config1()
    ff = ffmod.FuseFlow(rig)
    try:
        before = ff.tuning()
        assert before["count_chunks"] >= 1 and before["emit_blocks"] >= 1
        for cc, eb, pf, pg, th in [(0, 8, 0, 0, 0), (65, 8, 0, 0, 0), (1, 0, 0, 0, 0),
                                   (1, 65537, 0, 0, 0), (1, 8, -1, 0, 0), (1, 8, 0, 3, 0),
                                   (1, 8, 0, -1, 0), (1, 8, 0, 0, 7), (1, 8, 0, 0, 64),
                                   (1, 8, 0, 0, -16)]:
            assert ffmod.fuseflow_set_tuning(ff.ctx, cc, eb, pf, pg, th) == ffmod.FUSEFLOW_ERR_INVALID_ARG
            assert ff.tuning() == before
    finally:
        ff.close()


def test_autotune_keeps_the_result_and_a_setting_no_slower(ffmod):
    rig, _, fr = S.config3(frame=4)
    ff = ffmod.FuseFlow(rig)
    dev = torch.device("cuda")
    try:
        base = run_gpu(ff, fr, torch, with_trace=False)
        d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.depth]
        c = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.conf]
        r = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.rgb]
        # a registered trace is not written while tuning
        sentinel = torch.full((ff.n_pixels,), -7, dtype=torch.int32, device=dev)
        ff.set_trace(nview=sentinel)
        tu, us0, us1 = ff.autotune(d, c, r, reps=5)
        torch.cuda.synchronize()
        assert (sentinel == -7).all()
        ff.clear_trace()
        assert 0 < us1 <= us0
        assert ff.tuning() == tu.as_dict()
        assert 1 <= tu.count_chunks <= 64 and tu.emit_blocks >= 1 and tu.prefetch_tiles >= 0
        assert tu.programmatic in (0, 1, 2) and tu.tile_h in (8, 16, 32)
        check = _same if tu.tile_h == 16 else _close
        check(base, run_gpu(ff, fr, torch, with_trace=False), with_trace=False)
    finally:
        ff.close()


def test_autotune_rejects_bad_reps(ffmod):
    rig, _, fr = S.config1()
    ff = ffmod.FuseFlow(rig)
    dev = torch.device("cuda")
    try:
        d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.depth]
        c = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.conf]
        r = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.rgb]
        for reps in (2, 102):
            with pytest.raises(ffmod.FuseFlowError):
                ff.autotune(d, c, r, reps=reps)
    finally:
        ff.close()


def test_server_autotune_needs_an_idle_rig_and_keeps_results(ffmod):
    from paper_2602_01035_gb300 import serving as SV
    rig, _, fr = S.config1()
    ff = ffmod.FuseFlow(rig)
    try:
        alone = run_gpu(ff, fr, torch, with_trace=False)
    finally:
        ff.close()
    srv = SV.Server(4 << 30)
    try:
        rid = srv.add_rig(rig, n_slots=2)
        pf = SV.pinned_frame(fr)
        hc = SV.HostCloud(srv.rigs[rid]["capacity"])
        srv.submit(rid, pf, hc)
        with pytest.raises(ffmod.FuseFlowError):          # a frame is in flight
            srv.autotune(rid, pf, reps=3)
        srv.drain()
        tu, us0, us1 = srv.autotune(rid, pf, reps=3)
        assert 0 < us1 <= us0
        outs = [SV.HostCloud(srv.rigs[rid]["capacity"]) for _ in range(3)]
        reqs = {srv.submit(rid, pf, h): h for h in outs}
        for req, _, status, st in srv.drain():
            assert status == ffmod.FUSEFLOW_OK
            got = reqs[req].cells(st["n_cells"])
            for k in ("count", "rep", "key"):
                assert np.array_equal(got[k], alone["cells"][k]), k
            if tu.tile_h == 16:
                for k in ("pos", "rgb", "weight"):
                    assert np.array_equal(got[k], alone["cells"][k]), k
            else:
                _close(alone, {"status": alone["status"], "stats": alone["stats"],
                               "cells": {**alone["cells"], **{k: got[k] for k in ("pos", "rgb", "weight")}}},
                       with_trace=False)
    finally:
        srv.close()
