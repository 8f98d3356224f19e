"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Sizes span several 32x16 tiles and ragged tails; the full-size cases use the rig of the
benchmark (8 x 1280x720) and the 1024x1024 rigs, with the same launch configuration.
"""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import compare, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _fuse_and_compare(ffmod, oracle_mod, rig, fr, params=None, trace=True):
    params = dict(params or {})
    ff = ffmod.FuseFlow(rig, **params)
    try:
        gpu = run_gpu(ff, fr, torch, with_trace=trace)
        assert gpu["status"] == ffmod.FUSEFLOW_OK, gpu["stats"]
        nb = ff.neighbours()
    finally:
        ff.close()
    oparams = {k: v for k, v in params.items() if k not in ("max_cells",)}
    orc = oracle_mod.fuse_frame(rig, fr, oparams)
    np.testing.assert_array_equal(nb, oracle_mod.neighbours(rig, params.get("k_views", 4)))
    return compare(gpu, orc, oracle_mod), gpu, orc


def test_config1_float_depth(ffmod, oracle_mod, parity_log):
    rig, _, fr = S.config1()
    rep, gpu, orc = _fuse_and_compare(ffmod, oracle_mod, rig, fr)
    parity_log("cfg1_2x160x120", rep)
    assert rep["n_cells_matched"] > 150
    assert rep["n_points_compared"] > 10000


@pytest.mark.parametrize("n,w,h,fmt,k,zero,seed", [
    (1, 37, 29, "u16", 4, 0.05, 1),
    (2, 33, 17, "f32", 2, 0.0, 2),
    (3, 70, 45, "u16", 3, 0.1, 3),
    (4, 100, 61, "u16", 4, 0.02, 4),
    (5, 64, 48, "f32", 9, 0.3, 5),
    (2, 1, 1, "u16", 4, 0.0, 6),
    (3, 5, 300, "u16", 4, 0.0, 7),
])
def test_tiny_and_ragged(ffmod, oracle_mod, n, w, h, fmt, k, zero, seed):
    scale = 1.0 if fmt == "f32" else 0.001
    rig = S.tiny_rig(n=n, width=w, height=h, depth_format=fmt, depth_scale=scale, spread_deg=25.0,
                     fx=max(w, 8) * 0.9, fy=max(w, 8) * 0.85)
    fr = S.random_frame(rig, seed=seed, zero_frac=zero, flying_frac=0.01 if w > 4 else 0.0)
    _fuse_and_compare(ffmod, oracle_mod, rig, fr, {"k_views": k, "n_min": 4})


def test_config2_frames(ffmod, oracle_mod, parity_log):
    for f in (0, 17):
        rig, _, fr = S.config2(frame=f)
        rep, _, _ = _fuse_and_compare(ffmod, oracle_mod, rig, fr)
        parity_log(f"cfg2_4x640x480_frame{f}", rep)
        assert rep["n_cells_matched"] > 5000


def test_config3_full_frame(ffmod, oracle_mod, parity_log):
    """8 x 1280x720 uint16: the benchmark's rig and launch configuration."""
    rig, _, fr = S.config3(frame=0)
    rep, gpu, orc = _fuse_and_compare(ffmod, oracle_mod, rig, fr)
    parity_log("cfg3_8x1280x720_frame0", rep)
    assert rep["n_cells_oracle"] > 150000 and rep["excluded_fraction"] < 0.2
    lv = (gpu["cells"]["key"] >> np.uint64(60)).astype(int)
    assert len(np.unique(lv)) >= 3          # the adaptive partition uses several levels
    print(rep)


@pytest.mark.parametrize("n_cams", [2, 8])
def test_config4_rigs(ffmod, oracle_mod, parity_log, n_cams):
    rig, _, fr = S.config4(n_cams=n_cams)
    rep, _, _ = _fuse_and_compare(ffmod, oracle_mod, rig, fr)
    parity_log(f"cfg4_{n_cams}x1024x1024", rep)
    assert rep["n_cells_matched"] > 1000


def test_ablation_switches(ffmod, oracle_mod):
    rig, _, fr = S.config2(frame=3)
    _fuse_and_compare(ffmod, oracle_mod, rig, fr, {"use_conf": 0})
    _fuse_and_compare(ffmod, oracle_mod, rig, fr, {"use_consistency": 0})


def test_sigma_and_levels(ffmod, oracle_mod):
    rig, _, fr = S.config2(frame=5)
    _fuse_and_compare(ffmod, oracle_mod, rig, fr,
                      {"sigma_m": 0.005, "n_min": 8, "max_level": 6, "coarse_cell_m": 0.5})


def test_sparse_tiles_overflow_the_shared_accumulators(ffmod, oracle_mod):
    """Depths scattered over 0.5-40 m put nearly every pixel of a 32x16 tile in a cell of
    its own, past the 256 shared accumulators of a tile: those members file alone."""
    rig = S.tiny_rig(n=3, width=96, height=48)
    rng = np.random.default_rng(11)
    z = [rng.integers(500, 40000, size=(48, 96), dtype=np.uint16) for _ in range(3)]
    c = [rng.uniform(0.61, 1.0, size=(48, 96)).astype(np.float32) for _ in range(3)]
    col = [rng.integers(0, 256, size=(48, 96, 3), dtype=np.uint8) for _ in range(3)]
    rep, gpu, _ = _fuse_and_compare(ffmod, oracle_mod, rig, S.Frame(z, c, col),
                                    {"max_level": 6, "n_min": 1})
    assert gpu["stats"]["n_cells"] > 0.9 * gpu["stats"]["n_gated"]
    assert rep["n_cells_matched"] > 10000


def test_overflowing_tiles_are_bitwise_reproducible(ffmod, oracle_mod):
    """Tiles with more than 256 distinct cells, many of them with two members of unequal
    weight: which cells of such a tile would get a shared accumulator must not depend on
    the order of the threads' insertions, so every run gives the same bits."""
    rig = S.tiny_rig(n=3, width=128, height=64, fx=80.0, fy=80.0)
    rng = np.random.default_rng(12)
    z, c, col = [], [], []
    for _ in range(3):
        d = rng.integers(500, 40000, size=(64, 128)).astype(np.uint16)
        paired = (np.arange(64) % 3) != 0
        d[paired, 1::2] = d[paired, 0::2]            # adjacent pixels at one depth: one cell
        z.append(d)
        c.append(rng.uniform(0.61, 1.0, size=(64, 128)).astype(np.float32))
        col.append(rng.integers(0, 256, size=(64, 128, 3), dtype=np.uint8))
    fr = S.Frame(z, c, col)
    params = {"max_level": 0}
    rep, ref, _ = _fuse_and_compare(ffmod, oracle_mod, rig, fr, params)
    assert rep["n_cells_matched"] > 5000
    assert (ref["cells"]["count"] >= 2).sum() > 2000
    for trial in range(3):
        ff = ffmod.FuseFlow(rig, **params)
        try:
            if trial == 1:
                ff.set_tuning(1, 1, 0, 2 - ff.tuning()["programmatic"])
            for _ in range(3):
                o = run_gpu(ff, fr, torch, with_trace=True)
                assert o["stats"] == ref["stats"]
                for k in ref["cells"]:
                    assert np.array_equal(o["cells"][k], ref["cells"][k], equal_nan=True), k
                for k in ref["trace"]:
                    assert np.array_equal(o["trace"][k], ref["trace"][k], equal_nan=True), k
        finally:
            ff.close()


@pytest.mark.parametrize("k", [1, 3, 7])
def test_top_k_variant(ffmod, oracle_mod, k):
    """Sec. II.5(2)a: each cell fuses only its k most confident members; consistency and
    weights are computed for those alone."""
    rig, _, fr = S.config2(frame=4)
    rep, gpu, orc = _fuse_and_compare(ffmod, oracle_mod, rig, fr, {"top_k": k})
    assert rep["n_cells_matched"] > 5000


@pytest.mark.parametrize("n,w,h,fmt,seed", [(3, 70, 45, "u16", 51), (2, 33, 17, "f32", 52),
                                            (4, 100, 61, "u16", 53)])
def test_top_k_variant_ragged(ffmod, oracle_mod, n, w, h, fmt, seed):
    scale = 1.0 if fmt == "f32" else 0.001
    rig = S.tiny_rig(n=n, width=w, height=h, depth_format=fmt, depth_scale=scale, spread_deg=25.0)
    fr = S.random_frame(rig, seed=seed, zero_frac=0.05, flying_frac=0.01)
    _fuse_and_compare(ffmod, oracle_mod, rig, fr, {"top_k": 3, "n_min": 4})


def test_top_k_variant_benchmark_rig(ffmod, oracle_mod, parity_log):
    rig, _, fr = S.config3(frame=0)
    rep, _, _ = _fuse_and_compare(ffmod, oracle_mod, rig, fr, {"top_k": 3})
    parity_log("cfg3_8x1280x720_frame0_top3", rep)
    assert rep["n_cells_matched"] > 100000


def test_empty_and_all_gated_out(ffmod, oracle_mod):
    rig = S.tiny_rig(n=2, width=40, height=30)
    z = [np.zeros((30, 40), np.uint16) for _ in range(2)]
    c = [np.full((30, 40), 0.9, np.float32) for _ in range(2)]
    col = [np.zeros((30, 40, 3), np.uint8) for _ in range(2)]
    rep, gpu, _ = _fuse_and_compare(ffmod, oracle_mod, rig, S.Frame(z, c, col))
    assert gpu["stats"]["n_cells"] == 0 and gpu["stats"]["n_valid"] == 0
    z = [np.full((30, 40), 2000, np.uint16) for _ in range(2)]
    c = [np.full((30, 40), 0.6, np.float32) for _ in range(2)]      # C == tau is rejected
    rep, gpu, _ = _fuse_and_compare(ffmod, oracle_mod, rig, S.Frame(z, c, col))
    assert gpu["stats"]["n_valid"] == 2400 and gpu["stats"]["n_gated"] == 0


def test_invalid_float_depth_values(ffmod, oracle_mod):
    rig = S.tiny_rig(n=2, width=48, height=32, depth_format="f32", depth_scale=1.0)
    fr = S.random_frame(rig, seed=8)
    d = [x.copy() for x in fr.depth]
    d[0][0, :5] = [np.nan, np.inf, -np.inf, -1.0, 0.0]
    d[1][3, 3] = np.nan
    _fuse_and_compare(ffmod, oracle_mod, rig, S.Frame(d, fr.conf, fr.rgb))


def _patch_frame(fr, y0=40, x0=60, h=12, w=12):
    """The frame with every depth sample zeroed except one patch of camera 0."""
    depth = []
    for i, d in enumerate(fr.depth):
        z = np.zeros_like(d)
        if i == 0:
            z[y0:y0 + h, x0:x0 + w] = d[y0:y0 + h, x0:x0 + w]
        depth.append(z)
    return S.Frame(depth, fr.conf, fr.rgb)


def test_capacity_overflow_reports_and_recovers(ffmod, oracle_mod):
    """A frame with more cells than max_cells reports CAPACITY; the same context then fuses
    a frame that fits exactly as the oracle does (the overflowed frame left no state behind),
    and a context with room fuses the large frame."""
    rig, _, fr = S.config1()
    small = _patch_frame(fr)
    ff = ffmod.FuseFlow(rig, max_cells=50)
    try:
        gpu = run_gpu(ff, fr, torch, with_trace=False)
        assert gpu["status"] == ffmod.FUSEFLOW_ERR_CAPACITY
        assert gpu["stats"]["n_cells"] == 50
        for _ in range(2):                    # twice: the recovered frame leaves none either
            after = run_gpu(ff, small, torch, with_trace=True)
            assert after["status"] == ffmod.FUSEFLOW_OK, after["stats"]
            rep = compare(after, oracle_mod.fuse_frame(rig, small, {}), oracle_mod)
            assert 0 < rep["n_cells_oracle"] <= 50
            assert rep["n_cells_matched"] + rep["n_cells_excluded"] == rep["n_cells_oracle"]
    finally:
        ff.close()
    rep, _, _ = _fuse_and_compare(ffmod, oracle_mod, rig, fr)
    assert rep["n_cells_matched"] > 150


def test_deterministic_and_stateless(ffmod):
    rig, _, fa = S.config2(frame=0)
    _, _, fb = S.config2(frame=40)
    ff = ffmod.FuseFlow(rig)
    try:
        a1 = run_gpu(ff, fa, torch, with_trace=False)
        a2 = run_gpu(ff, fa, torch, with_trace=False)
        run_gpu(ff, fb, torch, with_trace=False)
        a3 = run_gpu(ff, fa, torch, with_trace=False)
    finally:
        ff.close()
    for other in (a2, a3):
        assert other["stats"] == a1["stats"]
        for k in a1["cells"]:
            assert np.array_equal(a1["cells"][k], other["cells"][k]), k


def test_host_entry_point_matches_device_path(ffmod):
    import ctypes as C
    rig, _, fr = S.config2(frame=2)
    ff = ffmod.FuseFlow(rig)
    try:
        dev = run_gpu(ff, fr, torch, with_trace=False)
        cap = ff.capacity
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        d = [pin(x) for x in fr.depth]
        c = [pin(x) for x in fr.conf]
        r = [pin(x) for x in fr.rgb]
        outs = {"pos": torch.empty((cap, 3), dtype=torch.float32).pin_memory(),
                "rgb": torch.empty((cap, 3), dtype=torch.float32).pin_memory(),
                "weight": torch.empty(cap, dtype=torch.float32).pin_memory(),
                "count": torch.empty(cap, dtype=torch.int32).pin_memory(),
                "rep": torch.empty(cap, dtype=torch.int32).pin_memory(),
                "key": torch.empty(cap, dtype=torch.int64).pin_memory()}
        status, st = ffmod.fuseflow_fuse_frame_host(
            ff.ctx, [t.data_ptr() for t in d], [t.data_ptr() for t in c], [t.data_ptr() for t in r],
            outs["pos"].data_ptr(), outs["rgb"].data_ptr(), outs["weight"].data_ptr(),
            outs["count"].data_ptr(), outs["rep"].data_ptr(), outs["key"].data_ptr(),
            torch.cuda.current_stream().cuda_stream)
        assert status == ffmod.FUSEFLOW_OK
        n = st.n_cells
        assert n == dev["stats"]["n_cells"]
        assert np.array_equal(outs["pos"][:n].numpy(), dev["cells"]["pos"])
        assert np.array_equal(outs["weight"][:n].numpy(), dev["cells"]["weight"])
        assert np.array_equal(outs["key"][:n].numpy().view(np.uint64), dev["cells"]["key"])
        assert np.array_equal(outs["rep"][:n].numpy().view(np.uint32), dev["cells"]["rep"])
    finally:
        ff.close()
