"""Eq. 12 (multi-camera depth consistency error) through the C ABI against the FP64 oracle.

Both sides evaluate the same float32 point sets (the fused cloud of the GPU path, and the
gated world points of the trace for the point-wise "No SA" ablation) on the same depth
maps.  Points whose projection lies within 5e-4 px of a half-pixel tie in some camera may
pick another pixel in float32 and are compared only through the aggregate bound."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIE_PX = 5e-4      # float32 projections of these points are within ~1.5e-4 px
ATOL_M = 1e-5          # float32 camera coordinates of points a few metres away: ~1e-6 m


@pytest.fixture(scope="module")
def ffmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _gpu_mc(F, ff, fr, pts):
    dev = torch.device("cuda")
    depth = [torch.from_numpy(np.ascontiguousarray(d)).to(dev) for d in fr.depth]
    p = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float32)).to(dev)
    n = p.shape[0]
    err = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    nvis = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    mc, used = F.fuseflow_mc_error(ff.ctx, p.data_ptr(), n, [d.data_ptr() for d in depth],
                                   err.data_ptr(), nvis.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    return mc, used, err[:n].cpu().numpy(), nvis[:n].cpu().numpy()


def _compare(F, oracle_mod, rig, fr, ff, pts):
    mc, used, err, nvis = _gpu_mc(F, ff, fr, pts)
    orc = oracle_mod.mc_error(rig, fr.depth, pts.astype(np.float64))
    ok = orc["tie_px"] >= TIE_PX
    assert ok.mean() > 0.98
    np.testing.assert_array_equal(nvis[ok], orc["nvis"][ok])
    seen = ok & (orc["nvis"] > 0)
    np.testing.assert_allclose(err[seen], orc["err_m"][seen], rtol=1e-5, atol=ATOL_M)
    assert np.isnan(err[ok & (orc["nvis"] == 0)]).all()
    # the aggregate: identical sets of points apart from the few near ties
    n_diff = int((~ok).sum())
    assert abs(used - orc["n_used"]) <= n_diff
    bound = ATOL_M + n_diff / max(orc["n_used"], 1) * 2 * np.nanmax(orc["err_m"])
    assert abs(mc - orc["mc_m"]) <= bound
    return mc, orc["mc_m"]


def test_mc_error_of_the_fused_cloud(ffmod, oracle_mod):
    for f in (0, 9):
        rig, _, fr = S.config2(frame=f)
        ff = ffmod.FuseFlow(rig)
        try:
            out = run_gpu(ff, fr, torch, with_trace=False)
            pos = out["cells"]["pos"]
            assert len(pos) > 5000
            mc, mc_orc = _compare(ffmod, oracle_mod, rig, fr, ff, pos)
            assert 0.0 < mc < 0.05
        finally:
            ff.close()


def test_mc_error_of_the_pointwise_cloud(ffmod, oracle_mod):
    """Table II "No SA": every gated point is its own output point."""
    rig, _, fr = S.config1()
    ff = ffmod.FuseFlow(rig)
    try:
        out = run_gpu(ff, fr, torch, with_trace=True)
        pw = out["trace"]["pw"]
        pts = pw[np.isfinite(pw[:, 0])]
        assert len(pts) > 10000
        _compare(ffmod, oracle_mod, rig, fr, ff, pts)
    finally:
        ff.close()


def test_mc_error_edge_cases(ffmod, oracle_mod):
    rig, _, fr = S.config1()
    ff = ffmod.FuseFlow(rig)
    try:
        mc, used, _, _ = _gpu_mc(ffmod, ff, fr, np.zeros((0, 3), np.float32))
        assert used == 0 and np.isnan(mc)
        far = np.array([[500.0, 0.0, 0.0], [0.0, 0.0, 50.0]], np.float32)   # seen by no camera
        mc, used, err, nvis = _gpu_mc(ffmod, ff, fr, far)
        assert used == 0 and (nvis == 0).all() and np.isnan(err).all()
    finally:
        ff.close()
