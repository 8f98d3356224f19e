"""Point-wise fusion, Table II's "No SA" ablation (fuseflow_fuse_points): every gated pixel
is an output point with its own joint weight.  Against the FP64 oracle's per-pixel values
(Eq. 8 world point, Eq. 10 weight; half-pixel ties excluded from the weight, as in the
other parity tests), and against the traced values of the fused path."""
import numpy as np
import pytest

from oracle.compare import W_ABS, W_FLOOR, point_masks
from paper_2602_01035_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _points(F, rig, fr, **params):
    dev = torch.device("cuda")
    d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.depth]
    c = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.conf]
    r = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.rgb]
    npx = rig.n_pixels
    pos = torch.zeros((npx, 3), dtype=torch.float32, device=dev)
    w = torch.full((npx,), -1.0, dtype=torch.float32, device=dev)
    col = torch.zeros((npx, 3), dtype=torch.uint8, device=dev)
    ff = F.FuseFlow(rig, **params)
    try:
        nv, ng = F.fuseflow_fuse_points(ff.ctx, [t.data_ptr() for t in d], [t.data_ptr() for t in c],
                                        [t.data_ptr() for t in r], pos.data_ptr(), w.data_ptr(),
                                        col.data_ptr(), torch.cuda.current_stream().cuda_stream)
    finally:
        ff.close()
    return nv, ng, pos.cpu().numpy(), w.cpu().numpy(), col.cpu().numpy()


@pytest.mark.parametrize("case", ["cfg2", "ragged_f32", "ragged_u16", "no_conf"])
def test_points_match_the_oracle(F, oracle_mod, case):
    params = {}
    if case == "cfg2":
        rig, _, fr = S.config2(frame=1)
    elif case == "ragged_f32":
        rig = S.tiny_rig(n=3, width=45, height=31, depth_format="f32", depth_scale=1.0, spread_deg=25.0)
        fr = S.random_frame(rig, seed=71, zero_frac=0.05)
    elif case == "ragged_u16":
        rig = S.tiny_rig(n=4, width=70, height=45, spread_deg=25.0)
        fr = S.random_frame(rig, seed=72, zero_frac=0.05, flying_frac=0.01)
    else:
        rig, _, fr = S.config2(frame=2)
        params = {"use_conf": 0}
    nv, ng, pos, w, col = _points(F, rig, fr, **params)
    orc = oracle_mod.fuse_frame(rig, fr, params)
    gated = orc["gated"].astype(bool)
    assert nv == orc["stats"]["n_valid"] and ng == orc["stats"]["n_gated"] == gated.sum()
    assert np.all(np.isnan(pos[~gated])) and np.all(w[~gated] == 0.0)
    assert np.all(np.isfinite(pos[gated]))
    dp = np.abs(pos[gated].astype(np.float64) - orc["pw"][gated])
    assert np.all(dp <= 1e-5 + 1e-6 * np.abs(orc["pw"][gated])), dp.max()
    _, _, tie = point_masks(orc)
    ok = gated & ~tie
    wo, wg = orc["omega"][ok], w[ok].astype(np.float64)
    big = wo >= W_FLOOR
    assert np.all(np.abs(wg[big] - wo[big]) <= 1e-5 * wo[big])
    assert np.all(np.abs(wg[~big] - wo[~big]) <= W_ABS)
    np.testing.assert_array_equal(col, np.concatenate([x.reshape(-1, 3) for x in fr.rgb]))
