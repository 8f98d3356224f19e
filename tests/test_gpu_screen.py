"""The depth screen D^r of Eq. 8 on the GPU against the oracle: screened images bit for bit
(a selection: every decision is taken in float32 on both sides), and whole frames fused with
a screen set, element by element under the parity rules of test_gpu_parity."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import compare, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SETTINGS = [{}, {"screen_edge_rel": 0.03}, {"screen_min_m": 1.0, "screen_max_m": 3.5},
            {"screen_min_m": 0.8, "screen_max_m": 4.0, "screen_edge_rel": 0.01}]


@pytest.fixture(scope="module")
def ffmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _rigs():
    r1, _, f1 = S.config1()
    d1 = [x.copy() for x in f1.depth]
    d1[0].flat[::13] = np.nan
    d1[1].flat[5::29] = -2.0
    f1 = S.Frame(d1, f1.conf, f1.rgb, f1.z_true, f1.surface_id)
    r2 = S.tiny_rig(n=3, width=37, height=29, spread_deg=25.0, fx=40.0, fy=40.0)
    f2 = S.random_frame(r2, seed=81, zero_frac=0.05, flying_frac=0.03)
    r3 = S.tiny_rig(n=2, width=1, height=1)
    f3 = S.random_frame(r3, seed=82)
    r4, _, f4 = S.config3(frame=1)
    return [(r1, f1), (r2, f2), (r3, f3), (r4, f4)]


@pytest.mark.parametrize("case", range(4))
def test_screened_images_match_the_oracle(ffmod, oracle_mod, case):
    rig, fr = _rigs()[case]
    dev = torch.device("cuda")
    src = [torch.from_numpy(np.ascontiguousarray(d)).to(dev) for d in fr.depth]
    for screen in SETTINGS:
        ff = ffmod.FuseFlow(rig, **screen)
        try:
            out = [torch.full_like(t, 7) for t in src]
            ffmod.fuseflow_screen_depth(ff.ctx, [t.data_ptr() for t in src],
                                        [t.data_ptr() for t in out],
                                        torch.cuda.current_stream().cuda_stream)
            for d, o in zip(fr.depth, out):
                ref = oracle_mod.screen_depth(d, rig.depth_format, rig.depth_scale, **screen)
                np.testing.assert_array_equal(o.cpu().numpy(), ref, err_msg=str(screen))
        finally:
            ff.close()


@pytest.mark.parametrize("case,screen,top_k", [(0, SETTINGS[3], 0), (1, SETTINGS[1], 0),
                                               (1, SETTINGS[3], 3), (3, SETTINGS[1], 0)])
def test_frames_with_a_screen_match_the_oracle(ffmod, oracle_mod, case, screen, top_k):
    rig, fr = _rigs()[case]
    params = dict(screen, top_k=top_k)
    ff = ffmod.FuseFlow(rig, **params)
    try:
        gpu = run_gpu(ff, fr, torch, with_trace=True)     # the trace places boundary points
        assert gpu["status"] == ffmod.FUSEFLOW_OK, gpu["stats"]
    finally:
        ff.close()
    orc = oracle_mod.fuse_frame(rig, fr, params)
    compare(gpu, orc, oracle_mod)
    plain = oracle_mod.fuse_frame(rig, fr, {"top_k": top_k})
    assert orc["stats"]["n_valid"] < plain["stats"]["n_valid"]         # the screen acts


def test_fusing_with_a_screen_equals_fusing_screened_images(ffmod):
    rig, fr = _rigs()[1]
    screen = SETTINGS[3]
    dev = torch.device("cuda")
    ff = ffmod.FuseFlow(rig, **screen)
    plain = ffmod.FuseFlow(rig)
    try:
        a = run_gpu(ff, fr, torch, with_trace=True)
        src = [torch.from_numpy(np.ascontiguousarray(d)).to(dev) for d in fr.depth]
        dr = [torch.empty_like(t) for t in src]
        ffmod.fuseflow_screen_depth(ff.ctx, [t.data_ptr() for t in src], [t.data_ptr() for t in dr],
                                    torch.cuda.current_stream().cuda_stream)
        fr2 = S.Frame([t.cpu().numpy() for t in dr], fr.conf, fr.rgb, fr.z_true, fr.surface_id)
        b = run_gpu(plain, fr2, torch, with_trace=True)
        assert a["stats"] == b["stats"]
        for k in a["cells"]:
            assert np.array_equal(a["cells"][k], b["cells"][k]), k
        for k in a["trace"]:
            assert np.array_equal(a["trace"][k], b["trace"][k], equal_nan=True), k
    finally:
        ff.close()
        plain.close()
