"""Eq. 3 confidence producer through the C ABI against the FP64 oracle, pixel by pixel:
the benchmark rig's uint16 depth, float32 depth, ragged image sizes and empty images."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ATOL = 2e-6     # C in [0, 1]; float32 evaluation of a few divisions and a square root


@pytest.fixture(scope="module")
def ffmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _gpu_conf(F, rig, depth, **weights):
    dev = torch.device("cuda")
    ff = F.FuseFlow(rig)
    try:
        d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in depth]
        out = [torch.full(x.shape, -1.0, dtype=torch.float32, device=dev) for x in depth]
        F.fuseflow_confidence(ff.ctx, [t.data_ptr() for t in d], [t.data_ptr() for t in out],
                              torch.cuda.current_stream().cuda_stream, **weights)
        return [t.cpu().numpy() for t in out]
    finally:
        ff.close()


def _check(oracle_mod, rig, depth, got, **weights):
    for i, (d, g) in enumerate(zip(depth, got)):
        ref = oracle_mod.confidence(d, rig.depth_format, rig.depth_scale, **weights)
        np.testing.assert_allclose(g, ref, rtol=0, atol=ATOL, err_msg=f"camera {i}")


def test_confidence_of_the_benchmark_rig(ffmod, oracle_mod):
    rig, _, fr = S.config3(frame=0)
    _check(oracle_mod, rig, fr.depth, _gpu_conf(ffmod, rig, fr.depth))


def test_confidence_of_float_depth_and_other_weights(ffmod, oracle_mod):
    rig, _, fr = S.config1()
    w = {"alpha": 0.7, "beta": 3.0, "gamma": 0.3, "delta": 200.0}
    _check(oracle_mod, rig, fr.depth, _gpu_conf(ffmod, rig, fr.depth, **w), **w)


@pytest.mark.parametrize("w,h,fmt", [(37, 29, "u16"), (5, 300, "u16"), (129, 9, "f32"),
                                     (1, 1, "u16"), (256, 16, "f32")])
def test_confidence_of_ragged_images(ffmod, oracle_mod, w, h, fmt):
    scale = 1.0 if fmt == "f32" else 0.001
    rig = S.tiny_rig(n=2, width=w, height=h, depth_format=fmt, depth_scale=scale)
    fr = S.random_frame(rig, seed=w + h, zero_frac=0.1, flying_frac=0.02 if w > 4 else 0.0)
    depth = [x.copy() for x in fr.depth]
    if fmt == "f32":
        depth[0].flat[::17] = np.nan                   # invalid samples are not used
    _check(oracle_mod, rig, depth, _gpu_conf(ffmod, rig, depth))


def test_confidence_of_an_empty_image_is_zero(ffmod):
    rig = S.tiny_rig(n=2, width=40, height=30)
    depth = [np.zeros((30, 40), np.uint16) for _ in range(2)]
    got = _gpu_conf(ffmod, rig, depth)
    assert all((g == 0).all() for g in got)
