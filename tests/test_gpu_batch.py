"""Batched fusion (fuseflow_batch_*): several contexts fused with every frame kernel launched
once for all of them.  Frames are independent (Sec. I, II.1), so each context's cloud,
statistics and trace must be bitwise those of fuseflow_fuse_frame on the same frame, for
frames of one rig and for rigs of different camera counts and resolutions in one batch,
plain and replayed from a recorded graph."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _dev(fr):
    d = torch.device("cuda")
    return ([torch.from_numpy(np.ascontiguousarray(x)).to(d) for x in fr.depth],
            [torch.from_numpy(np.ascontiguousarray(x)).to(d) for x in fr.conf],
            [torch.from_numpy(np.ascontiguousarray(x)).to(d) for x in fr.rgb])


def _read(F, ff):
    status, st = ff.stats(check=False)
    cloud = F.fuseflow_get_cloud(ff.ctx)
    n = int(st.n_cells)
    out = {k: v.cpu().numpy().copy() for k, v in ff.cloud_tensors(cloud, n).items()}
    return status, st.as_dict(), out


def _plain(F, rig, fr, **params):
    ff = F.FuseFlow(rig, **params)
    try:
        ref = run_gpu(ff, fr, torch, with_trace=False)
    finally:
        ff.close()
    assert ref["status"] == F.FUSEFLOW_OK, ref["stats"]
    return ref


def _same(ref, got):
    status, st, out = got
    assert status == 0
    assert st == ref["stats"]
    for k, v in ref["cells"].items():
        assert np.array_equal(out[k].view(v.dtype), v), k


def _batch_vs_plain(F, rigs_frames, graph=False, **params):
    refs = [_plain(F, rig, fr, **params) for rig, fr in rigs_frames]
    ctxs = [F.FuseFlow(rig, **params) for rig, _ in rigs_frames]
    frames = [_dev(fr) for _, fr in rigs_frames]
    b = F.Batch(ctxs)
    try:
        for _ in range(2):                       # twice: the tables are left clean
            if graph:
                g = b.graph(frames)
                g.launch()
                torch.cuda.synchronize()
                g.close()
            else:
                assert b.fuse(frames) == F.FUSEFLOW_OK
                torch.cuda.synchronize()
            for ref, ff in zip(refs, ctxs):
                _same(ref, _read(F, ff))
    finally:
        b.close()
        for c in ctxs:
            c.close()


def test_four_frames_of_the_benchmark_rig(F):
    cache = {}
    rf = []
    for f in range(4):
        rig, _, fr = S.config3(frame=f, cache=cache)
        rf.append((rig, fr))
    _batch_vs_plain(F, rf)


@pytest.mark.parametrize("graph", [False, True])
def test_mixed_rig_scaling_batch(F, graph):
    """One frame each of the 2, 8, 16 and 32 camera 1024x1024 rigs in one batch."""
    rf = []
    for n in (2, 8, 16, 32):
        rig, _, fr = S.config4(n_cams=n)
        rf.append((rig, fr))
    _batch_vs_plain(F, rf, graph=graph)


def test_eight_ragged_rigs_top3(F):
    """The largest batch: eight rigs of ragged sizes and camera counts, top-3 variant."""
    rf = []
    for k in range(8):
        rig = S.tiny_rig(n=2 + k % 4, width=37 + 23 * k, height=29 + 11 * k, spread_deg=25.0)
        rf.append((rig, S.random_frame(rig, seed=60 + k, zero_frac=0.05, flying_frac=0.01)))
    _batch_vs_plain(F, rf, top_k=3, n_min=4)
    _batch_vs_plain(F, rf, n_min=4)


def test_batch_refusals(F):
    a = F.FuseFlow(S.tiny_rig(n=2, width=32, height=16))
    b = F.FuseFlow(S.tiny_rig(n=2, width=32, height=16, depth_format="f32", depth_scale=1.0))
    c = F.FuseFlow(S.tiny_rig(n=2, width=32, height=16), top_k=3)
    d = F.FuseFlow(S.tiny_rig(n=2, width=32, height=16), screen_edge_rel=0.05)
    try:
        for bad in ([a, b], [a, c], [a, d], [a, a], [a] * 9, []):
            with pytest.raises(F.FuseFlowError):
                F.Batch(bad)
    finally:
        for x in (a, b, c, d):
            x.close()
