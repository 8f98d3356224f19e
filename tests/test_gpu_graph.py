"""A fuse call recorded as a CUDA graph (fuseflow_graph_*) replays bitwise the same cloud,
statistics and trace as the plain call, for new contents of the same input buffers, and
keeps the launch geometry it was recorded with."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def _cells(ff, cloud):
    status, st = ff.stats(check=False)
    n = int(st.n_cells)
    out = {k: v.cpu().numpy().copy() for k, v in ff.cloud_tensors(cloud, n).items()}
    return status, st.as_dict(), out


def _buffers(fr, dev):
    return ([torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.depth],
            [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.conf],
            [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fr.rgb])


def _refill(bufs, fr):
    for dst, src in zip(bufs[0] + bufs[1] + bufs[2], list(fr.depth) + list(fr.conf) + list(fr.rgb)):
        dst.copy_(torch.from_numpy(np.ascontiguousarray(src)))


@pytest.mark.parametrize("top_k", [0, 3])
def test_replay_matches_the_plain_call_for_new_contents(ffmod, top_k):
    rig = S.tiny_rig(n=4, width=120, height=90, spread_deg=25.0, fx=100.0, fy=98.0)
    frames = [S.random_frame(rig, seed=50 + k, zero_frac=0.03, flying_frac=0.01) for k in range(4)]
    dev = torch.device("cuda")
    ff = ffmod.FuseFlow(rig, top_k=top_k)
    try:
        alone = [run_gpu(ff, fr, torch, with_trace=False) for fr in frames]
        bufs = _buffers(frames[0], dev)
        graph = ff.graph(*bufs)
        try:
            for k, fr in enumerate(frames + frames[::-1]):
                _refill(bufs, fr)
                status, st, out = _cells(ff, graph.launch())
                ref = alone[k if k < len(frames) else 2 * len(frames) - 1 - k]
                assert status == ref["status"] and st == ref["stats"]
                for key in ("pos", "rgb", "weight"):
                    assert np.array_equal(out[key], ref["cells"][key]), key
                for key, dt in (("count", np.uint32), ("rep", np.uint32), ("key", np.uint64)):
                    assert np.array_equal(out[key].view(dt), ref["cells"][key]), key
        finally:
            graph.close()
    finally:
        ff.close()


def test_replay_keeps_its_geometry_and_trace(ffmod):
    rig, _, fr = S.config1()
    dev = torch.device("cuda")
    ff = ffmod.FuseFlow(rig)
    try:
        ref = run_gpu(ff, fr, torch, with_trace=True)
        bufs = _buffers(fr, dev)
        npx = ff.n_pixels
        nview = torch.full((npx,), -7, dtype=torch.int32, device=dev)
        key = torch.zeros((npx,), dtype=torch.int64, device=dev)
        ff.set_trace(nview=nview, key=key)
        ff.set_tuning(1, 1, 0, 2)
        graph = ff.graph(*bufs)
        ff.clear_trace()
        ff.set_tuning(64, 4096, 1, 0)       # later changes do not reach the recorded call
        try:
            status, st, out = _cells(ff, graph.launch())
            torch.cuda.synchronize()
            assert st == ref["stats"]
            assert np.array_equal(out["pos"], ref["cells"]["pos"])
            assert np.array_equal(nview.cpu().numpy(), ref["trace"]["nview"])
            assert np.array_equal(key.cpu().numpy().view(np.uint64), ref["trace"]["key"])
        finally:
            graph.close()
    finally:
        ff.close()
