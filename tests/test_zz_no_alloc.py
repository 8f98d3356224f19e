"""The allocation-free entry point against the context-based one.

fuseflow_fuse_frame_static serves callers that cannot allocate device memory while they
run (an application whose memory pool owns the GPU budget, a real-time loop that cannot
absorb cudaMalloc's device-wide synchronisation).  It keeps its scratch in a static device
array; this test fuses two frames in a row through it and checks each against
fuseflow_fuse_frame on the same input, with the tolerances of the other parity tests.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _outputs(cap, dev):
    return {"pos": torch.full((cap, 3), float("nan"), device=dev),
            "rgb": torch.full((cap, 3), float("nan"), device=dev),
            "weight": torch.full((cap,), float("nan"), device=dev),
            "count": torch.zeros(cap, dtype=torch.int32, device=dev),
            "rep": torch.zeros(cap, dtype=torch.int32, device=dev),
            "key": torch.zeros(cap, dtype=torch.int64, device=dev),
            "stats": torch.zeros(64, dtype=torch.uint8, device=dev)}


def _check_same(ref_cells, ref_stats, got, n):
    assert n == ref_stats["n_cells"]
    np.testing.assert_array_equal(got["key"][:n].cpu().numpy().view(np.uint64), ref_cells["key"])
    np.testing.assert_array_equal(got["count"][:n].cpu().numpy().view(np.uint32), ref_cells["count"])
    np.testing.assert_array_equal(got["rep"][:n].cpu().numpy().view(np.uint32), ref_cells["rep"])
    w_ref = ref_cells["weight"].astype(np.float64)
    w = got["weight"][:n].cpu().numpy().astype(np.float64)
    big = w_ref >= 1e-30
    assert np.all(np.abs(w[big] - w_ref[big]) <= 1e-5 * w_ref[big])
    assert np.all(np.abs(w[~big] - w_ref[~big]) <= 1e-35)
    p_ref = ref_cells["pos"].astype(np.float64)
    p = got["pos"][:n].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(p - p_ref) <= 1e-5 + 1e-5 * np.abs(p_ref))
    c = got["rgb"][:n].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(c - ref_cells["rgb"]) <= 6e-3)


def _static_call(F, rig, fr, cap, dev, stream, **params):
    """One fuseflow_fuse_frame_static call on device copies of `fr`; returns (status, stats,
    outputs) after the stream has finished."""
    p = F.fuseflow_default_params(depth_format=F.FUSEFLOW_DEPTH_U16, depth_scale=rig.depth_scale,
                                  max_cells=cap, **params)
    intr, extr = F.rig_arrays(rig)
    d = [torch.from_numpy(x).to(dev) for x in fr.depth]
    c = [torch.from_numpy(x).to(dev) for x in fr.conf]
    r = [torch.from_numpy(x).to(dev) for x in fr.rgb]
    out = _outputs(cap, dev)
    st = F.fuseflow_fuse_frame_static(
        intr, extr, rig.n_cams, p, [t.data_ptr() for t in d], [t.data_ptr() for t in c],
        [t.data_ptr() for t in r], out["pos"].data_ptr(), out["rgb"].data_ptr(),
        out["weight"].data_ptr(), out["count"].data_ptr(), out["rep"].data_ptr(),
        out["key"].data_ptr(), out["stats"].data_ptr(), stream)
    torch.cuda.synchronize()
    raw = out["stats"].cpu().numpy().tobytes()[:ctypes.sizeof(F.fuseflow_stats)]
    return st, F.fuseflow_stats.from_buffer_copy(raw), out


def _context_reference(F, rig, fr, cap, **params):
    from parity import run_gpu
    ff = F.FuseFlow(rig, max_cells=cap, **params)
    try:
        ref = run_gpu(ff, fr, torch, with_trace=False)
    finally:
        ff.close()
    assert ref["status"] == F.FUSEFLOW_OK and ref["stats"]["n_cells"] > 100
    return ref


def test_static_entry_point_after_a_larger_rig_and_an_overflow():
    """Three calls in a row share the array: a frame of a larger rig (4 x 320x240), a frame
    of that rig whose scattered depths need more partial records and cells than the array
    holds (reported in stats->error), then a frame of a smaller rig, which must match the
    context path as if the array were fresh."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow as F
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cap = 32768
    big = S.tiny_rig(n=4, width=320, height=240, spread_deg=30.0)
    fr_big = S.random_frame(big, seed=33, flying_frac=0.01)
    ref = _context_reference(F, big, fr_big, cap)
    st, stats, out = _static_call(F, big, fr_big, cap, dev, stream)
    assert st == F.FUSEFLOW_OK and stats.error == 0
    _check_same(ref["cells"], ref["stats"], out, int(stats.n_cells))
    rng = np.random.default_rng(34)
    scattered = S.Frame([rng.integers(500, 40000, size=(240, 320), dtype=np.uint16) for _ in range(4)],
                        [rng.uniform(0.61, 1.0, size=(240, 320)).astype(np.float32) for _ in range(4)],
                        [rng.integers(0, 256, size=(240, 320, 3), dtype=np.uint8) for _ in range(4)])
    st, stats, _ = _static_call(F, big, scattered, cap, dev, stream, max_level=6, n_min=1)
    assert st == F.FUSEFLOW_OK                      # asynchronous: the error is in the stats
    assert stats.error != 0 and stats.n_cells == cap
    small = S.tiny_rig(n=3, width=160, height=120, spread_deg=30.0)
    fr_small = S.random_frame(small, seed=35, flying_frac=0.01)
    ref = _context_reference(F, small, fr_small, 8192)
    for _ in range(2):
        st, stats, out = _static_call(F, small, fr_small, 8192, dev, stream)
        assert st == F.FUSEFLOW_OK and stats.error == 0
        for k in ("n_valid", "n_gated", "n_out_of_range"):
            assert getattr(stats, k) == ref["stats"][k]
        _check_same(ref["cells"], ref["stats"], out, int(stats.n_cells))


def test_static_entry_point_refuses_stream_capture():
    """The call stages rig constants through host arrays that the next call overwrites, so
    it refuses to be recorded into a CUDA graph and enqueues nothing."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow as F
    rig = S.tiny_rig(n=2, width=64, height=48)
    fr = S.random_frame(rig, seed=36)
    dev = torch.device("cuda")
    d = [torch.from_numpy(x).to(dev) for x in fr.depth]
    c = [torch.from_numpy(x).to(dev) for x in fr.conf]
    r = [torch.from_numpy(x).to(dev) for x in fr.rgb]
    out = _outputs(1024, dev)
    p = F.fuseflow_default_params(max_cells=1024)
    intr, extr = F.rig_arrays(rig)
    x = torch.zeros(16, device=dev)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        x.add_(1.0)
        st = F.fuseflow_fuse_frame_static(
            intr, extr, 2, p, [t.data_ptr() for t in d], [t.data_ptr() for t in c],
            [t.data_ptr() for t in r], out["pos"].data_ptr(), out["rgb"].data_ptr(),
            out["weight"].data_ptr(), out["count"].data_ptr(), out["rep"].data_ptr(),
            out["key"].data_ptr(), out["stats"].data_ptr(), side.cuda_stream)
    assert st == F.FUSEFLOW_ERR_INVALID_ARG
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    assert int(out["stats"].sum()) == 0              # nothing was written


@pytest.mark.parametrize("top_k", [0, 3])
def test_static_entry_point_matches_context_path_twice(top_k):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow as F
    from parity import run_gpu
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rig = S.tiny_rig(n=3, width=160, height=120, spread_deg=30.0)
    frames = [S.random_frame(rig, seed=s, flying_frac=0.01) for s in (31, 32)]
    cap = 8192
    for fr in frames:
        ff = F.FuseFlow(rig, max_cells=cap, top_k=top_k)
        try:
            ref = run_gpu(ff, fr, torch, with_trace=False)
        finally:
            ff.close()
        assert ref["status"] == F.FUSEFLOW_OK and ref["stats"]["n_cells"] > 100
        p = F.fuseflow_default_params(depth_format=F.FUSEFLOW_DEPTH_U16,
                                      depth_scale=rig.depth_scale, max_cells=cap, top_k=top_k)
        intr, extr = F.rig_arrays(rig)
        d = [torch.from_numpy(x).to(dev) for x in fr.depth]
        c = [torch.from_numpy(x).to(dev) for x in fr.conf]
        r = [torch.from_numpy(x).to(dev) for x in fr.rgb]
        out = _outputs(cap, dev)
        st = F.fuseflow_fuse_frame_static(
            intr, extr, rig.n_cams, p, [t.data_ptr() for t in d], [t.data_ptr() for t in c],
            [t.data_ptr() for t in r], out["pos"].data_ptr(), out["rgb"].data_ptr(),
            out["weight"].data_ptr(), out["count"].data_ptr(), out["rep"].data_ptr(),
            out["key"].data_ptr(), out["stats"].data_ptr(), stream)
        assert st == F.FUSEFLOW_OK
        torch.cuda.synchronize()
        raw = out["stats"].cpu().numpy().tobytes()[:ctypes.sizeof(F.fuseflow_stats)]
        stats = F.fuseflow_stats.from_buffer_copy(raw)
        assert stats.error == 0
        for k in ("n_valid", "n_gated", "n_out_of_range"):
            assert getattr(stats, k) == ref["stats"][k]
        _check_same(ref["cells"], ref["stats"], out, int(stats.n_cells))


def test_static_entry_point_rejects_oversized_requests():
    from paper_2602_01035_gb300 import fuseflow as F
    rig = S.tiny_rig(n=2, width=1024, height=512)          # 1,048,576 pixels > 524,288
    intr, extr = F.rig_arrays(rig)
    p = F.fuseflow_default_params()
    st = F.fuseflow_fuse_frame_static(intr, extr, 2, p, [1, 1], [1, 1], [1, 1], 1, 1, 1, 1, 1,
                                      1, 1, 0)
    assert st == F.FUSEFLOW_ERR_CAPACITY
    small = S.tiny_rig(n=2, width=64, height=48)
    intr, extr = F.rig_arrays(small)
    p = F.fuseflow_default_params(max_cells=40000)
    st = F.fuseflow_fuse_frame_static(intr, extr, 2, p, [1, 1], [1, 1], [1, 1], 1, 1, 1, 1, 1,
                                      1, 1, 0)
    assert st == F.FUSEFLOW_ERR_CAPACITY
