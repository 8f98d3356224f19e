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
