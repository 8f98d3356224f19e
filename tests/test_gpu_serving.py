"""The serving runtime (fuseflow_server_*): results alone and in a mix, budget admission,
continuous batching over slots.  Frames come from pinned host memory and results land in
pinned host arrays; every comparison is bitwise against the plain device path, whose
parity with the oracle is checked in test_gpu_parity.py."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S
from parity import run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01035_gb300 import fuseflow, serving
    fuseflow.load()
    return fuseflow, serving


def _cases():
    r1, _, f1 = S.config1()
    r2 = S.tiny_rig(n=3, width=96, height=64, spread_deg=25.0, fx=80.0, fy=78.0)
    f2 = S.random_frame(r2, seed=21, zero_frac=0.02, flying_frac=0.01)
    r3 = S.tiny_rig(n=5, width=64, height=48, depth_format="f32", depth_scale=1.0, spread_deg=20.0)
    f3 = S.random_frame(r3, seed=22, zero_frac=0.05)
    return [(r1, f1), (r2, f2), (r3, f3)]


def _alone(F, rig, fr):
    ff = F.FuseFlow(rig)
    try:
        out = run_gpu(ff, fr, torch, with_trace=False)
    finally:
        ff.close()
    return out


def _same(a: dict, b: dict):
    for k in ("pos", "rgb", "weight", "count", "rep", "key"):
        assert np.array_equal(a[k], b[k]), k


def test_results_alone_and_in_the_mix(mods):
    F, SV = mods
    cases = _cases()
    alone = [_alone(F, r, f) for r, f in cases]
    srv = SV.Server(8 << 30)
    try:
        rids = [srv.add_rig(r, n_slots=2) for r, _ in cases]
        frames = [SV.pinned_frame(f) for _, f in cases]
        # every rig three times, interleaved, all in flight at once: more frames than slots
        order = [0, 1, 2, 2, 1, 0, 1, 2, 0]
        bufs, reqs = {}, {}
        for k, r in enumerate(order):
            hc = SV.HostCloud(srv.rigs[r]["capacity"])
            req = srv.submit(rids[r], frames[r], hc)
            bufs[req] = (r, hc)
        done = srv.drain()
        assert len(done) == len(order) and srv.pending() == 0
        for req, rig, status, st in done:
            r, hc = bufs[req]
            assert rig == rids[r] and status == F.FUSEFLOW_OK
            assert st["n_cells"] == alone[r]["stats"]["n_cells"]
            _same(hc.cells(st["n_cells"]), alone[r]["cells"])
    finally:
        srv.close()


def _slot_bytes(SV, rig):
    srv = SV.Server(1 << 40)
    try:
        srv.add_rig(rig, n_slots=1)
        return srv.device_bytes()
    finally:
        srv.close()


def test_budget_admission(mods):
    F, SV = mods
    (r1, f1), (r2, _), _ = _cases()
    b1 = _slot_bytes(SV, r1)
    srv = SV.Server(b1 + (1 << 20))
    try:
        rid = srv.add_rig(r1, n_slots=1)
        used = srv.device_bytes()
        assert used == b1
        # a rig whose first slot does not fit is refused and leaves nothing behind
        status, _ = F.fuseflow_server_add_rig(srv.srv, *F.rig_arrays(r2), len(r2.cameras),
                                              F.fuseflow_default_params(), 4)
        assert status == F.FUSEFLOW_ERR_CAPACITY
        assert srv.device_bytes() == used
        hc = SV.HostCloud(srv.rigs[rid]["capacity"])
        pf = SV.pinned_frame(f1)                # inputs stay alive until completion
        srv.submit(rid, pf, hc)
        (req, rig, status, st), = srv.drain()
        assert status == F.FUSEFLOW_OK and st["n_cells"] > 0
    finally:
        srv.close()


def test_one_slot_serves_a_queue_in_order(mods):
    F, SV = mods
    r2 = S.tiny_rig(n=2, width=64, height=48)
    frs = [S.random_frame(r2, seed=30 + k) for k in range(5)]
    alone = [_alone(F, r2, f) for f in frs]
    srv = SV.Server(2 << 30)
    try:
        rid = srv.add_rig(r2, n_slots=1)
        bufs = {}
        pinned = [SV.pinned_frame(f) for f in frs]   # alive until every frame completes
        for k in range(len(frs)):
            hc = SV.HostCloud(srv.rigs[rid]["capacity"])
            bufs[srv.submit(rid, pinned[k], hc)] = (k, hc)
        assert srv.pending() == 5
        done = srv.drain()
        assert [d[0] for d in done] == sorted(bufs)            # FIFO on the single slot
        for req, _, status, st in done:
            k, hc = bufs[req]
            assert status == F.FUSEFLOW_OK
            _same(hc.cells(st["n_cells"]), alone[k]["cells"])
    finally:
        srv.close()


def test_capacity_of_the_host_arrays_is_reported(mods):
    F, SV = mods
    r1, _, f1 = S.config1()
    srv = SV.Server(1 << 30)
    try:
        rid = srv.add_rig(r1, n_slots=1)
        hc = SV.HostCloud(10)
        pf = SV.pinned_frame(f1)
        srv.submit(rid, pf, hc)
        (_, _, status, st), = srv.drain()
        assert status == F.FUSEFLOW_ERR_CAPACITY and st["n_cells"] > 10
    finally:
        srv.close()


def test_top_k_and_screened_rigs_serve_the_same_results(mods):
    F, SV = mods
    r1, _, f1 = S.config1()
    r2 = S.tiny_rig(n=3, width=96, height=64, spread_deg=25.0, fx=80.0, fy=78.0)
    f2 = S.random_frame(r2, seed=23, zero_frac=0.02, flying_frac=0.02)
    cases = [(r1, f1, {"top_k": 3}), (r2, f2, {"screen_edge_rel": 0.03, "screen_max_m": 4.0})]
    alone = []
    for rig, fr, prm in cases:
        ff = F.FuseFlow(rig, **prm)
        try:
            alone.append(run_gpu(ff, fr, torch, with_trace=False))
        finally:
            ff.close()
    srv = SV.Server(4 << 30)
    try:
        rids = [srv.add_rig(rig, n_slots=2, **prm) for rig, _, prm in cases]
        frames = [SV.pinned_frame(fr) for _, fr, _ in cases]
        bufs = {}
        for k in (0, 1, 1, 0):
            hc = SV.HostCloud(srv.rigs[rids[k]]["capacity"])
            bufs[srv.submit(rids[k], frames[k], hc)] = (k, hc)
        for req, _, status, st in srv.drain():
            k, hc = bufs[req]
            assert status == F.FUSEFLOW_OK
            _same(hc.cells(st["n_cells"]), alone[k]["cells"])
    finally:
        srv.close()



def test_in_flight_cap_starts_frames_in_submission_order(mods):
    F, SV = mods
    cases = _cases()
    alone = [_alone(F, r, f) for r, f in cases]
    srv = SV.Server(8 << 30)
    try:
        rids = [srv.add_rig(r, n_slots=2) for r, _ in cases]
        srv.set_max_inflight(1)                  # one frame at a time: strict FIFO over rigs
        frames = [SV.pinned_frame(f) for _, f in cases]
        order = [2, 0, 1, 1, 2, 0]
        bufs = {}
        for r in order:
            hc = SV.HostCloud(srv.rigs[r]["capacity"])
            bufs[srv.submit(rids[r], frames[r], hc)] = (r, hc)
        done = srv.drain()
        assert [d[0] for d in done] == sorted(bufs)
        for req, rig, status, st in done:
            r, hc = bufs[req]
            assert status == F.FUSEFLOW_OK and rig == rids[r]
            _same(hc.cells(st["n_cells"]), alone[r]["cells"])
        with pytest.raises(F.FuseFlowError):
            srv.set_max_inflight(-1)
    finally:
        srv.close()


def _submit_all(SV, srv, rid, pinned, n):
    bufs = {}
    for k in range(n):
        hc = SV.HostCloud(srv.rigs[rid]["capacity"])
        bufs[srv.submit(rid, pinned[k % len(pinned)], hc)] = (k % len(pinned), hc)
    return bufs


def test_a_binding_budget_limits_the_slots_and_frames_wait_for_memory(mods):
    """A rig asking for 4 frames in flight under a budget of 2.5 slots holds 2 after
    reserving; of six frames submitted at once the ones that find both busy wait (deferred
    by the budget), and every result is the one the frame gives alone."""
    F, SV = mods
    r2 = S.tiny_rig(n=3, width=96, height=64, spread_deg=25.0)
    frs = [S.random_frame(r2, seed=40 + k) for k in range(3)]
    alone = [_alone(F, r2, f) for f in frs]
    b = _slot_bytes(SV, r2)
    srv = SV.Server(int(2.5 * b))
    try:
        rid = srv.add_rig(r2, n_slots=4)
        assert srv.stats()["slots"] == 1
        assert srv.reserve(rid, 4) == 2
        pinned = [SV.pinned_frame(f) for f in frs]
        bufs = _submit_all(SV, srv, rid, pinned, 6)
        done = srv.drain()
        st = srv.stats()
        assert st["slots"] == 2 and st["used_bytes"] == 2 * b <= st["budget_bytes"]
        assert st["deferred_by_budget"] >= 1 and st["frames_completed"] == 6
        for req, _, status, s_ in done:
            k, hc = bufs[req]
            assert status == F.FUSEFLOW_OK
            _same(hc.cells(s_["n_cells"]), alone[k]["cells"])
    finally:
        srv.close()


def test_a_removed_rigs_memory_goes_to_rigs_below_their_request(mods):
    F, SV = mods
    r2 = S.tiny_rig(n=3, width=96, height=64, spread_deg=25.0)
    fr = S.random_frame(r2, seed=44)
    alone = _alone(F, r2, fr)
    b = _slot_bytes(SV, r2)
    srv = SV.Server(3 * b + (1 << 20))
    try:
        a = srv.add_rig(r2, n_slots=1)
        c = srv.add_rig(r2, n_slots=3)
        assert srv.reserve(c, 3) == 2                 # the budget is full: 3 slots
        srv.remove_rig(a)
        st = srv.stats()
        assert st["rigs"] == 1 and st["slots"] == 3 and st["used_bytes"] == 3 * b
        pinned = [SV.pinned_frame(fr)]
        bufs = _submit_all(SV, srv, c, pinned, 3)     # all three start at once
        assert srv.stats()["inflight"] == 3
        for req, rig, status, s_ in srv.drain():
            assert rig == c and status == F.FUSEFLOW_OK
            _same(bufs[req][1].cells(s_["n_cells"]), alone["cells"])
    finally:
        srv.close()


def test_removing_a_rig_finishes_its_frames_cancels_the_waiting_ones_and_frees_memory(mods):
    F, SV = mods
    (r1, f1), (r2, f2), _ = _cases()
    alone = _alone(F, r1, f1)
    srv = SV.Server(4 << 30)
    try:
        a = srv.add_rig(r1, n_slots=1)
        c = srv.add_rig(r2, n_slots=1)
        used_c = _slot_bytes(SV, r2)
        pa = [SV.pinned_frame(f1)]
        bufs = _submit_all(SV, srv, a, pa, 3)       # one on the slot, two waiting
        srv.remove_rig(a)
        assert srv.device_bytes() == used_c
        done = srv.drain()
        assert sorted(d[0] for d in done) == sorted(bufs)
        status = {req: st_ for req, _, st_, _ in done}
        first = min(bufs)
        assert status[first] == F.FUSEFLOW_OK
        _same(bufs[first][1].cells(next(d[3] for d in done if d[0] == first)["n_cells"]), alone["cells"])
        assert all(status[r] == F.FUSEFLOW_ERR_CANCELLED for r in bufs if r != first)
        st = srv.stats()
        assert st["rigs"] == 1 and st["frames_cancelled"] == 2
        with pytest.raises(F.FuseFlowError):
            srv.submit(a, pa[0], SV.HostCloud(16))
        pc = SV.pinned_frame(f2)                    # the remaining rig still serves
        srv.submit(c, pc, SV.HostCloud(srv.rigs[c]["capacity"]))
        (_, rig, st_, _), = srv.drain()
        assert rig == c and st_ == F.FUSEFLOW_OK
    finally:
        srv.close()


@pytest.mark.parametrize("after_copies", [False, True])
def test_a_frame_whose_start_fails_is_reported_with_its_error(mods, after_copies):
    """A start that fails (made on the host with the server's injection hook, before or after
    the frame's image copies were queued) is reported by poll with its request id and the
    error, the latter only once its copies are done; the next frame runs normally."""
    F, SV = mods
    r1, _, f1 = S.config1()
    alone = _alone(F, r1, f1)
    srv = SV.Server(1 << 30)
    try:
        rid = srv.add_rig(r1, n_slots=1)
        pf = SV.pinned_frame(f1)
        cap = srv.rigs[rid]["capacity"]
        F.fuseflow_server_inject_start_failure(srv.srv, 1, F.FUSEFLOW_ERR_CUDA, after_copies)
        bad, good = SV.HostCloud(cap), SV.HostCloud(cap)
        req = srv.submit(rid, pf, bad)
        req2 = srv.submit(rid, pf, good)
        done = {d[0]: d for d in srv.drain()}
        assert set(done) == {req, req2}
        assert done[req][2] == F.FUSEFLOW_ERR_CUDA
        assert done[req2][2] == F.FUSEFLOW_OK
        _same(good.cells(done[req2][3]["n_cells"]), alone["cells"])
        st = srv.stats()
        assert st["frames_failed"] == 1 and st["frames_completed"] == 1 and srv.pending() == 0
        with pytest.raises(F.FuseFlowError):
            F.fuseflow_server_inject_start_failure(srv.srv, 1, F.FUSEFLOW_OK, False)
    finally:
        srv.close()
