"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/fuseflow.h declares; argument validation needs no GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fuseflow.h")


@pytest.fixture(scope="module")
def ffmod():
    from paper_2602_01035_gb300 import fuseflow
    fuseflow.load()
    return fuseflow


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fuseflow_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fuseflow_create", "fuseflow_fuse_frame", "fuseflow_destroy",
                     "fuseflow_read_stats", "fuseflow_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(ffmod):
    lib = C.CDLL(ffmod.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in ffmod.EXPORTS, f"binding lacks {name}"


def test_status_strings(ffmod):
    for s in range(7):
        assert ffmod.fuseflow_status_string(s)
    assert "unknown" in ffmod.fuseflow_status_string(99)


def test_default_params_follow_the_paper(ffmod):
    import json
    const = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = ffmod.fuseflow_default_params()
    assert p.tau == np.float32(const["tau"]["value"])
    assert p.k_views == 4 and p.use_conf == 1 and p.use_consistency == 1


def _rig(n=2):
    from paper_2602_01035_gb300 import scenes as S
    return S.tiny_rig(n=n, width=16, height=12)


@pytest.mark.parametrize("field,value", [("k_views", 0), ("sigma_m", 0.0), ("sigma_m", -1.0),
                                         ("coarse_cell_m", 0.0), ("max_level", 15),
                                         ("max_level", -1), ("n_min", 0), ("depth_format", 7),
                                         ("depth_scale", 0.0), ("max_cells", -5),
                                         ("tau", float("nan")), ("tau", -0.5)])
def test_create_rejects_bad_parameters(ffmod, field, value):
    rig = _rig()
    intr, extr = ffmod.rig_arrays(rig)
    p = ffmod.fuseflow_default_params()
    setattr(p, field, value)
    ctx = C.c_void_p()
    st = ffmod.load().fuseflow_create(intr, extr, 2, C.byref(p), C.byref(ctx))
    assert st == ffmod.FUSEFLOW_ERR_INVALID_ARG
    assert not ctx.value


def test_create_rejects_bad_rigs(ffmod):
    lib = ffmod.load()
    rig = _rig(3)
    intr, extr = ffmod.rig_arrays(rig)
    p = ffmod.fuseflow_default_params()
    ctx = C.c_void_p()
    assert lib.fuseflow_create(intr, extr, 0, C.byref(p), C.byref(ctx)) == 1
    assert lib.fuseflow_create(intr, extr, 65, C.byref(p), C.byref(ctx)) == 1
    assert lib.fuseflow_create(None, extr, 3, C.byref(p), C.byref(ctx)) == 1
    bad = (ffmod.fuseflow_intrinsics * 3)(*intr)
    bad[1].fx = -1.0
    assert lib.fuseflow_create(bad, extr, 3, C.byref(p), C.byref(ctx)) == 1
    bad = (ffmod.fuseflow_intrinsics * 3)(*intr)
    bad[2].width = 0
    assert lib.fuseflow_create(bad, extr, 3, C.byref(p), C.byref(ctx)) == 1
    badx = (ffmod.fuseflow_extrinsics * 3)(*extr)
    badx[0].t[1] = float("inf")
    assert lib.fuseflow_create(intr, badx, 3, C.byref(p), C.byref(ctx)) == 1
    p.k_views = 10     # K - 1 = 9 neighbours exceeds the 8 the kernels carry
    big = _rig(12)
    bi, be = ffmod.rig_arrays(big)
    assert lib.fuseflow_create(bi, be, 12, C.byref(p), C.byref(ctx)) == 1


def test_null_arguments_are_rejected(ffmod):
    lib = ffmod.load()
    assert lib.fuseflow_fuse_frame(None, None, None, None, None, None) == 1
    assert lib.fuseflow_read_stats(None, None, None) == 1
    assert lib.fuseflow_set_trace(None, None) == 1
    assert lib.fuseflow_num_pixels(None) == 0
    lib.fuseflow_destroy(None)


def test_header_has_no_torch_types():
    text = open(HEADER).read()
    assert "torch" not in text.lower().replace("pytorch", "") or "at::" not in text
    assert "at::Tensor" not in text and "c10" not in text


def test_server_rejects_bad_arguments_without_a_gpu(ffmod):
    lib = ffmod.load()
    srv = C.c_void_p()
    assert lib.fuseflow_server_create(0, C.byref(srv)) == ffmod.FUSEFLOW_ERR_INVALID_ARG
    assert lib.fuseflow_server_create(-5, C.byref(srv)) == ffmod.FUSEFLOW_ERR_INVALID_ARG
    n = C.c_int32(7)
    assert lib.fuseflow_server_poll(None, None, 0, C.byref(n)) == ffmod.FUSEFLOW_ERR_INVALID_ARG
    rid = C.c_int32()
    p = ffmod.fuseflow_default_params()
    assert lib.fuseflow_server_add_rig(None, None, None, 1, C.byref(p), 1,
                                       C.byref(rid)) == ffmod.FUSEFLOW_ERR_INVALID_ARG
    req = C.c_int64()
    assert lib.fuseflow_server_submit(None, 0, None, None, None, None,
                                      C.byref(req)) == ffmod.FUSEFLOW_ERR_INVALID_ARG
    assert lib.fuseflow_server_pending(None) == 0
    assert lib.fuseflow_server_device_bytes(None) == 0
    lib.fuseflow_server_destroy(None)


def test_tuning_entry_points_reject_bad_arguments_without_a_gpu(ffmod):
    lib = ffmod.load()
    tu = ffmod.fuseflow_tuning(4, 1216, 608, 0)
    bad = ffmod.FUSEFLOW_ERR_INVALID_ARG
    assert lib.fuseflow_get_tuning(None, C.byref(tu)) == bad
    assert lib.fuseflow_set_tuning(None, C.byref(tu)) == bad
    us = (C.c_double * 2)()
    assert lib.fuseflow_autotune(None, None, None, None, 9, C.byref(tu), us, None) == bad
    assert lib.fuseflow_server_autotune(None, 0, None, None, None, 9, C.byref(tu), us) == bad


def test_graph_entry_points_reject_bad_arguments_without_a_gpu(ffmod):
    lib = ffmod.load()
    g = C.c_void_p()
    bad = ffmod.FUSEFLOW_ERR_INVALID_ARG
    assert lib.fuseflow_graph_create(None, None, None, None, C.byref(g)) == bad
    assert lib.fuseflow_graph_launch(None, None, None) == bad
    lib.fuseflow_graph_destroy(None)
