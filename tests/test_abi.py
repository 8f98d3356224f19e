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
    assert ffmod.FUSEFLOW_ERR_CANCELLED == 7
    for s in range(8):
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
                                         ("tau", float("nan")), ("tau", -0.5),
                                         ("screen_min_m", float("inf")),
                                         ("screen_max_m", float("nan")),
                                         ("screen_edge_rel", float("inf")), ("reserved1", 3)])
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
    held = C.c_int32()
    assert lib.fuseflow_server_reserve(None, 0, 2, C.byref(held)) == ffmod.FUSEFLOW_ERR_INVALID_ARG
    assert lib.fuseflow_server_remove_rig(None, 0) == ffmod.FUSEFLOW_ERR_INVALID_ARG
    st = ffmod.fuseflow_server_stats()
    assert lib.fuseflow_server_get_stats(None, C.byref(st)) == ffmod.FUSEFLOW_ERR_INVALID_ARG
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
    # batches: counts and NULL arguments are refused before any context is touched
    b = C.c_void_p()
    assert lib.fuseflow_batch_create(None, 2, C.byref(b)) == bad
    ctxs = (C.c_void_p * 9)()
    assert lib.fuseflow_batch_create(ctxs, 0, C.byref(b)) == bad
    assert lib.fuseflow_batch_create(ctxs, 9, C.byref(b)) == bad
    assert lib.fuseflow_batch_create(ctxs, 2, None) == bad
    assert lib.fuseflow_batch_fuse(None, None, None, None, None) == bad
    assert lib.fuseflow_batch_graph_create(None, None, None, None, C.byref(g)) == bad
    lib.fuseflow_batch_destroy(None)
    cl = ffmod.fuseflow_cloud()
    assert lib.fuseflow_get_cloud(None, C.byref(cl)) == bad
    assert lib.fuseflow_fuse_points(None, None, None, None, None, None, None, None, None, None) == bad


def test_screen_bounds_must_be_ordered_and_static_entry_has_no_screen(ffmod):
    lib = ffmod.load()
    rig = _rig()
    intr, extr = ffmod.rig_arrays(rig)
    p = ffmod.fuseflow_default_params()
    assert p.screen_min_m == 0 and p.screen_max_m == 0 and p.screen_edge_rel == 0
    p.screen_min_m, p.screen_max_m = 3.0, 2.0
    ctx = C.c_void_p()
    assert lib.fuseflow_create(intr, extr, 2, C.byref(p), C.byref(ctx)) == 1 and not ctx.value
    # the allocation-free entry has no buffer for D^r: refused before any GPU work
    p = ffmod.fuseflow_default_params(screen_edge_rel=0.05)
    dummy = (C.c_void_p * 2)(1, 1)
    out = C.c_void_p(1)
    st = lib.fuseflow_fuse_frame_static(intr, extr, 2, C.byref(p), dummy, dummy, dummy, out, out,
                                        out, out, out, out, out, None)
    assert st == ffmod.FUSEFLOW_ERR_INVALID_ARG
    assert lib.fuseflow_screen_depth(None, dummy, dummy, None) == ffmod.FUSEFLOW_ERR_INVALID_ARG


def test_struct_layouts_match_the_header(ffmod, tmp_path):
    """sizeof/offsetof of every ABI struct from a C compiler against the ctypes binding."""
    import subprocess
    structs = {"fuseflow_params": ffmod.fuseflow_params, "fuseflow_stats": ffmod.fuseflow_stats,
               "fuseflow_cloud": ffmod.fuseflow_cloud, "fuseflow_trace": ffmod.fuseflow_trace,
               "fuseflow_intrinsics": ffmod.fuseflow_intrinsics,
               "fuseflow_extrinsics": ffmod.fuseflow_extrinsics,
               "fuseflow_conf_params": ffmod.fuseflow_conf_params,
               "fuseflow_tuning": ffmod.fuseflow_tuning,
               "fuseflow_host_cloud": ffmod.fuseflow_host_cloud,
               "fuseflow_completion": ffmod.fuseflow_completion,
               "fuseflow_server_stats": ffmod.fuseflow_server_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fuseflow.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, f"{name}.{field}"


def test_server_cap_rejects_bad_arguments_without_a_gpu(ffmod):
    lib = ffmod.load()
    assert lib.fuseflow_server_set_max_inflight(None, 2) == ffmod.FUSEFLOW_ERR_INVALID_ARG


def test_binding_fails_loudly_without_the_library(ffmod, tmp_path):
    """No fallback: with the library missing, loading raises instead of computing elsewhere."""
    saved_lib, saved_path = ffmod._lib, ffmod._build.LIB
    try:
        ffmod._lib = None
        ffmod._build.LIB = str(tmp_path / "missing" / "libfuseflow.so")
        with pytest.raises(ImportError):
            ffmod.load(build_if_missing=False)
    finally:
        ffmod._lib, ffmod._build.LIB = saved_lib, saved_path


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: nothing in the package may import or run it."""
    pkg = os.path.join(ROOT, "paper_2602_01035_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            text = open(os.path.join(pkg, name)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), name
            assert "liboracle" not in text, name
