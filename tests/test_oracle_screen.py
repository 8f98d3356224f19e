"""Pins of the oracle's depth screen D^r (the preprocessed depth of Eq. 8; the rule is stated
with orc_screen_depth) against closed forms on constructed images, and of its wiring into
the frame: a frame fused with a screen set equals the frame fused, unscreened, from the
screened images."""
import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S


def _step(w=12, h=7, x0=5, z0=1000, z1=2000):
    d = np.full((h, w), z0, np.uint16)
    d[:, x0:] = z1
    return d


def test_no_screen_keeps_every_valid_sample(oracle_mod):
    rng = np.random.default_rng(3)
    d = rng.integers(0, 5000, size=(9, 13)).astype(np.uint16)
    np.testing.assert_array_equal(oracle_mod.screen_depth(d, "u16", 0.001), d)
    f = rng.uniform(0.5, 4.0, size=(9, 13)).astype(np.float32)
    f[0, 0], f[1, 1], f[2, 2], f[3, 3] = np.nan, -1.0, np.inf, 0.0
    ref = f.copy()
    ref[0, 0] = ref[1, 1] = ref[2, 2] = 0.0               # invalid samples become 0
    np.testing.assert_array_equal(oracle_mod.screen_depth(f, "f32", 1.0), ref)


def test_a_depth_step_screens_exactly_the_two_columns_beside_it(oracle_mod):
    d = _step()
    out = oracle_mod.screen_depth(d, "u16", 0.001, screen_edge_rel=0.1)
    ref = d.copy()
    ref[:, 4:6] = 0                                       # |1 - 2| > 0.1 z on both sides
    np.testing.assert_array_equal(out, ref)
    # the test is relative to the pixel's own depth: a 0.8 m jump exceeds 0.5 z on the
    # near side (0.6 m) but not on the far side (1.0 m)
    d2 = _step(z0=1200, z1=2000)
    out2 = oracle_mod.screen_depth(d2, "u16", 0.001, screen_edge_rel=0.5)
    ref2 = d2.copy()
    ref2[:, 4] = 0
    np.testing.assert_array_equal(out2, ref2)


def test_a_gentle_slope_is_kept(oracle_mod):
    # z = 2 m + 1 mm per column: relative jump 1/2000 < 0.01 everywhere
    d = (2000 + np.arange(40)[None, :] + np.zeros((6, 1), np.int64)).astype(np.uint16)
    np.testing.assert_array_equal(oracle_mod.screen_depth(d, "u16", 0.001, screen_edge_rel=0.01), d)


def test_an_isolated_flying_pixel_removes_a_plus_shape(oracle_mod):
    d = np.full((7, 9), 2000, np.uint16)
    d[3, 4] = 5000
    out = oracle_mod.screen_depth(d, "u16", 0.001, screen_edge_rel=0.05)
    ref = d.copy()
    for y, x in [(3, 4), (2, 4), (4, 4), (3, 3), (3, 5)]:
        ref[y, x] = 0
    np.testing.assert_array_equal(out, ref)


def test_invalid_and_out_of_range_neighbours_do_not_screen(oracle_mod):
    d = np.full((5, 6), 2000, np.uint16)
    d[:, 0] = 0                                           # invalid column
    d[:, 5] = 9000                                        # beyond the upper bound
    out = oracle_mod.screen_depth(d, "u16", 0.001, screen_max_m=5.0, screen_edge_rel=0.05)
    ref = d.copy()
    ref[:, 5] = 0                                         # out of range itself
    np.testing.assert_array_equal(out, ref)


def test_range_bounds_are_inclusive(oracle_mod):
    d = np.array([[499, 500, 501, 2999, 3000, 3001]], np.uint16)
    out = oracle_mod.screen_depth(d, "u16", 0.001, screen_min_m=0.5, screen_max_m=3.0)
    np.testing.assert_array_equal(out, [[0, 500, 501, 2999, 3000, 0]])
    f = np.array([[0.25, 0.5, 3.0, 3.5]], np.float32)
    out = oracle_mod.screen_depth(f, "f32", 1.0, screen_min_m=0.5, screen_max_m=3.0)
    np.testing.assert_array_equal(out, [[0.0, 0.5, 3.0, 0.0]])


@pytest.mark.parametrize("screen", [{"screen_edge_rel": 0.03},
                                    {"screen_min_m": 1.0, "screen_max_m": 3.5},
                                    {"screen_min_m": 1.5, "screen_edge_rel": 0.02}])
def test_screened_frame_equals_the_frame_of_screened_images(oracle_mod, screen):
    rig = S.tiny_rig(n=3, width=48, height=36, spread_deg=25.0, fx=40.0, fy=40.0)
    fr = S.random_frame(rig, seed=77, zero_frac=0.05, flying_frac=0.03)
    a = oracle_mod.fuse_frame(rig, fr, dict(screen))
    dr = [oracle_mod.screen_depth(d, rig.depth_format, rig.depth_scale, **screen) for d in fr.depth]
    assert any((x != d).any() for x, d in zip(dr, fr.depth))          # the screen acts
    b = oracle_mod.fuse_frame(rig, S.Frame(dr, fr.conf, fr.rgb, fr.z_true, fr.surface_id), {})
    assert a["stats"] == b["stats"]
    for k in a["cells"]:
        np.testing.assert_array_equal(a["cells"][k], b["cells"][k])
    for k in ("valid", "gated", "key", "nview", "omega"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["stats"]["n_valid"] == sum(int((x > 0).sum()) for x in dr)
