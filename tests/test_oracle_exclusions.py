"""Pins of the oracle parts that decide what the parity tests compare.

* the neighbour rule of Sec. II.5(2)b (optical-axis angle first, then centre distance,
  then index) on rigs where the angle order and the distance order differ;
* the tie order of the Sec. II.5(2)a top-k selection (equal confidences: lowest pixel
  index first) on a cell with duplicated confidences;
* the three exclusion sets the oracle reports (points within 1e-5 m of a cell face at
  their own level, coarse cells whose level could flip when such points move, and
  projections within 1e-6 px of a half-pixel tie), each on a constructed case placed
  just inside and just outside the band.

Every expected value follows from the construction (camera poses, exact depths in FP64),
not from the oracle's own arithmetic.
"""
import math

import numpy as np

from paper_2602_01035_gb300 import scenes as S


def _rot_to_axis(axis):
    """Camera-from-world rotation whose optical axis (R^T e_z) is the unit vector `axis`."""
    z = np.asarray(axis, float) / np.linalg.norm(axis)
    helper = np.array([0.0, 1.0, 0.0]) if abs(z[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(helper, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z])          # rows: camera axes in world coordinates


def _cam(centre, axis, fx=100.0, fy=100.0, cx=4.0, cy=3.0, w=8, h=6):
    R = _rot_to_axis(axis)
    t = -R @ np.asarray(centre, float)
    return S.Camera(fx, fy, cx, cy, w, h, R, t)


def _axis_at(deg, azimuth_deg=0.0):
    a, b = math.radians(deg), math.radians(azimuth_deg)
    return (math.sin(a) * math.cos(b), math.sin(a) * math.sin(b), math.cos(a))


# ------------------------------------------------------------------ Sec. II.5(2)b order
def test_neighbour_order_is_angle_before_distance(oracle_mod):
    """Camera 0 looks along +z from the origin; cameras 1, 2, 3 sit at 1, 5 and 2 m with
    axes at 40, 10 and 80 degrees.  By angle camera 0's list is [2, 1, 3]; by distance
    it would be [1, 3, 2].  Seen from camera 2 (axis 10 deg) the angles are 10, 30, 70
    degrees to cameras 0, 1, 3, the distances 5, 4, 3 m."""
    cams = [_cam((0, 0, 0), _axis_at(0)), _cam((1, 0, 0), _axis_at(40)),
            _cam((5, 0, 0), _axis_at(10)), _cam((2, 0, 0), _axis_at(80))]
    rig = S.Rig(cams, "u16", 0.001)
    nb = oracle_mod.neighbours(rig, 4)
    assert nb[0].tolist() == [2, 1, 3]
    assert nb[2].tolist() == [0, 1, 3]
    assert oracle_mod.neighbours(rig, 2)[0].tolist() == [2]


def test_neighbour_order_breaks_equal_angles_by_distance(oracle_mod):
    """Cameras 1, 2, 3 all at 20 degrees to camera 0's axis (different azimuths) and at 3,
    1 and 2 m: equal angles, so distance decides: [2, 3, 1]."""
    cams = [_cam((0, 0, 0), _axis_at(0)), _cam((3, 0, 0), _axis_at(20, 0)),
            _cam((0, 1, 0), _axis_at(20, 120)), _cam((0, 0, -2), _axis_at(20, 240))]
    rig = S.Rig(cams, "u16", 0.001)
    assert oracle_mod.neighbours(rig, 4)[0].tolist() == [2, 3, 1]


# ------------------------------------------------------------------ Sec. II.5(2)a ties
def test_top_k_ties_go_to_the_lowest_pixel_index(oracle_mod):
    """One camera (N = 1, so V = 1 and omega = C) looking straight down at a flat patch
    inside one coarse cell; six valid pixels with confidences 0.9, 0.8, 0.9, 0.9, 0.7, 0.9
    form one cell.  top_k = 3 fuses the three 0.9 members of lowest index (pixels 0, 2, 3),
    so the fused position is their mean and W = 2.7; the reverse tie order would take
    pixels 5, 3, 2 and another mean."""
    cam = S.Camera(4000.0, 4000.0, 1.5, 0.5, 4, 2, np.eye(3), np.array([-0.16, -0.16, 0.0]))
    rig = S.Rig([cam], "f64", 1.0)
    depth = np.zeros((2, 4), np.float64)
    depth.ravel()[:6] = [1.10, 1.11, 1.12, 1.13, 1.14, 1.15]   # distinct z, one coarse cell
    conf = np.zeros((2, 4), np.float32)
    conf.ravel()[:6] = [0.9, 0.8, 0.9, 0.9, 0.7, 0.9]
    fr = S.Frame([depth], [conf], [np.zeros((2, 4, 3), np.uint8)])
    res = oracle_mod.fuse_frame(rig, fr, {"n_min": 32, "top_k": 3}, depth_format="f64")
    cells = res["cells"]
    assert len(cells["key"]) == 1 and cells["count"][0] == 6
    assert cells["rep"][0] == 0                      # largest C, lowest index
    pw = res["pw"]
    want = pw[[0, 2, 3]].mean(axis=0)
    wrong = pw[[2, 3, 5]].mean(axis=0)
    np.testing.assert_allclose(cells["pos"][0], want, rtol=0, atol=1e-12)
    assert np.abs(cells["pos"][0] - wrong).max() > 1e-3
    assert abs(cells["weight"][0] - 3 * float(np.float32(0.9))) < 1e-12


# ------------------------------------------------------------------ boundary band
def _point_rig(p_world):
    """A 1x1 camera with R = I whose only pixel's ray (fx = fy = 1, cx = cy = 0) meets the
    world point p_world at depth p_world[2]: the camera centre sits below it."""
    t = np.array([-p_world[0], -p_world[1], 0.0])
    return S.Rig([S.Camera(1.0, 1.0, 0.0, 0.0, 1, 1, np.eye(3), t)], "f64", 1.0)


def _one_point(oracle_mod, p, params=None):
    rig = _point_rig(p)
    fr = S.Frame([np.array([[p[2]]], np.float64)], [np.full((1, 1), 0.9, np.float32)],
                 [np.zeros((1, 1, 3), np.uint8)])
    return oracle_mod.fuse_frame(rig, fr, dict({"n_min": 1}, **(params or {})), depth_format="f64")


def test_boundary_band_flags_points_within_1e5_m_of_a_face(oracle_mod):
    """A single point at x = y = 0.16 (mid-cell) and z = 0.96 + delta (the face z = 3 s0 of
    the 0.32 m lattice): flagged for |delta| = 5e-6 m on either side, not for 2e-5 m."""
    for delta, flagged in ((5e-6, True), (-5e-6, True), (2e-5, False), (-2e-5, False)):
        res = _one_point(oracle_mod, (0.16, 0.16, 0.96 + delta))
        assert res["level"][0] == 0
        assert abs(res["margin_cell_m"][0] - abs(delta)) < 1e-12
        assert res["stats"]["n_boundary_points"] == int(flagged)
        has = (res["cells"]["flags"][0] & oracle_mod.CELL_BOUNDARY) != 0
        assert has == flagged


def test_boundary_band_uses_the_points_own_level(oracle_mod):
    """16 points in one coarse cell with n_min = 1 refine it to level 2 (edge 0.08 m).  The
    point at z = 1.04 + 5e-6 lies 5e-6 m from a level-2 face (1.04 = 13 x 0.08) but 0.08 m
    from every coarse face: it is flagged, the others (z = 1.0, mid-cell) are not."""
    cam = S.Camera(1.0e6, 1.0e6, 1.5, 1.5, 4, 4, np.eye(3), np.array([-0.2, -0.2, 0.0]))
    rig = S.Rig([cam], "f64", 1.0)
    depth = np.full((4, 4), 1.0, np.float64)
    depth[3, 3] = 1.04 + 5e-6
    fr = S.Frame([depth], [np.full((4, 4), 0.9, np.float32)], [np.zeros((4, 4, 3), np.uint8)])
    res = oracle_mod.fuse_frame(rig, fr, {"n_min": 1, "max_level": 2}, depth_format="f64")
    assert np.all(res["level"] == 2)
    assert res["stats"]["n_boundary_points"] == 1
    m = res["margin_cell_m"].reshape(4, 4)
    assert abs(m[3, 3] - 5e-6) < 1e-12
    assert np.all(np.delete(m.ravel(), 15) > 0.039)
    flagged = (res["cells"]["flags"] & oracle_mod.CELL_BOUNDARY) != 0
    assert flagged.sum() == 1
    assert res["cells"]["count"][flagged][0] == 1


# ------------------------------------------------------------------ ambiguous level
def _column(oracle_mod, z_values):
    """Points at x = y = 0.2 (mid-cell laterally) and the given depths, one per pixel of a
    4x5 image (the rest invalid), n_min = 4, Lmax = 1: a coarse cell refines at 16 points."""
    cam = S.Camera(1.0e6, 1.0e6, 2.0, 1.5, 5, 4, np.eye(3), np.array([-0.2, -0.2, 0.0]))
    rig = S.Rig([cam], "f64", 1.0)
    depth = np.zeros((4, 5), np.float64)
    depth.ravel()[:len(z_values)] = z_values
    fr = S.Frame([depth], [np.full((4, 5), 0.9, np.float32)], [np.zeros((4, 5, 3), np.uint8)])
    return oracle_mod.fuse_frame(rig, fr, {"n_min": 4, "max_level": 1}, depth_format="f64")


def _ambiguous_counts(oracle_mod, res):
    amb = (res["cells"]["flags"] & oracle_mod.CELL_AMBIGUOUS_LEVEL) != 0
    return res["stats"]["n_ambiguous_coarse"], int(res["cells"]["count"][amb].sum())


def test_ambiguous_level_when_a_boundary_point_inside_decides(oracle_mod):
    """n_c = 16 = n_min 4^1 with one of the 16 points 5e-6 m inside the coarse face
    z = 0.96: without it the cell would have level 0, so the coarse cell is ambiguous.
    With 17 points (16 without the boundary point) it is not."""
    res = _column(oracle_mod, [1.1] * 15 + [0.96 + 5e-6])
    assert np.all(res["level"][res["gated"].astype(bool)] == 1)
    assert _ambiguous_counts(oracle_mod, res) == (1, 16)
    res = _column(oracle_mod, [1.1] * 16 + [0.96 + 5e-6])
    assert _ambiguous_counts(oracle_mod, res) == (0, 0)


def test_ambiguous_level_when_a_boundary_point_outside_decides(oracle_mod):
    """15 points in the coarse cell and one 5e-6 m below its face (in the cell below): with
    that point the count would reach 16, so the 15-point cell is ambiguous; 2e-5 m below
    the face (outside the band) it is not, and the lone point's own cell never is."""
    res = _column(oracle_mod, [1.1] * 15 + [0.96 - 5e-6])
    assert res["stats"]["n_coarse"] == 2
    assert _ambiguous_counts(oracle_mod, res) == (1, 15)
    res = _column(oracle_mod, [1.1] * 15 + [0.96 - 2e-5])
    assert _ambiguous_counts(oracle_mod, res) == (0, 0)


# ------------------------------------------------------------------ half-pixel ties
def _tie_rig(eps_px):
    """Camera 1 (R = I at the origin, fx = fy = 100, cx = cy = 0, 8x8 depth of 1 m) sees the
    world point P = (0.025 + eps/100, 0.012, 1) at u = 2.5 + eps, v = 1.2.  Camera 0 (1x1,
    centre at x = -0.1) has its only pixel's ray through P at depth 1."""
    px = 0.025 + eps_px / 100.0
    c1 = S.Camera(100.0, 100.0, 0.0, 0.0, 8, 8, np.eye(3), np.zeros(3))
    c0 = S.Camera(1.0, 1.0, -(px + 0.1), -0.012, 1, 1, np.eye(3), np.array([0.1, 0.0, 0.0]))
    rig = S.Rig([c0, c1], "f64", 1.0)
    fr = S.Frame([np.ones((1, 1)), np.ones((8, 8))],
                 [np.full((1, 1), 0.9, np.float32), np.full((8, 8), 0.9, np.float32)],
                 [np.zeros((1, 1, 3), np.uint8), np.zeros((8, 8, 3), np.uint8)])
    return rig, fr


def test_half_pixel_tie_flag(oracle_mod):
    """Camera 0's point projects 1e-7 px from the half-pixel u = 2.5 of camera 1: flagged
    (margin below 1e-6 px) and its cell marked; at 1e-5 px it is not."""
    for eps, flagged in ((1e-7, True), (-1e-7, True), (1e-5, False)):
        rig, fr = _tie_rig(eps)
        res = oracle_mod.fuse_frame(rig, fr, {"k_views": 2, "n_min": 1}, depth_format="f64")
        np.testing.assert_allclose(res["pw"][0], [0.025 + eps / 100, 0.012, 1.0], atol=1e-15)
        assert abs(res["margin_tie_px"][0] - abs(eps)) < 1e-9
        assert res["nview"][0] == 1
        assert (res["stats"]["n_tie_points"] >= 1) == flagged
        cell = np.flatnonzero(res["cells"]["key"] == res["key"][0])[0]
        assert bool(res["cells"]["flags"][cell] & oracle_mod.CELL_TIE) == flagged
