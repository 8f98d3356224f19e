"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a closed form, an
invariant, a special case, or a brute-force computation written differently (projection
matrices, pixel search, explicit inverses, independent grouping).
"""
import copy
import json
import os

import numpy as np
import pytest

from paper_2602_01035_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frame_f64(fr):
    return S.Frame([z.astype(np.float64) for z in fr.z_true], fr.conf, fr.rgb, fr.z_true,
                   fr.surface_id)


def _kinv(cam):
    K = np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1.0]])
    return np.linalg.inv(K)


def _proj_matrix(cam):
    K = np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1.0]])
    return K @ np.hstack([cam.R, cam.t[:, None]])


def _pixel_table(rig):
    rows = []
    for i, c in enumerate(rig.cameras):
        yy, xx = np.mgrid[0:c.height, 0:c.width]
        rows.append(np.stack([np.full(xx.size, i), xx.ravel(), yy.ravel()], axis=1))
    return np.concatenate(rows)


# ------------------------------------------------------------------------ Eq. 8 closed form
def test_backprojection_lands_on_analytic_surfaces(oracle_mod):
    """Noiseless FP64 depth of the plane z=0 and the sphere c=(0,0,0.4), r=0.4 must
    back-project onto those surfaces within 1e-9 m (Eq. 8), and re-project through the
    forward camera model onto the same pixel with the same z (Eq. 4 inverse)."""
    cams = [S.look_at((2.0, 0.3, 1.0), (0, 0, 0), 151.0, 149.0, 81.3, 58.7, 160, 120),
            S.look_at((1.0, 1.73, 1.2), (0, 0, 0.1), 140.0, 155.0, 77.0, 62.5, 160, 120)]
    rig = S.Rig(cams, "f64", 1.0)
    prims = [S.Plane((0, 0, 1), 0.0), S.Sphere((0.0, 0.0, 0.4), 0.4)]
    fr = S.render_frame(S.Rig(cams, "f32", 1.0), prims, seed=0, noiseless=True, keep_truth=True)
    res = oracle_mod.fuse_frame(rig, _frame_f64(fr), {"tau": 0.0}, depth_format="f64")
    sid = np.concatenate([s.ravel() for s in fr.surface_id])
    g = res["gated"].astype(bool)
    assert g.sum() > 20000
    pw = res["pw"]
    plane = g & (sid == 0)
    sphere = g & (sid == 1)
    assert plane.sum() > 5000 and sphere.sum() > 2000
    assert np.max(np.abs(pw[plane, 2])) < 1e-9
    rad = np.linalg.norm(pw[sphere] - np.array([0, 0, 0.4]), axis=1)
    assert np.max(np.abs(rad - 0.4)) < 1e-9
    tab = _pixel_table(rig)
    zt = np.concatenate([z.ravel() for z in fr.z_true])
    for i, cam in enumerate(cams):
        sel = g & (tab[:, 0] == i)
        h = np.hstack([pw[sel], np.ones((sel.sum(), 1))]) @ _proj_matrix(cam).T
        assert np.max(np.abs(h[:, 0] / h[:, 2] - tab[sel, 1])) < 1e-9
        assert np.max(np.abs(h[:, 1] / h[:, 2] - tab[sel, 2])) < 1e-9
        assert np.max(np.abs(h[:, 2] - zt[sel])) < 1e-9


# ------------------------------------------------------------------------ Eq. 9 gate
def test_gate_is_strict_and_in_float32(oracle_mod):
    rig = S.tiny_rig(n=1, width=8, height=6, depth_format="f32", depth_scale=1.0)
    depth = np.full((6, 8), 2.0, np.float32)
    conf = np.full((6, 8), 0.9, np.float32)
    conf[0, 0] = np.float32(0.6)
    conf[0, 1] = np.nextafter(np.float32(0.6), np.float32(1))
    conf[0, 2] = np.nextafter(np.float32(0.6), np.float32(0))
    depth[1, 0] = 0.0
    depth[1, 1] = np.nan
    depth[1, 2] = np.inf
    depth[1, 3] = -1.0
    fr = S.Frame([depth], [conf], [np.zeros((6, 8, 3), np.uint8)])
    res = oracle_mod.fuse_frame(rig, fr, {})
    gated = res["gated"].reshape(6, 8)
    valid = res["valid"].reshape(6, 8)
    assert gated[0, 0] == 0 and gated[0, 1] == 1 and gated[0, 2] == 0
    assert list(valid[1, :4]) == [0, 0, 0, 0]
    assert res["stats"]["n_valid"] == 48 - 4
    assert res["stats"]["n_gated"] == 48 - 4 - 2
    # u16 depth: 0 is the only invalid code
    rig16 = S.tiny_rig(n=1, width=8, height=6)
    d16 = np.full((6, 8), 1500, np.uint16)
    d16[2, 2] = 0
    d16[2, 3] = 1
    fr16 = S.Frame([d16], [np.full((6, 8), 0.9, np.float32)], [np.zeros((6, 8, 3), np.uint8)])
    r16 = oracle_mod.fuse_frame(rig16, fr16, {})
    assert r16["stats"]["n_valid"] == 47
    cam = rig16.cameras[0]
    zc = (cam.R @ r16["pw"].reshape(6, 8, 3)[2, 3] + cam.t)[2]
    assert zc == pytest.approx(0.001, rel=1e-12)        # one depth unit = 1 mm


def test_ablation_switches(oracle_mod):
    rig = S.tiny_rig(n=3, width=16, height=12)
    fr = S.random_frame(rig, seed=3)
    full = oracle_mod.fuse_frame(rig, fr, {})
    noc = oracle_mod.fuse_frame(rig, fr, {"use_consistency": 0})
    nomf = oracle_mod.fuse_frame(rig, fr, {"use_conf": 0})
    conf = np.concatenate([c.ravel() for c in fr.conf]).astype(np.float64)
    g = noc["gated"].astype(bool)
    assert np.all(noc["e"][g] == 0.0)
    np.testing.assert_array_equal(noc["omega"][g], conf[g])
    # without measurement confidence every valid pixel is kept and omega = V
    np.testing.assert_array_equal(nomf["gated"], nomf["valid"])
    gn = nomf["gated"].astype(bool)
    np.testing.assert_allclose(nomf["omega"][gn], np.exp(-nomf["e"][gn]), rtol=1e-15)
    assert full["stats"]["n_gated"] < nomf["stats"]["n_gated"]


# ------------------------------------------------------------------------ Eq. 4-7
def test_single_camera_has_unit_consistency(oracle_mod):
    rig = S.tiny_rig(n=1, width=32, height=24)
    fr = S.random_frame(rig, seed=1)
    res = oracle_mod.fuse_frame(rig, fr, {})
    g = res["gated"].astype(bool)
    assert g.sum() > 100
    assert np.all(res["e"][g] == 0.0)
    assert np.all(res["nview"][g] == 0)
    conf = fr.conf[0].ravel().astype(np.float64)
    np.testing.assert_array_equal(res["omega"][g], conf[g])


def _two_identical(rig1, fr1):
    cam2 = copy.deepcopy(rig1.cameras[0])
    rig2 = S.Rig([rig1.cameras[0], cam2], rig1.depth_format, rig1.depth_scale)
    fr2 = S.Frame(fr1.depth * 2, fr1.conf * 2, fr1.rgb * 2)
    return rig2, fr2


def test_coincident_cameras_fuse_to_single_view(oracle_mod):
    """Two identical cameras with identical images: every point projects onto its own
    pixel, d = 0, V = 1, omega = C; the fused cloud is the single-view cloud with counts
    and weights doubled (density threshold halved so the refinement levels coincide)."""
    rig1 = S.Rig([S.look_at((1.8, -0.6, 1.3), (0, 0, 0.2), 200.0, 190.0, 61.0, 47.0, 120, 90)],
                 "u16", 0.001)
    fr1 = S.random_frame(rig1, seed=7)
    rig2, fr2 = _two_identical(rig1, fr1)
    r1 = oracle_mod.fuse_frame(rig1, fr1, {"n_min": 8})
    r2 = oracle_mod.fuse_frame(rig2, fr2, {"n_min": 16})
    g2 = r2["gated"].astype(bool)
    assert np.all(r2["e"][g2] == 0.0)
    assert np.all(r2["nview"][g2] == 1)
    c1, c2 = r1["cells"], r2["cells"]
    assert len(c1["key"]) == len(c2["key"]) > 50
    np.testing.assert_array_equal(c1["key"], c2["key"])
    np.testing.assert_array_equal(c1["rep"], c2["rep"])        # camera-0 pixel wins the tie
    np.testing.assert_array_equal(2 * c1["count"], c2["count"])
    np.testing.assert_allclose(2 * c1["weight"], c2["weight"], rtol=1e-14)
    np.testing.assert_allclose(c1["pos"], c2["pos"], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(c1["rgb"], c2["rgb"], rtol=1e-14, atol=1e-12)


def _brute_force_consistency(rig, fr, nbr, sigma, K):
    """Eq. 4-7 by exhaustive pixel search with projection matrices and explicit inverses."""
    tab = _pixel_table(rig)
    offs = np.cumsum([0] + [c.width * c.height for c in rig.cameras])
    scale = rig.depth_scale
    out_e, out_n = {}, {}
    for gidx, (i, x, y) in enumerate(tab):
        ci = rig.cameras[i]
        D = float(fr.depth[i][y, x])
        if not (D > 0 and np.isfinite(D)) or not (fr.conf[i][y, x] > np.float32(0.6)):
            continue
        Xw = ci.centre + D * scale * (ci.R.T @ (_kinv(ci) @ np.array([x, y, 1.0])))
        total, nv = 0.0, 0
        for j in nbr[i]:
            cj = rig.cameras[j]
            h = _proj_matrix(cj) @ np.append(Xw, 1.0)
            if not h[2] > 0:
                continue
            u, v = h[0] / h[2], h[1] / h[2]
            yy, xx = np.mgrid[0:cj.height, 0:cj.width]
            dist = np.maximum(np.abs(xx - u), np.abs(yy - v))
            k = np.unravel_index(np.argmin(dist), dist.shape)
            if dist[k] > 0.5:
                continue
            py, px = int(k[0]), int(k[1])
            Dj = float(fr.depth[j][py, px])
            if not (Dj > 0 and np.isfinite(Dj)):
                continue
            Qw = cj.centre + Dj * scale * (cj.R.T @ (_kinv(cj) @ np.array([px, py, 1.0])))
            total += float(np.sum((Xw - Qw) ** 2)) / sigma ** 2
            nv += 1
        out_e[gidx] = total / (K - 1)
        out_n[gidx] = nv
    return out_e, out_n


@pytest.mark.parametrize("n,k_views,zero_frac,seed", [(2, 4, 0.0, 11), (3, 3, 0.25, 12),
                                                      (4, 4, 0.1, 13)])
def test_consistency_matches_brute_force(oracle_mod, n, k_views, zero_frac, seed):
    rig = S.tiny_rig(n=n, width=8, height=6, spread_deg=20.0)
    fr = S.random_frame(rig, seed=seed, zero_frac=zero_frac)
    sigma = 0.05
    res = oracle_mod.fuse_frame(rig, fr, {"k_views": k_views, "sigma_m": sigma})
    nbr = oracle_mod.neighbours(rig, k_views)
    K = min(k_views, n)
    e_bf, n_bf = _brute_force_consistency(rig, fr, nbr, sigma, K)
    g = np.flatnonzero(res["gated"])
    assert set(g.tolist()) == set(e_bf.keys()) and len(g) > 20
    used = 0
    for idx in g:
        if res["margin_tie_px"][idx] < 1e-6:
            continue
        assert res["nview"][idx] == n_bf[idx]
        assert res["e"][idx] == pytest.approx(e_bf[idx], rel=1e-9, abs=1e-12)
        used += n_bf[idx]
    assert used > 10


def test_neighbour_table_on_symmetric_ring(oracle_mod):
    rig = S.ring_rig(4, 3.0, 1.5, 525.0, 525.0, 320.0, 240.0, 640, 480, start_deg=45.0)
    nb = oracle_mod.neighbours(rig, 4)
    # 90 deg apart on a ring: the two adjacent cameras tie on angle and distance -> index
    assert nb.tolist() == [[1, 3, 2], [0, 2, 3], [1, 3, 0], [0, 2, 1]]
    assert oracle_mod.neighbours(rig, 2).tolist() == [[1], [0], [1], [0]]
    assert oracle_mod.neighbours(rig, 1).shape == (4, 0)


def test_neighbour_table_generic(oracle_mod):
    rig = S.fibonacci_rig(9, 5.0, 100.0, 64)
    nb = oracle_mod.neighbours(rig, 4)
    axes = np.stack([c.R[2] for c in rig.cameras])
    ctr = np.stack([c.centre for c in rig.cameras])
    for i in range(9):
        cand = []
        for j in range(9):
            if j == i:
                continue
            ang = np.arccos(np.clip(axes[i] @ axes[j], -1, 1))
            cand.append((round(ang, 9), round(float(np.linalg.norm(ctr[i] - ctr[j])), 9), j))
        cand.sort()
        assert nb[i].tolist() == [c[2] for c in cand[:3]]


# ------------------------------------------------------------------------ Sec. II.5(1)
def _coarse_level(n_c, n_min, lmax):
    q = n_c // n_min
    return 0 if q < 1 else min(lmax, (int(q).bit_length() - 1) // 2)


@pytest.mark.parametrize("count,level", [(31, 0), (32, 0), (127, 0), (128, 1), (511, 1),
                                         (512, 2), (1000, 2)])
def test_level_thresholds_on_a_controlled_patch(oracle_mod, count, level):
    """A camera looking straight down at a flat patch inside one coarse cell; zeroing
    depth pixels fixes the coarse count n_c exactly, and the level must follow n_min 4^l."""
    cam = S.look_at((0.16, 0.16, 1.05), (0.16, 0.16, 0.05), 4000.0, 4000.0, 15.5, 15.5, 32, 32,
                    up=(0, 1, 0))
    rig = S.Rig([cam], "f32", 1.0)
    depth = np.zeros((32, 32), np.float32)
    depth.ravel()[:count] = 1.0
    fr = S.Frame([depth], [np.full((32, 32), 0.9, np.float32)], [np.zeros((32, 32, 3), np.uint8)])
    res = oracle_mod.fuse_frame(rig, fr, {"n_min": 32, "max_level": 4})
    g = res["gated"].astype(bool)
    assert g.sum() == count
    assert np.all(np.floor(res["pw"][g] / 0.32) == 0)     # one coarse cell
    assert np.all(res["level"][g] == level)
    lv, kx, ky, kz = oracle_mod.key_fields(res["key"][g])
    assert np.all(lv == level)


def test_partition_keys_and_levels(oracle_mod):
    rig, _, fr = S.config1()
    p = {"n_min": 8, "max_level": 4}
    res = oracle_mod.fuse_frame(rig, fr, p)
    st = res["stats"]
    g = res["in_range"].astype(bool)
    assert st["n_gated"] - st["n_out_of_range"] == g.sum()
    # every gated point is in exactly one cell: counts partition the points
    assert int(res["cells"]["count"].sum()) == g.sum()
    keys = res["key"][g]
    assert np.all(keys != oracle_mod.KEY_NONE)
    assert len(np.unique(keys)) == st["n_cells"]
    pw = res["pw"][g]
    lv, kx, ky, kz = oracle_mod.key_fields(keys)
    k = np.stack([kx, ky, kz], axis=1)
    edge = 0.32 / 2.0 ** lv
    # the cell is the lattice cube that contains the point
    assert np.all(pw >= k * edge[:, None] - 1e-12)
    assert np.all(pw < (k + 1) * edge[:, None] + 1e-12)
    # nesting: finer lattices refine the coarse cube
    coarse = np.floor(pw / 0.32).astype(np.int64)
    np.testing.assert_array_equal(k >> lv[:, None], coarse)
    # level of each coarse cell from an independent count
    _, inv, cnt = np.unique(coarse, axis=0, return_inverse=True, return_counts=True)
    expect = np.array([_coarse_level(int(c), 8, 4) for c in cnt])[inv.ravel()]
    np.testing.assert_array_equal(lv, expect)
    assert len(np.unique(lv)) >= 2


def test_pairwise_same_cell_brute_force(oracle_mod):
    rig = S.tiny_rig(n=2, width=12, height=9)
    fr = S.random_frame(rig, seed=5)
    res = oracle_mod.fuse_frame(rig, fr, {"n_min": 2, "max_level": 3, "coarse_cell_m": 0.2})
    g = np.flatnonzero(res["in_range"])
    pw = res["pw"][g]
    coarse = np.floor(pw / 0.2).astype(np.int64)
    n = len(g)
    cnt = np.array([np.sum(np.all(coarse == coarse[a], axis=1)) for a in range(n)])
    lev = np.array([_coarse_level(int(c), 2, 3) for c in cnt])
    for a in range(n):
        for b in range(a + 1, n):
            same_coarse = np.all(coarse[a] == coarse[b])
            same = same_coarse and np.all(np.floor(pw[a] / 0.2 * 2.0 ** lev[a]) ==
                                          np.floor(pw[b] / 0.2 * 2.0 ** lev[b]))
            assert same == (res["key"][g[a]] == res["key"][g[b]])


def test_out_of_range_points_are_dropped_and_counted(oracle_mod):
    rig = S.tiny_rig(n=1, width=8, height=6, depth_format="f32", depth_scale=1.0)
    depth = np.full((6, 8), 2.0, np.float32)
    depth[0, :3] = 1.0e6          # ~1000 km away: beyond 2^19 cells of 2 cm
    fr = S.Frame([depth], [np.full((6, 8), 0.9, np.float32)], [np.zeros((6, 8, 3), np.uint8)])
    res = oracle_mod.fuse_frame(rig, fr, {})
    assert res["stats"]["n_out_of_range"] == 3
    assert int(res["cells"]["count"].sum()) == 45
    assert np.all(res["key"].reshape(6, 8)[0, :3] == oracle_mod.KEY_NONE)


# ------------------------------------------------------------------------ Sec. II.5(2)-(3)
def _members(res, rig):
    g = np.flatnonzero(res["in_range"])
    order = np.argsort(res["key"][g], kind="stable")
    return g[order], res["key"][g[order]]


def test_fusion_weights_hull_and_representative(oracle_mod):
    rig, _, fr = S.config1()
    res = oracle_mod.fuse_frame(rig, fr, {"n_min": 8})
    cells = res["cells"]
    g, keys = _members(res, rig)
    conf = np.concatenate([c.ravel() for c in fr.conf])
    rgb = np.concatenate([r.reshape(-1, 3) for r in fr.rgb]).astype(np.float64)
    # weight sums: sum over cells of W = sum over points of omega
    assert cells["weight"].sum() == pytest.approx(res["omega"][g].sum(), rel=1e-12)
    # output order: representative index ascending
    assert np.all(np.diff(cells["rep"].astype(np.int64)) > 0)
    pos_of = {int(k): i for i, k in enumerate(cells["key"])}
    starts = np.flatnonzero(np.r_[True, keys[1:] != keys[:-1]])
    ends = np.r_[starts[1:], len(keys)]
    n_single = 0
    for s, e in zip(starts, ends):
        mem = g[s:e]
        c = pos_of[int(keys[s])]
        assert cells["count"][c] == len(mem)
        # representative: largest C, ties to the lowest index (brute force)
        best = max(mem, key=lambda q: (conf[q], -q))
        assert cells["rep"][c] == best
        w = res["omega"][mem]
        P = res["pw"][mem]
        lo, hi = P.min(axis=0), P.max(axis=0)
        assert np.all(cells["pos"][c] >= lo - 1e-12) and np.all(cells["pos"][c] <= hi + 1e-12)
        if len(mem) == 1:
            n_single += 1
            np.testing.assert_array_equal(cells["pos"][c], P[0])
            np.testing.assert_array_equal(cells["rgb"][c], rgb[mem[0]])
        if w.sum() > 1e-200:
            np.testing.assert_allclose(cells["pos"][c], (w[:, None] * P).sum(0) / w.sum(),
                                       rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(cells["rgb"][c], (w[:, None] * rgb[mem]).sum(0) / w.sum(),
                                       rtol=1e-12, atol=1e-10)
        lv, kx, ky, kz = oracle_mod.key_fields(np.array([keys[s]]))
        edge = 0.32 / 2.0 ** lv[0]
        k = np.array([kx[0], ky[0], kz[0]])
        assert np.all(cells["pos"][c] >= k * edge - 1e-12)
        assert np.all(cells["pos"][c] < (k + 1) * edge + 1e-12)
    assert n_single > 0


def test_fusion_defined_when_all_weights_underflow(oracle_mod):
    """With a tiny sigma every omega underflows to 0 in FP64; Eq. 11's normalised mean is
    still defined (weights relative to the cell's largest) and lies in the member hull."""
    rig = S.tiny_rig(n=3, width=24, height=18)
    fr = S.random_frame(rig, seed=9)
    res = oracle_mod.fuse_frame(rig, fr, {"sigma_m": 1e-6, "n_min": 4})
    g = np.flatnonzero(res["in_range"])
    assert np.mean(res["omega"][g] == 0.0) > 0.5
    cells = res["cells"]
    assert np.all(np.isfinite(cells["pos"])) and np.all(np.isfinite(cells["rgb"]))
    gg, keys = _members(res, rig)
    pos_of = {int(k): i for i, k in enumerate(cells["key"])}
    starts = np.flatnonzero(np.r_[True, keys[1:] != keys[:-1]])
    ends = np.r_[starts[1:], len(keys)]
    for s, e in zip(starts, ends):
        mem = gg[s:e]
        c = pos_of[int(keys[s])]
        P = res["pw"][mem]
        assert np.all(cells["pos"][c] >= P.min(0) - 1e-12)
        assert np.all(cells["pos"][c] <= P.max(0) + 1e-12)
        # the member of largest log-weight dominates: exact mean over the maximisers
        lw = res["log_omega"][mem]
        top = lw >= lw.max() - 1e-300
        if np.all(lw[~top] < lw.max() - 800):
            np.testing.assert_allclose(cells["pos"][c], P[top].mean(0), rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------------ paper constants
def test_paper_constants(oracle_mod):
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        const = json.load(f)
    p = oracle_mod.default_params()
    assert p["tau"] == np.float32(const["tau"]["value"])


def test_golden_tiny_frame(oracle_mod):
    """Regression fixture written by tests/golden/make_golden.py from the oracle alone."""
    with open(os.path.join(GOLDEN, "tiny_frame_cells.json")) as f:
        gold = json.load(f)
    rig = S.tiny_rig(**gold["rig"])
    fr = S.random_frame(rig, seed=gold["seed"])
    res = oracle_mod.fuse_frame(rig, fr, gold["params"])
    cells = res["cells"]
    assert [str(int(k)) for k in cells["key"]] == gold["key"]
    assert cells["count"].tolist() == gold["count"]
    assert cells["rep"].tolist() == gold["rep"]
    np.testing.assert_allclose(cells["weight"], gold["weight"], rtol=1e-12)
    np.testing.assert_allclose(cells["pos"], gold["pos"], rtol=1e-12, atol=1e-15)
    for k in ("n_valid", "n_gated", "n_cells"):
        assert res["stats"][k] == gold["stats"][k]


# ------------------------------------------------------------------ Eq. 12 (MC error)
def _down_camera(x0, h, f=100.0, w=64, hgt=48):
    """Camera at (x0, 0, h) looking straight down: x_cam = (x - x0, -y, h - z)."""
    R = np.diag([1.0, -1.0, -1.0])
    t = -R @ np.array([x0, 0.0, h])
    return S.Camera(f, f, (w - 1) / 2, (hgt - 1) / 2, w, hgt, R, t)


def test_mc_error_of_offsets_above_a_fronto_parallel_plane(oracle_mod):
    """Depth 2 m everywhere under a camera 2 m above z = 0: a point at height d has
    z(T P) = 2 - d, so its MC error is |d| exactly; points behind the camera, outside the
    image or over an invalid depth sample are not visible and leave the mean."""
    cam = _down_camera(0.0, 2.0)
    rig = S.Rig([cam], "u16", 0.001)
    depth = np.full((48, 64), 2000, np.uint16)
    depth[0, 0] = 0                                   # invalid sample at pixel (0, 0)
    corner = np.array([(0 - cam.cx) / cam.fx, -(0 - cam.cy) / cam.fy]) * 2.0
    pts = np.array([[0.10, 0.05, 0.01], [-0.20, 0.10, 0.02], [0.0, 0.0, -0.03],
                    [0.1, 0.1, 3.0],                  # behind the camera
                    [50.0, 0.0, 0.0],                 # outside the image
                    [corner[0], corner[1], 0.0]])     # lands on the invalid sample
    r = oracle_mod.mc_error(rig, [depth], pts)
    assert list(r["nvis"]) == [1, 1, 1, 0, 0, 0]
    np.testing.assert_allclose(r["err_m"][:3], [0.01, 0.02, 0.03], rtol=0, atol=1e-12)
    assert np.isnan(r["err_m"][3:]).all()
    assert r["n_used"] == 3
    assert abs(r["mc_m"] - 0.02) < 1e-12


def test_mc_error_averages_over_the_visible_cameras(oracle_mod):
    """Two downward cameras whose depth maps read 2.0 m and 2.1 m: a point at height d
    (d > 0) has errors d and 0.1 + d, mean d + 0.05."""
    rig = S.Rig([_down_camera(0.0, 2.0), _down_camera(0.3, 2.0)], "u16", 0.001)
    depth = [np.full((48, 64), 2000, np.uint16), np.full((48, 64), 2100, np.uint16)]
    pts = np.array([[0.15, 0.0, 0.01], [0.15, 0.05, 0.04]])
    r = oracle_mod.mc_error(rig, depth, pts)
    assert list(r["nvis"]) == [2, 2]
    np.testing.assert_allclose(r["err_m"], [0.06, 0.09], rtol=0, atol=1e-12)
    assert abs(r["mc_m"] - 0.075) < 1e-12


def test_mc_error_of_a_noiseless_fused_plane_is_zero(oracle_mod):
    """Two downward cameras over the plane z = 0 with exact depth: every fused point lies on
    the plane, so Eq. 12 gives 0 for the fused cloud."""
    rig = S.Rig([_down_camera(0.0, 2.0), _down_camera(0.2, 2.0)], "u16", 0.001)
    depth = [np.full((48, 64), 2000, np.uint16) for _ in range(2)]
    conf = [np.full((48, 64), 0.9, np.float32) for _ in range(2)]
    rgb = [np.zeros((48, 64, 3), np.uint8) for _ in range(2)]
    out = oracle_mod.fuse_frame(rig, S.Frame(depth, conf, rgb), {"n_min": 4}, points=False)
    pos = out["cells"]["pos"]
    assert len(pos) > 10
    r = oracle_mod.mc_error(rig, depth, pos)
    assert r["n_used"] == len(pos)
    assert r["mc_m"] < 1e-12


def test_mc_error_skips_points_hidden_behind_the_observed_surface(oracle_mod):
    """A point 0.1 m under the plane lies 0.1 m behind the surface the camera sees: beyond a
    0.05 m occlusion margin it is not visible; with no occlusion test its error is 0.1 m."""
    rig = S.Rig([_down_camera(0.0, 2.0)], "u16", 0.001)
    depth = [np.full((48, 64), 2000, np.uint16)]
    pts = np.array([[0.1, 0.0, -0.1], [0.1, 0.0, -0.04]])
    r = oracle_mod.mc_error(rig, depth, pts, occlusion_m=0.05)
    assert list(r["nvis"]) == [0, 1] and abs(r["mc_m"] - 0.04) < 1e-12
    r = oracle_mod.mc_error(rig, depth, pts, occlusion_m=np.inf)
    assert list(r["nvis"]) == [1, 1] and abs(r["mc_m"] - 0.07) < 1e-12


# ------------------------------------------------------------------ Eq. 3 (confidence)
def test_confidence_of_a_constant_depth_is_one(oracle_mod):
    d = np.full((7, 9), 2500, np.uint16)
    c = oracle_mod.confidence(d, "u16", 0.001)
    np.testing.assert_allclose(c, 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1])
def test_confidence_of_a_linear_ramp_has_closed_form(oracle_mod, axis):
    """z = 2 + b t along one image axis: the central difference is exactly b, every interior
    3x3 window holds b (-1, 0, 1) three times (population variance 2 b^2 / 3), border pixels
    use one-sided differences (still b) and their 2x3 windows (variance b^2 / 4)."""
    b = 0.004                                          # 4 mm per pixel
    h, w = 6, 8
    t = np.arange(w if axis == 0 else h)
    ramp = 2000 + 4 * t                                # millimetres
    d = np.tile(ramp, (h, 1)) if axis == 0 else np.tile(ramp[:, None], (1, w))
    c = oracle_mod.confidence(d.astype(np.uint16), "u16", 0.001)
    a_, be, ga, de = 0.5, 0.5, 1.0, 1.0
    f = lambda var: (a_ / (1 + be * b) + ga / (1 + de * var)) / (a_ + ga)
    interior = c[1:-1, 1:-1]
    np.testing.assert_allclose(interior, f(2 * b * b / 3), rtol=1e-13)
    edge = c[1:-1, 0] if axis == 0 else c[0, 1:-1]     # first column / row along the ramp
    np.testing.assert_allclose(edge, f(b * b / 4), rtol=1e-13)


def test_confidence_of_invalid_and_isolated_pixels(oracle_mod):
    """Invalid depth gives C = 0; a valid pixel with no valid neighbour has G = 0 and a
    one-sample window (variance 0), so C = 1; the paper's constants keep C in [0, 1]."""
    d = np.zeros((5, 5), np.float32)
    d[2, 2] = 1.7
    c = oracle_mod.confidence(d, "f32", 1.0)
    assert c[2, 2] == 1.0 and c.sum() == 1.0
    rng = np.random.default_rng(3)
    noisy = rng.uniform(0.5, 8.0, size=(40, 50)).astype(np.float32)
    noisy[rng.random((40, 50)) < 0.1] = 0.0
    c = oracle_mod.confidence(noisy, "f32", 1.0)
    assert c.min() >= 0.0 and c.max() <= 1.0 and (c[noisy == 0] == 0).all()
    # a depth step lowers the confidence on both sides of the edge
    step = np.full((6, 10), 2000, np.uint16)
    step[:, 5:] = 3000
    c = oracle_mod.confidence(step, "u16", 0.001)
    assert c[3, 4] < 0.9 and c[3, 5] < 0.9 and c[3, 0] == 1.0 and c[3, 9] == 1.0


# ------------------------------------------------------------------ Sec. II.5(2)a top-k variant
def _topk_case():
    rig = S.tiny_rig(n=3, width=40, height=30, spread_deg=20.0)
    fr = S.random_frame(rig, seed=41, zero_frac=0.02)
    return rig, fr


def test_top_k_fuses_the_k_most_confident_members(oracle_mod):
    """Brute force over the oracle's per-point outputs: each cell's W, position and colour
    come from its top-3 members by C (ties to the lowest pixel index); count, key and
    representative are those of the full cell."""
    rig, fr = _topk_case()
    full = oracle_mod.fuse_frame(rig, fr, {"n_min": 2})
    top = oracle_mod.fuse_frame(rig, fr, {"n_min": 2, "top_k": 3})
    assert np.array_equal(full["cells"]["key"], top["cells"]["key"])
    assert np.array_equal(full["cells"]["count"], top["cells"]["count"])
    assert np.array_equal(full["cells"]["rep"], top["cells"]["rep"])
    conf = np.concatenate([c.ravel() for c in fr.conf])
    rgb = np.concatenate([c.reshape(-1, 3) for c in fr.rgb]).astype(np.float64)
    key, pw, om = top["key"], top["pw"], top["omega"]
    n_multi = 0
    for c, k in enumerate(top["cells"]["key"]):
        g = np.nonzero(key == k)[0]
        order = sorted(g, key=lambda q: (-conf[q], q))[:3]
        n_multi += len(g) > 3
        w = om[order]
        assert abs(top["cells"]["weight"][c] - w.sum()) <= 1e-12 * max(1.0, w.sum())
        if w.sum() > 0:
            np.testing.assert_allclose(top["cells"]["pos"][c], (w[:, None] * pw[order]).sum(0) / w.sum(),
                                       rtol=0, atol=1e-12)
            np.testing.assert_allclose(top["cells"]["rgb"][c], (w[:, None] * rgb[order]).sum(0) / w.sum(),
                                       rtol=0, atol=1e-9)
    assert n_multi > 20                                   # cells where the selection matters


def test_top_k_limits(oracle_mod):
    """top_k = 1 fuses the representative alone; top_k at least the largest cell is the
    full method."""
    rig, fr = _topk_case()
    full = oracle_mod.fuse_frame(rig, fr, {"n_min": 2})
    one = oracle_mod.fuse_frame(rig, fr, {"n_min": 2, "top_k": 1})
    big = oracle_mod.fuse_frame(rig, fr, {"n_min": 2, "top_k": int(full["cells"]["count"].max())})
    for k in ("pos", "weight", "rgb"):
        np.testing.assert_array_equal(big["cells"][k], full["cells"][k])
    rep = one["cells"]["rep"]
    np.testing.assert_array_equal(one["cells"]["pos"], one["pw"][rep])
    np.testing.assert_allclose(one["cells"]["weight"], one["omega"][rep], rtol=1e-15)
