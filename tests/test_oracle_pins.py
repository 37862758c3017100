"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, hand-computed composites of the rendering equation (Sec. 3.3),
invariants, brute force and an independent rotation library."""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

from paper_2412_09723_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _logit(lam):
    return math.log(lam / (1.0 - lam))


def _coincident_scene(depths, lams, rgbs, scale=0.01):
    n = len(depths)
    return scenes.Scene(
        mean=np.array([[0.0, 0.0, z] for z in depths]),
        log_scale=np.full((n, 3), math.log(scale)),
        quat=np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (n, 1)),
        opacity_logit=np.array([_logit(l) for l in lams]),
        rgb=np.array(rgbs, dtype=np.float64),
    )


# ---------------------------------------------------------------------------
# project exp (Cody & Waite + Taylor): error bound against the true exp
# ---------------------------------------------------------------------------
def test_exp_within_one_ulp(orc):
    x = np.linspace(-87.0, 88.0, 400_001).astype(np.float32)
    x = np.concatenate([x, np.float32([0.0, -1e-30, 1e-30, -0.5, 0.5, -5.5413, -80.0])])
    y = orc.exp_f32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(y - ref) / ulp) <= 1.0
    assert orc.exp_f32(np.float32([0.0]))[0] == 1.0


def test_exp_special_values(orc):
    y = orc.exp_f32(np.float32([np.nan, 88.5, np.inf, -87.5, -np.inf]))
    assert np.isnan(y[0]) and y[1] == np.inf and y[2] == np.inf and y[3] == 0.0 and y[4] == 0.0


# ---------------------------------------------------------------------------
# single isotropic Gaussian on the optical axis: closed form
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 2e-6)])
def test_single_isotropic_closed_form(orc, dtype, tol):
    cam = scenes.Camera(40, 30, 80.0, 80.0, 20.0, 15.0)
    z, s, lam = 2.0, 0.05, 0.7
    sc = _coincident_scene([z], [lam], [[0.9, 0.4, 0.1]], scale=s).astype(dtype)
    w2c = np.eye(4)
    var = (cam.fx * s / z) ** 2 + 0.3  # EWA at the axis: J = diag(f/z), Sigma = s^2 I
    pr = orc.project(sc, w2c, cam, dtype=dtype)
    assert pr["xyzo"][0, :2] == pytest.approx([cam.cx, cam.cy], abs=tol * 10)
    assert pr["xyzo"][0, 2] == pytest.approx(z, rel=tol)
    assert pr["xyzo"][0, 3] == pytest.approx(lam, rel=tol * 10)
    assert pr["conic"][0, :3] == pytest.approx([1 / var, 0.0, 1 / var], rel=tol * 10, abs=tol)
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(var))
    out = orc.render_fwd(sc, w2c, cam, np.zeros(3), dtype=dtype)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    d2 = (xs + 0.5 - cam.cx) ** 2 + (ys + 0.5 - cam.cy) ** 2
    alpha = np.minimum(0.99, lam * np.exp(-0.5 * d2 / var))
    # pixels inside the tile rectangle with alpha above the floor composite one Gaussian
    r = pr["rect"][0]
    in_rect = (xs // 16 >= r[0]) & (xs // 16 < r[2]) & (ys // 16 >= r[1]) & (ys // 16 < r[3])
    on = in_rect & (alpha >= 1 / 255)
    expect_a = np.where(on, alpha, 0.0)
    np.testing.assert_allclose(out["sil"], expect_a, atol=tol * 10)
    np.testing.assert_allclose(out["t_final"], 1 - expect_a, atol=tol * 10)
    np.testing.assert_allclose(out["depth"], z * expect_a, atol=tol * 20)
    np.testing.assert_allclose(out["rgb"], expect_a[..., None] * np.array([0.9, 0.4, 0.1]), atol=tol * 10)
    # away from the floor the membership decision is unambiguous
    clear = np.abs(alpha - 1 / 255) > 1e-4
    assert np.array_equal(out["max_id"][clear], np.where(on, 0, -1)[clear])
    assert np.array_equal(out["n_contrib"][clear], np.where(on, 1, 0)[clear])


# ---------------------------------------------------------------------------
# hand-computed 2- and 3-Gaussian composites (tests/golden/composite_cases.json)
# ---------------------------------------------------------------------------
def _golden_cases():
    with open(os.path.join(GOLDEN, "composite_cases.json")) as f:
        g = json.load(f)
    return g, g["cases"]


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-9), (np.float32, 2e-6)])
@pytest.mark.parametrize("case", range(3))
def test_hand_composites(orc, dtype, tol, case):
    g, cases = _golden_cases()
    c = cases[case]
    cam = scenes.Camera(**g["camera"])
    sc = _coincident_scene(c["depth"], c["lambda"], c["rgb"]).astype(dtype)
    out = orc.render_fwd(sc, np.eye(4), cam, np.array(c["bg"]), dtype=dtype)
    x, y = g["pixel"]
    e = c["expect"]
    np.testing.assert_allclose(out["rgb"][y, x], e["rgb"], atol=tol)
    assert out["depth"][y, x] == pytest.approx(e["depth"], abs=tol * 5)
    assert out["sil"][y, x] == pytest.approx(e["sil"], abs=tol)
    assert out["t_final"][y, x] == pytest.approx(e["t_final"], abs=tol)
    assert out["max_id"][y, x] == e["max_id"]
    assert out["n_contrib"][y, x] == e["n_contrib"]


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_zero_opacity_returns_background(orc, dtype):
    sc, w2c, cam, _ = scenes.workload_small_forward(seed=7)
    sc = sc.subset(slice(0, 300)).astype(dtype)
    sc.opacity_logit[:] = -np.inf
    bg = np.array([0.25, 0.5, 0.75])
    out = orc.render_fwd(sc, w2c, cam, bg, dtype=dtype)
    assert np.all(out["rgb"] == bg.astype(dtype))
    assert np.all(out["t_final"] == 1) and np.all(out["depth"] == 0) and np.all(out["sil"] == 0)
    assert np.all(out["max_id"] == -1) and np.all(out["n_contrib"] == 0)


def test_permutation_invariance(orc):
    sc, w2c, cam, bg = scenes.workload_small_forward(seed=3)
    sc = sc.subset(slice(0, 500)).astype(np.float64)
    perm = np.random.default_rng(0).permutation(sc.n)
    a = orc.render_fwd(sc, w2c, cam, bg, dtype=np.float64)
    b = orc.render_fwd(sc.subset(perm), w2c, cam, bg, dtype=np.float64)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)
    np.testing.assert_allclose(a["depth"], b["depth"], atol=1e-12)
    ida, idb = a["max_id"], b["max_id"]
    mapped = np.where(idb >= 0, perm[np.maximum(idb, 0)], -1)
    assert np.mean(mapped == ida) > 0.999


def test_rigid_motion_invariance(orc):
    """Moving the scene and the camera by the same rigid motion changes nothing."""
    sc, w2c, cam, bg = scenes.workload_small_forward(seed=4)
    sc = sc.subset(slice(0, 400)).astype(np.float64)
    M = scenes.perturbed_w2c(11, trans_m=0.7, rot_deg=25.0).astype(np.float64)
    moved = scenes.Scene(sc.mean @ M[:3, :3].T + M[:3, 3], sc.log_scale.copy(), None, sc.opacity_logit.copy(),
                         sc.rgb.copy())
    # rotate each Gaussian's orientation with the motion: q' = q_M * q
    from scipy.spatial.transform import Rotation

    qm = Rotation.from_matrix(M[:3, :3])
    rot = qm * Rotation.from_quat(sc.quat[:, [1, 2, 3, 0]])
    q = rot.as_quat()
    moved.quat = np.ascontiguousarray(q[:, [3, 0, 1, 2]])
    w2c2 = np.asarray(w2c, np.float64) @ np.linalg.inv(M)
    a = orc.render_fwd(sc, w2c, cam, bg, dtype=np.float64)
    b = orc.render_fwd(moved, w2c2, cam, bg, dtype=np.float64)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-8)
    np.testing.assert_allclose(a["depth"], b["depth"], atol=1e-8)
    assert np.mean(a["max_id"] == b["max_id"]) > 0.999


# ---------------------------------------------------------------------------
# projection: independent rotation library and numerical Jacobian
# ---------------------------------------------------------------------------
def test_ewa_covariance_matches_numerical_linearisation(orc):
    from scipy.spatial.transform import Rotation

    cam = scenes.CAM_VGA
    sc = scenes.scene_room(3000, 9).astype(np.float64)
    w2c = scenes.perturbed_w2c(5, 0.05, 10.0).astype(np.float64)
    pr = orc.project(sc, w2c, cam, dtype=np.float64)
    lim = 1.3 * np.array([cam.width / (2 * cam.fx), cam.height / (2 * cam.fy)])
    pc = sc.mean @ w2c[:3, :3].T + w2c[:3, 3]
    ok = (pr["radius"] > 0) & np.all(np.abs(pc[:, :2] / pc[:, 2:3]) < lim * 0.99, axis=1)
    idx = np.nonzero(ok)[0][:200]
    assert idx.size > 50
    R = Rotation.from_quat(sc.quat[idx][:, [1, 2, 3, 0]]).as_matrix()
    s2 = np.exp(2 * sc.log_scale[idx])
    h = 1e-6
    for k, g in enumerate(idx):
        # numerical Jacobian of the projected centre (u, v) w.r.t. the world mean
        Jn = np.zeros((2, 3))
        for j in range(3):
            sp, sm = sc.subset([g]), sc.subset([g])
            sp.mean[0, j] += h
            sm.mean[0, j] -= h
            up = orc.project(sp, w2c, cam, dtype=np.float64)["xyzo"][0, :2]
            um = orc.project(sm, w2c, cam, dtype=np.float64)["xyzo"][0, :2]
            Jn[:, j] = (up - um) / (2 * h)
        Sig = R[k] @ np.diag(s2[k]) @ R[k].T
        cov = Jn @ Sig @ Jn.T + 0.3 * np.eye(2)
        got = pr["cov"][g]
        np.testing.assert_allclose([got[0], got[1], got[2]], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-6,
                                   atol=1e-6)
        con = pr["conic"][g]
        Q = np.array([[con[0], con[1]], [con[1], con[2]]])
        np.testing.assert_allclose(Q @ cov, np.eye(2), atol=1e-8)
        lmax = np.linalg.eigvalsh(cov)[-1]
        assert pr["radius"][g] == math.ceil(3 * math.sqrt(lmax))


def test_projected_centre_is_pinhole(orc):
    cam = scenes.CAM_SMALL
    sc = scenes.scene_uniform(500, 2).astype(np.float64)
    w2c = scenes.perturbed_w2c(3, 0.1, 5.0).astype(np.float64)
    pr = orc.project(sc, w2c, cam, dtype=np.float64)
    pc = sc.mean @ w2c[:3, :3].T + w2c[:3, 3]
    vis = pr["radius"] > 0
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    np.testing.assert_allclose(pr["xyzo"][vis, 0], u[vis], rtol=1e-12)
    np.testing.assert_allclose(pr["xyzo"][vis, 1], v[vis], rtol=1e-12)
    np.testing.assert_allclose(pr["xyzo"][vis, 2], pc[vis, 2], rtol=1e-12)


def test_near_plane_cull(orc):
    sc = _coincident_scene([0.15, 0.2, 0.25], [0.5, 0.5, 0.5], [[1, 1, 1]] * 3, scale=0.001)
    pr = orc.project(sc, np.eye(4), scenes.CAM_SMALL, dtype=np.float64)
    assert list(pr["radius"] > 0) == [False, False, True]


# ---------------------------------------------------------------------------
# tile membership and order: brute force
# ---------------------------------------------------------------------------
def _tile_min_q(u, v, a, b, c, tx, ty):
    """Minimum of a dx^2 + 2 b dx dy + c dy^2 over the tile's rectangle of
    pixel centres, by dense sampling (65 x 65 points, float64) refined with
    the exact value at the centre when it lies inside."""
    xs = np.linspace(16 * tx + 0.5, 16 * tx + 15.5, 65) - u
    ys = np.linspace(16 * ty + 0.5, 16 * ty + 15.5, 65) - v
    dx, dy = np.meshgrid(xs, ys)
    q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
    if xs[0] <= 0 <= xs[-1] and ys[0] <= 0 <= ys[-1]:
        return 0.0
    return float(q.min())


@pytest.mark.parametrize("seed,w,h", [(0, 40, 35), (1, 64, 48), (2, 17, 90)])
def test_bins_match_brute_force(orc, seed, w, h):
    cam = scenes.Camera(w, h, 60.0, 60.0, w / 2, h / 2)
    sc = scenes.scene_uniform(150, seed)
    pr = orc.project(sc, np.eye(4), cam)
    keys, vals, ranges = orc.bin_sort(sc, np.eye(4), cam)
    xyzo, rad, rect, con = pr["xyzo"], pr["radius"], pr["rect"], pr["conic"]
    # the rectangle covers every tile that holds a pixel centre within the radius box
    for g in np.nonzero(rad > 0)[0]:
        u, v, r = float(xyzo[g, 0]), float(xyzo[g, 1]), int(rad[g])
        xs = np.arange(w) + 0.5
        ys = np.arange(h) + 0.5
        tx = np.unique((xs[(xs >= u - r) & (xs <= u + r)] // 16).astype(int))
        ty = np.unique((ys[(ys >= v - r) & (ys <= v + r)] // 16).astype(int))
        for t in tx:
            assert rect[g, 0] <= t < rect[g, 2]
        for t in ty:
            assert rect[g, 1] <= t < rect[g, 3]
        if tx.size:
            assert rect[g, 2] - rect[g, 0] <= tx.size + 1
    members = {}  # tile -> Gaussians holding it
    for t in range(cam.n_tiles):
        s0, s1 = ranges[t]
        members[t] = set(int(x) for x in vals[s0:s1])
    gx = np.arange(16) + 0.5
    for g in np.nonzero(rad > 0)[0]:
        u, v, lam = float(xyzo[g, 0]), float(xyzo[g, 1]), float(xyzo[g, 3])
        a, b, c = (float(x) for x in con[g, :3])
        for ty_ in range(rect[g, 1], rect[g, 3]):
            row = []
            for tx_ in range(rect[g, 0], rect[g, 2]):
                t = ty_ * cam.tiles_x + tx_
                # soundness: a tile with a pixel centre at alpha >= 1/255 holds the Gaussian
                dx, dy = np.meshgrid(16 * tx_ + gx - u, 16 * ty_ + gx - v)
                alpha = lam * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
                if alpha.max() >= 1 / 255:
                    assert g in members[t], (g, t)
                if g in members[t]:
                    row.append(tx_)
                    reach = lam * np.exp(-0.5 * _tile_min_q(u, v, a, b, c, tx_, ty_)) >= 0.99 / 255 * (1 - 1e-3)
                    row[-1] = (tx_, reach)
            # members of a row are contiguous, and the ones at its ends reach the threshold
            if row:
                xs_ = [x for x, _ in row]
                assert xs_ == list(range(xs_[0], xs_[-1] + 1))
                assert row[0][1] and row[-1][1]
    # per tile: members in ascending (depth bits, gid), flattened in tile order
    k = 0
    for t in range(cam.n_tiles):
        cand = sorted(members[t], key=lambda g: (int(xyzo[g, 2:3].view(np.uint32)[0]), g))
        assert list(vals[k:k + len(cand)]) == cand
        for j, g in enumerate(cand):
            assert int(keys[k + j]) == (t << 32) | int(xyzo[g, 2:3].view(np.uint32)[0])
        if cand:
            assert tuple(ranges[t]) == (k, k + len(cand))
        else:
            assert tuple(ranges[t]) == (0, 0)
        k += len(cand)
    assert k == len(vals) <= int(pr["tiles_touched"].sum())


def test_tile_membership_leaves_the_images_unchanged(orc):
    """Dropping the rect tiles that no pixel can take a Gaussian in changes
    nothing rendered: images, ids and transmittance equal the whole-rect ones,
    and fewer (Gaussian, tile) pairs are walked."""
    sc = scenes.scene_room(6000, 6)
    w2c = scenes.perturbed_w2c(7, 0.2, 10.0)
    cam = scenes.Camera(96, 72, 80.0, 80.0, 48.0, 36.0)
    bg = np.float32([0.1, 0.2, 0.3])
    a = orc.render_fwd(sc, w2c, cam, bg)
    try:
        orc.set_exact_tiles(False)
        b = orc.render_fwd(sc, w2c, cam, bg)
        kb = len(orc.bin_sort(sc, w2c, cam)[1])
    finally:
        orc.set_exact_tiles(True)
    ka = len(orc.bin_sort(sc, w2c, cam)[1])
    for key in ("rgb", "depth", "sil", "t_final", "max_id"):
        assert np.array_equal(a[key], b[key]), key
    assert ka < 0.8 * kb
    assert a["n_pairs"] < b["n_pairs"]


# ---------------------------------------------------------------------------
# loss, Adam, association
# ---------------------------------------------------------------------------
def test_l1_loss_closed_form(orc):
    H, W = 6, 5
    rgb = np.full((H, W, 3), 0.3, np.float32)
    trgb = np.full((H, W, 3), 0.1, np.float32)
    d = np.full((H, W), 2.0, np.float32)
    td = np.full((H, W), 2.5, np.float32)
    L, gr, gd = orc.loss_l1(rgb, d, trgb, td, 1.0, 0.5)
    assert L == pytest.approx(0.2 + 0.5 * 0.5, rel=1e-6)
    assert np.allclose(gr, 1.0 / (3 * H * W)) and np.allclose(gd, -0.5 / (H * W))
    L0, gr0, gd0 = orc.loss_l1(rgb, d, rgb, d, 1.0, 0.5)
    assert L0 == 0.0 and not gr0.any() and not gd0.any()


def test_adam_textbook(orc):
    p, m, v = orc.adam([1.0, -2.0, 0.5], [0.5, -3.0, 0.0], [0, 0, 0], [0, 0, 0], 1, 0.1)
    # first step: m_hat = g, v_hat = g^2, so the step is lr * sign(g)
    np.testing.assert_allclose(p, [0.9, -1.9, 0.5], rtol=1e-6)
    p2, m2, v2 = orc.adam(p, [0.5, -3.0, 0.0], m, v, 2, 0.1)
    mh = (0.9 * 0.05 + 0.1 * 0.5) / (1 - 0.9 ** 2)
    vh = (0.999 * 0.001 * 0.25 + 0.001 * 0.25) / (1 - 0.999 ** 2)
    assert p2[0] == pytest.approx(0.9 - 0.1 * mh / math.sqrt(vh), rel=1e-5)


def test_assoc_brute_force(orc):
    rng = np.random.default_rng(0)
    ia = rng.integers(-1, 20, size=(30, 40)).astype(np.int32)
    ib = rng.integers(-1, 25, size=(30, 40)).astype(np.int32)
    ta = rng.uniform(0, 1, size=(30, 40)).astype(np.float32)
    tb = rng.uniform(0, 1, size=(30, 40)).astype(np.float32)
    pairs, counts = orc.assoc(ia, ta, ib, tb, 0.5)
    ref = {}
    for a, b, x, y in zip(ia.ravel(), ib.ravel(), ta.ravel(), tb.ravel()):
        if a >= 0 and b >= 0 and x <= 0.5 and y <= 0.5:
            ref[(int(a), int(b))] = ref.get((int(a), int(b)), 0) + 1
    keys = sorted(ref)
    assert [tuple(p) for p in pairs] == keys
    assert list(counts) == [ref[k] for k in keys]


def test_assoc_self_is_diagonal(orc):
    sc, w2c, cam, bg = scenes.workload_small_forward()
    out = orc.render_fwd(sc, w2c, cam, bg)
    pairs, counts = orc.assoc(out["max_id"], out["t_final"], out["max_id"], out["t_final"], 0.5)
    assert np.all(pairs[:, 0] == pairs[:, 1])
    vis = (out["max_id"] >= 0) & (out["t_final"] <= 0.5)
    assert counts.sum() == vis.sum()
    assert set(pairs[:, 0]) == set(np.unique(out["max_id"][vis]))


def test_row_band_equals_full_frame_rows(orc):
    """Rendering / differentiating only a band of rows gives exactly the rows
    of the full-frame result (the band is a restriction, not a new computation)."""
    sc, w2c, cam, bg = scenes.workload_small_forward(seed=5)
    full = orc.render_fwd(sc, w2c, cam, bg)
    band = orc.render_fwd(sc, w2c, cam, bg, rows=(32, 64))
    for k in ("rgb", "depth", "sil", "t_final", "n_contrib", "max_id"):
        assert np.array_equal(band[k][32:64], full[k][32:64])
    rng = np.random.default_rng(0)
    g = rng.normal(size=(cam.height, cam.width, 3)).astype(np.float32)
    g[:32] = 0
    g[64:] = 0
    a = orc.render_bwd(sc, w2c, cam, bg, g)
    b = orc.render_bwd(sc, w2c, cam, bg, g, rows=(32, 64))
    for k in ("mean", "opacity_logit", "rgb", "pose"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-5, atol=1e-7)


# ---------------------------------------------------------------------------
# candidate selection by distance (Sec. 3.4 step 1)
# ---------------------------------------------------------------------------
def test_distance_selection_single_gaussian(orc):
    cam = scenes.Camera(64, 48, 60.0, 60.0, 32.0, 24.0)
    sc = scenes.Scene(np.float32([[0.1, -0.05, 2.0]]), np.full((1, 3), -3.0, np.float32),
                      np.float32([[1, 0, 0, 0]]), np.float32([2.0]), np.float32([[1, 0, 0]]))
    d = float(np.sqrt(0.1 ** 2 + 0.05 ** 2 + 2.0 ** 2))
    near = dataclasses.replace(cam, max_dist=d * (1 - 1e-4))
    far = dataclasses.replace(cam, max_dist=d * (1 + 1e-4))
    assert orc.project(sc, np.eye(4, dtype=np.float32), near)["radius"][0] == 0
    assert orc.project(sc, np.eye(4, dtype=np.float32), far)["radius"][0] > 0


def test_distance_selection_equals_rendering_the_selected_subset(orc):
    """Rendering with a distance limit equals rendering, without the limit,
    only the Gaussians whose camera-space distance is within it."""
    sc = scenes.scene_room(4000, 21)
    w2c = scenes.perturbed_w2c(22, 0.3, 20.0)
    cam = scenes.Camera(96, 72, 80.0, 80.0, 48.0, 36.0)
    W = w2c.astype(np.float64)
    dist = np.linalg.norm(sc.mean.astype(np.float64) @ W[:3, :3].T + W[:3, 3], axis=1)
    r = np.sort(dist)
    lo, hi = int(0.3 * len(r)), int(0.7 * len(r))
    j = lo + int(np.argmax(np.diff(r[lo:hi])))
    d = 0.5 * (r[j] + r[j + 1])
    assert r[j + 1] - r[j] > 1e-5
    keep = np.nonzero(dist <= d)[0]
    assert 0.1 < len(keep) / sc.n < 0.9
    a = orc.render_fwd(sc, w2c, dataclasses.replace(cam, max_dist=d), np.zeros(3, np.float32))
    b = orc.render_fwd(sc.subset(keep), w2c, cam, np.zeros(3, np.float32))
    for k in ("rgb", "depth", "sil", "t_final", "n_contrib"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["max_id"], np.where(b["max_id"] >= 0, keep[np.maximum(b["max_id"], 0)], -1))
