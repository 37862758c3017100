"""Pins of the consensus-term and pruning oracles (oracle/consensus.py) to
facts that do not come from the oracle itself: SSIM identities and closed
forms, a brute-force per-pixel SSIM, central finite differences of the SSIM
and loss adjoints, exact pose recovery and the closed-form (SVD) rigid
alignment for the Mahalanobis step, an independent rotation library, and hand
cases at the pruning thresholds."""
import math

import numpy as np
import pytest

import oracle
from oracle import consensus as C
from paper_2412_09723_gb300 import scenes


def _imgs(seed, H=9, W=8, ch=3):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (H, W, ch))
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1)
    return x, y


# ---------------------------------------------------------------------------
# SSIM
# ---------------------------------------------------------------------------
def test_window_is_normalised_gaussian():
    w = C.ssim_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w, w.T, atol=0)
    np.testing.assert_allclose(w, w[::-1, ::-1], atol=0)
    # neighbouring taps along an axis differ by exp(-(2k+1) / (2 sigma^2))
    for k in range(5):
        assert abs(w[5, 5 + k + 1] / w[5, 5 + k] - math.exp(-(2 * k + 1) / (2 * 1.5 ** 2))) < 1e-12


def test_ssim_of_identical_images_is_one_and_stationary():
    x, _ = _imgs(1)
    assert abs(C.ssim(x, x) - 1.0) < 1e-12
    assert np.abs(C.ssim_grad(x, x)).max() < 1e-12


def test_ssim_constant_images_closed_form():
    a, b = 0.3, 0.7
    x = np.full((30, 31, 1), a)
    y = np.full((30, 31, 1), b)
    s = C.ssim_parts(x, y)["s"]
    want = (2 * a * b + C.SSIM_C1) / (a * a + b * b + C.SSIM_C1)
    np.testing.assert_allclose(s[5:-5, 5:-5], want, rtol=1e-12)  # full windows
    # at a corner only the 6 x 6 in-image part of the window carries weight
    w = C.ssim_window()[5:, 5:].sum()
    mx, my = a * w, b * w
    vx, vy, cxy = a * a * w - mx * mx, b * b * w - my * my, a * b * w - mx * my
    corner = ((2 * mx * my + C.SSIM_C1) * (2 * cxy + C.SSIM_C2)) / ((mx * mx + my * my + C.SSIM_C1) * (vx + vy + C.SSIM_C2))
    assert abs(s[0, 0, 0] - corner) < 1e-12


def test_ssim_brute_force_per_pixel():
    x, y = _imgs(2, 6, 7, 2)
    r = np.arange(-5, 6)
    g = np.exp(-r.astype(float) ** 2 / 4.5)
    tot = g.sum() ** 2
    H, W, ch = x.shape
    vals = []
    for c in range(ch):
        for i in range(H):
            for j in range(W):
                sx = sy = sxx = syy = sxy = 0.0
                for di in range(-5, 6):
                    for dj in range(-5, 6):
                        ii, jj = i + di, j + dj
                        if 0 <= ii < H and 0 <= jj < W:
                            wt = g[di + 5] * g[dj + 5] / tot
                            u, v = x[ii, jj, c], y[ii, jj, c]
                            sx += wt * u
                            sy += wt * v
                            sxx += wt * u * u
                            syy += wt * v * v
                            sxy += wt * u * v
                num = (2 * sx * sy + 1e-4) * (2 * (sxy - sx * sy) + 9e-4)
                den = (sx * sx + sy * sy + 1e-4) * ((sxx - sx * sx) + (syy - sy * sy) + 9e-4)
                vals.append(num / den)
    assert abs(np.mean(vals) - C.ssim(x, y)) < 1e-13


def _fd_grad(f, x, idx, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp[idx] += h
    xm[idx] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_ssim_adjoint_finite_differences():
    x, y = _imgs(3)
    g = C.ssim_grad(x, y)
    rng = np.random.default_rng(0)
    for _ in range(40):
        idx = tuple(int(rng.integers(0, s)) for s in x.shape)
        fd = _fd_grad(lambda z: C.ssim(z, y), x, idx)
        assert abs(fd - g[idx]) <= 1e-7 + 1e-6 * abs(fd), (idx, fd, g[idx])


def test_ssim_planted_mistake_fails_fd():
    """Dropping the factor 2 of the E[x^2] term is caught."""
    x, y = _imgs(4)
    p = C.ssim_parts(x, y)
    cd = p["c"] * p["d"]
    A = (2 * p["my"] * p["b"] - 2 * p["my"] * p["a"]) / cd - p["s"] * (2 * p["mx"] / p["c"] - 2 * p["mx"] / p["d"])
    wrong = (C.window_sum(A) + x * C.window_sum(-p["s"] / p["d"]) + y * C.window_sum(2 * p["a"] / cd)) / x.size
    bad = 0
    for idx in [(1, 1, 0), (4, 3, 1), (7, 6, 2), (0, 5, 1)]:
        fd = _fd_grad(lambda z: C.ssim(z, y), x, idx)
        bad += abs(fd - wrong[idx]) > 1e-7 + 1e-6 * abs(fd)
    assert bad >= 3


def test_paper_loss_gradients_finite_differences():
    rgb, t_rgb = _imgs(5)
    rng = np.random.default_rng(6)
    depth = rng.uniform(1, 3, rgb.shape[:2])
    t_depth = depth + rng.normal(0, 0.1, depth.shape)
    L, S, g_rgb, g_depth = C.paper_loss(rgb, depth, t_rgb, t_depth)
    want = 0.8 * np.abs(rgb - t_rgb).mean() + 0.2 * (1 - S) + 0.1 * np.abs(depth - t_depth).mean()
    assert abs(L - want) < 1e-15
    for idx in [(0, 0, 0), (3, 4, 1), (8, 7, 2)]:
        fd = _fd_grad(lambda z: C.paper_loss(z, depth, t_rgb, t_depth)[0], rgb, idx)
        assert abs(fd - g_rgb[idx]) < 1e-7
    for idx in [(0, 0), (5, 2)]:
        fd = _fd_grad(lambda z: C.paper_loss(rgb, z, t_rgb, t_depth)[0], depth, idx)
        assert abs(fd - g_depth[idx]) < 1e-7


# ---------------------------------------------------------------------------
# Mahalanobis alignment
# ---------------------------------------------------------------------------
def test_covariances_match_independent_rotation():
    from scipy.spatial.transform import Rotation

    sc = scenes.scene_uniform(50, 7)
    cov = C.covariances(sc.log_scale, sc.quat)
    R = Rotation.from_quat(sc.quat[:, [1, 2, 3, 0]].astype(np.float64)).as_matrix()
    s2 = np.exp(2 * sc.log_scale.astype(np.float64))
    for i in range(sc.n):
        np.testing.assert_allclose(cov[i], R[i] @ np.diag(s2[i]) @ R[i].T, rtol=1e-10, atol=1e-16)


def _pairs(seed, n=60, noise=0.0):
    rng = np.random.default_rng(seed)
    x_k = rng.uniform(-1, 1, (n, 3)) + np.array([0, 0, 2.0])
    T_true = C.se3_exp(np.concatenate([rng.normal(0, 0.1, 3), rng.normal(0, 0.12, 3)]))  # orthonormal in float64
    x_l = x_k @ T_true[:3, :3].T + T_true[:3, 3] + rng.normal(0, noise, (n, 3))
    sc_k, sc_l = scenes.scene_uniform(n, seed + 1), scenes.scene_uniform(n, seed + 2)
    cov_k = C.covariances(sc_k.log_scale, sc_k.quat)
    cov_l = C.covariances(sc_l.log_scale, sc_l.quat)
    return x_k, x_l, cov_k, cov_l, T_true


def test_mahalanobis_recovers_exact_transform():
    x_k, x_l, cov_k, cov_l, T_true = _pairs(8)
    T = C.se3_exp([0.006, -0.005, 0.005, 0.005, -0.004, 0.006]) @ T_true  # ~1 cm / 0.5 degrees off
    for _ in range(6):
        T, delta, cost = C.mahalanobis_step(T, x_k, cov_k, x_l, cov_l)
    np.testing.assert_allclose(T, T_true, atol=1e-10)


def test_mahalanobis_isotropic_equals_closed_form_rigid_fit():
    """With every covariance sigma^2 I the objective is point-to-point least
    squares, whose minimiser is the SVD (Kabsch) solution."""
    x_k, x_l, _, _, T_true = _pairs(10, noise=0.01)
    n = len(x_k)
    iso = np.tile(np.eye(3) * 1e-4, (n, 1, 1))
    T = C.se3_exp([0.01, 0.012, -0.01, -0.01, 0.008, 0.01]) @ T_true
    for _ in range(8):
        T, _, _ = C.mahalanobis_step(T, x_k, iso, x_l, iso)
    ck, cl = x_k.mean(0), x_l.mean(0)
    U, _, Vt = np.linalg.svd((x_k - ck).T @ (x_l - cl))
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    np.testing.assert_allclose(T[:3, :3], R, atol=1e-9)
    np.testing.assert_allclose(T[:3, 3], cl - R @ ck, atol=1e-9)


def test_mahalanobis_gradient_and_translation_block():
    """g is the derivative of the cost with M frozen at T; for translations the
    residual is linear, so the Hessian block there equals H[:3, :3]."""
    x_k, x_l, cov_k, cov_l, T_true = _pairs(12, noise=0.02)
    T = scenes.perturbed_w2c(13, 0.03, 2.0, base=T_true).astype(np.float64)
    cost, g, H = C.mahalanobis_system(T, x_k, cov_k, x_l, cov_l)
    R = T[:3, :3]
    Ms = [np.linalg.inv(R @ ck @ R.T + cl) for ck, cl in zip(cov_k, cov_l)]

    def frozen(d):
        Td = C.se3_exp(d) @ T
        r = x_k @ Td[:3, :3].T + Td[:3, 3] - x_l
        return sum(float(ri @ M @ ri) for ri, M in zip(r, Ms))

    assert abs(frozen(np.zeros(6)) - cost) < 1e-9 * cost
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd = (frozen(e) - frozen(-e)) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 * (1 + abs(g[k])), (k, fd, g[k])
    for i in range(3):
        for j in range(3):
            ei, ej = np.zeros(6), np.zeros(6)
            ei[i], ej[j] = 1e-3, 1e-3
            fd2 = (frozen(ei + ej) - frozen(ei - ej) - frozen(-ei + ej) + frozen(-ei - ej)) / (4e-6)
            assert abs(fd2 - H[i, j]) < 1e-6 * (1 + abs(H[i, j]))
    np.testing.assert_allclose(H, H.T, atol=1e-9)
    assert np.linalg.eigvalsh(H).min() > 0


# ---------------------------------------------------------------------------
# Pruning (Algorithm 1)
# ---------------------------------------------------------------------------
def _logit(p):
    return math.log(p / (1 - p))


def test_prune_hand_cases():
    ls = np.log(np.array([
        [0.05, 0.05, 0.05],    # keep
        [0.05, 0.05, 0.05],    # transparent (opacity 0.004)
        [0.30, 0.10, 0.10],    # large
        [0.20, 0.010, 0.009],  # elongated: 0.2 > 10 * 0.019
        [0.20, 0.010, 0.011],  # not elongated: 0.2 < 10 * 0.021
        [0.26, 0.20, 0.20],    # large only
    ], np.float64)).astype(np.float32)
    logit = np.float32([2.0, _logit(0.004), 2.0, 2.0, 2.0, 2.0])
    mask = C.prune_mask(logit, ls, oracle.exp_f32)
    assert mask.tolist() == [False, True, True, True, False, True]
    # tau_s unset: only the opacity criterion (Algorithm 1, the conditional block)
    assert C.prune_mask(logit, ls, oracle.exp_f32, tau_s=None).tolist() == [False, True, False, False, False, False]


def test_prune_mask_agrees_with_float64_definition_away_from_thresholds():
    rng = np.random.default_rng(14)
    n = 200000
    logit = rng.normal(-3.0, 2.5, n).astype(np.float32)
    ls = rng.normal(-3.0, 1.2, (n, 3)).astype(np.float32)
    got = C.prune_mask(logit, ls, oracle.exp_f32)
    lam = 1 / (1 + np.exp(-logit.astype(np.float64)))
    s = np.exp(ls.astype(np.float64))
    mx = s.max(1)
    other = s.sum(1) - mx
    want = (lam < 0.005) | (mx > 0.25) | (mx > 10 * other)
    near = (np.abs(lam / 0.005 - 1) < 1e-5) | (np.abs(mx / 0.25 - 1) < 1e-5) | (np.abs(mx / (10 * other) - 1) < 1e-5)
    assert np.array_equal(got[~near], want[~near])
    assert 0.05 < got.mean() < 0.95  # every criterion is exercised


def test_prune_keeps_order_and_moves_rows_together():
    rng = np.random.default_rng(15)
    a = rng.normal(size=(10, 3))
    b = np.arange(10)
    mask = np.array([0, 1, 0, 0, 1, 1, 0, 0, 0, 1], bool)
    a2, b2 = C.prune([a, b], mask)
    assert b2.tolist() == [0, 2, 3, 6, 7, 8]
    np.testing.assert_array_equal(a2, a[b2])


def test_mahalanobis_distance_threshold_drops_far_pairs():
    """Pairs beyond max_dist contribute nothing: the system equals the one
    built from the near pairs alone, and outliers beyond it cannot bias the
    exact recovery."""
    x_k, x_l, cov_k, cov_l, T_true = _pairs(16)
    T = C.se3_exp([0.004, -0.003, 0.002, 0.002, -0.001, 0.002]) @ T_true
    rng = np.random.default_rng(17)
    out = rng.choice(len(x_k), 15, replace=False)
    x_bad = x_l.copy()
    x_bad[out] += rng.normal(0, 0.3, (15, 3)) + 0.2  # gross outliers, far beyond 2 cm
    r = np.linalg.norm(x_k @ T[:3, :3].T + T[:3, 3] - x_bad, axis=1)
    near = r <= 0.02
    assert near.sum() == len(x_k) - 15
    full = C.mahalanobis_system(T, x_k, cov_k, x_bad, cov_l, max_dist=0.02)
    ref = C.mahalanobis_system(T, x_k[near], cov_k[near], x_bad[near], cov_l[near])
    for a, b in zip(full, ref):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    for _ in range(5):
        T, _, _ = C.mahalanobis_step(T, x_k, cov_k, x_bad, cov_l, max_dist=0.02)
    np.testing.assert_allclose(T, T_true, atol=1e-10)
