"""Plain numpy oracles of the inter-agent consensus terms and of map pruning.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it.  Float64 unless
a decision must be taken in float32 (the pruning mask), where the float32
operations are spelled out one by one.

- Inter-agent loss, Eq. (optim) of Sec. 3.5 step 4, with the weights of
  Sec. 4.1 (lambda_L1 = 0.8, lambda_SSIM = 0.2, lambda_geom = 0.1) and the
  SSIM term read as lambda_SSIM * (1 - SSIM), since the loss is minimised.
  SSIM is the windowed form of the appendix's definition: an 11 x 11 Gaussian
  window (sigma 1.5, normalised to sum 1) gives the local means, variances and
  covariance of every channel, the image is zero outside its border,
  C1 = 0.01^2, C2 = 0.03^2, and SSIM is the mean of the per-pixel, per-channel
  values.
- Mahalanobis alignment, Sec. 3.5 step 3: one Gauss-Newton step of
  sum_(k,l) r^T M r with r = T x_k - x_l over associated pairs, the combined
  covariance M^-1 = R Sigma_k R^T + Sigma_l evaluated at the current T and
  held fixed in the step (with R = I this is the printed Sigma_k + Sigma_l),
  and T <- exp(delta^) T; optionally only pairs within a correspondence
  distance (the G-ICP point-selection threshold of Sec. 4.1, 0.02).
- Pruning, Algorithm 1: opacity below tau_o, or largest scale above tau_s, or
  largest scale above tau_e times the sum of the other two.
"""
from __future__ import annotations

import math

import numpy as np

W_L1, W_SSIM, W_GEOM = 0.8, 0.2, 0.1
SSIM_RADIUS = 5
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


# ---------------------------------------------------------------------------
# SSIM
# ---------------------------------------------------------------------------
def ssim_window():
    """11 x 11 Gaussian window, sigma 1.5, summing to 1 (float64)."""
    r = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    g = np.exp(-(r * r) / (2.0 * SSIM_SIGMA ** 2))
    w = np.outer(g, g)
    return w / w.sum()


def window_sum(img):
    """out(p) = sum_o w(o) img(p + o) over the 11 x 11 offsets o, with img = 0
    outside the image ([H, W] or [H, W, C], float64)."""
    img = np.asarray(img, np.float64)
    w = ssim_window()
    R = SSIM_RADIUS
    H, W = img.shape[:2]
    pad = np.zeros((H + 2 * R, W + 2 * R) + img.shape[2:])
    pad[R:R + H, R:R + W] = img
    out = np.zeros_like(img)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            out += w[dy + R, dx + R] * pad[R + dy:R + dy + H, R + dx:R + dx + W]
    return out


def ssim_parts(x, y):
    """Per-pixel, per-channel local statistics and SSIM values."""
    x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
    mx, my = window_sum(x), window_sum(y)
    exx, eyy, exy = window_sum(x * x), window_sum(y * y), window_sum(x * y)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a = 2.0 * mx * my + SSIM_C1
    b = 2.0 * cxy + SSIM_C2
    c = mx * mx + my * my + SSIM_C1
    d = vx + vy + SSIM_C2
    return dict(mx=mx, my=my, a=a, b=b, c=c, d=d, s=(a * b) / (c * d))


def ssim(x, y):
    """Mean SSIM of two images [H, W, C] (or [H, W])."""
    return float(ssim_parts(x, y)["s"].mean())


def ssim_grad(x, y):
    """d mean-SSIM / d x.  The per-pixel value depends on x through the window
    sums mu_x, E[x^2] and E[xy]; their partial derivatives A, B, C are spread
    back by the same (symmetric) window: dS/dx(q) = [W*A + 2 x(q) W*B + y(q) W*C] / count."""
    x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
    p = ssim_parts(x, y)
    cd = p["c"] * p["d"]
    s = p["s"]
    A = (2.0 * p["my"] * p["b"] - 2.0 * p["my"] * p["a"]) / cd - s * (2.0 * p["mx"] / p["c"] - 2.0 * p["mx"] / p["d"])
    Bm = -s / p["d"]
    Cm = 2.0 * p["a"] / cd
    return (window_sum(A) + 2.0 * x * window_sum(Bm) + y * window_sum(Cm)) / x.size


def paper_loss(rgb, depth, t_rgb, t_depth, w=(W_L1, W_SSIM, W_GEOM)):
    """L = w_L1 mean|C - C*| + w_SSIM (1 - SSIM(C, C*)) + w_geom mean|D - D*|
    and its gradients with respect to C and D (sign(0) = 0)."""
    rgb, depth = np.asarray(rgb, np.float64), np.asarray(depth, np.float64)
    t_rgb, t_depth = np.asarray(t_rgb, np.float64), np.asarray(t_depth, np.float64)
    S = ssim(rgb, t_rgb)
    L = w[0] * np.abs(rgb - t_rgb).mean() + w[1] * (1.0 - S) + w[2] * np.abs(depth - t_depth).mean()
    g_rgb = w[0] * np.sign(rgb - t_rgb) / rgb.size - w[1] * ssim_grad(rgb, t_rgb)
    g_depth = w[2] * np.sign(depth - t_depth) / depth.size
    return float(L), S, g_rgb, g_depth


# ---------------------------------------------------------------------------
# Mahalanobis alignment
# ---------------------------------------------------------------------------
def quat_rotation(q):
    """Rotation matrices [N, 3, 3] of (w, x, y, z) quaternions (normalised
    here; zero norm -> identity)."""
    q = np.asarray(q, np.float64)
    n = np.linalg.norm(q, axis=1, keepdims=True)
    q = np.where(n > 0, q / np.where(n > 0, n, 1.0), np.array([1.0, 0, 0, 0]))
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def covariances(log_scale, quat):
    """Sigma = R diag(s^2) R^T with s = exp(log_scale) ([N, 3, 3], float64)."""
    R = quat_rotation(quat)
    s2 = np.exp(2.0 * np.asarray(log_scale, np.float64))
    return np.einsum("nij,nj,nkj->nik", R, s2, R)


def skew(v):
    v = np.asarray(v, np.float64)
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def se3_exp(d):
    """4 x 4 exp of a 6-vector (rho, phi)."""
    rho, phi = np.asarray(d[:3], np.float64), np.asarray(d[3:], np.float64)
    th = float(np.linalg.norm(phi))
    K = skew(phi)
    if th < 1e-12:
        R, V = np.eye(3) + K, np.eye(3) + 0.5 * K
    else:
        R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, V @ rho
    return T


def mahalanobis_system(T, x_k, cov_k, x_l, cov_l, weights=None, max_dist=None):
    """Cost, gradient g (6) and Gauss-Newton matrix H (6 x 6) of
    sum_(k,l) w r^T M r at T (left perturbation delta = (rho, phi)).  With
    max_dist, pairs whose Euclidean residual |r| at T exceeds it are left out
    (the correspondence distance threshold of the G-ICP point selection,
    0.02 in Sec. 4.1)."""
    T = np.asarray(T, np.float64)
    R, t = T[:3, :3], T[:3, 3]
    cost, g, H = 0.0, np.zeros(6), np.zeros((6, 6))
    for i in range(len(x_k)):
        wi = 1.0 if weights is None else float(weights[i])
        p = R @ x_k[i] + t
        r = p - x_l[i]
        if max_dist is not None and float(r @ r) > max_dist * max_dist:
            continue
        M = np.linalg.inv(R @ cov_k[i] @ R.T + cov_l[i])
        J = np.hstack([np.eye(3), -skew(p)])  # d(exp(delta^) p)/d delta at 0
        cost += wi * float(r @ M @ r)
        g += wi * 2.0 * J.T @ M @ r
        H += wi * 2.0 * J.T @ M @ J
    return cost, g, H


def mahalanobis_step(T, x_k, cov_k, x_l, cov_l, weights=None, max_dist=None):
    """One Gauss-Newton step: delta = -H^-1 g, T <- exp(delta^) T."""
    cost, g, H = mahalanobis_system(T, x_k, cov_k, x_l, cov_l, weights, max_dist)
    delta = -np.linalg.solve(H, g)
    return se3_exp(delta) @ np.asarray(T, np.float64), delta, cost


# ---------------------------------------------------------------------------
# Pruning (Algorithm 1)
# ---------------------------------------------------------------------------
TAU_O, TAU_S, TAU_E = 0.005, 0.25, 10.0


def prune_mask(opacity_logit, log_scale, exp_f32, tau_o=TAU_O, tau_s=TAU_S, tau_e=TAU_E):
    """Boolean mask of the Gaussians Algorithm 1 removes.  Every decision is
    taken in float32: opacity = 1 / (1 + exp(-logit)), s = exp(log_scale)
    (exp_f32 is the project exponential), largest = max(s), sum = (s0 + s1) +
    s2, elongated if largest > tau_e * (sum - largest).  tau_s = None skips the
    scale and elongation criteria, as the algorithm does."""
    f = np.float32
    logit = np.asarray(opacity_logit, f)
    lam = f(1.0) / (f(1.0) + exp_f32(-logit))
    prune = lam < f(tau_o)
    if tau_s is not None:
        s = exp_f32(np.asarray(log_scale, f).reshape(-1)).reshape(-1, 3)
        largest = np.maximum(np.maximum(s[:, 0], s[:, 1]), s[:, 2])
        total = (s[:, 0] + s[:, 1]) + s[:, 2]
        prune |= largest > f(tau_s)
        prune |= largest > f(tau_e) * (total - largest)
    return prune


def prune(arrays, mask):
    """The kept rows of every array, in their original order."""
    keep = ~np.asarray(mask, bool)
    return [np.ascontiguousarray(np.asarray(a)[keep]) for a in arrays]
