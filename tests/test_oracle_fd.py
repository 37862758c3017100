"""The oracle's adjoint against central finite differences of its own forward
render in float64 (a 64-Gaussian 32x24 sub-scene of the room workload), and
the float32 adjoint against the float64 one.

The forward is piecewise smooth: a finite difference is only meaningful when
no discrete decision (tile rectangle, radius, alpha floor, stop rule) changes
between theta - h and theta + h.  The oracle hashes every such decision; a
parameter whose perturbation changes the hash is retried with a smaller step
and otherwise skipped (and counted)."""
import math

import numpy as np
import pytest

from paper_2412_09723_gb300 import scenes

CAM = scenes.Camera(32, 24, 525.0, 525.0, 16.0, 12.0)  # centre window of the 640x480 camera
BG = np.array([0.1, 0.2, 0.3])


def se3_exp(d):
    """exp of a 6-vector (rho, phi) as a 4x4 matrix (Rodrigues + left Jacobian)."""
    rho, phi = np.asarray(d[:3], float), np.asarray(d[3:], float)
    th = float(np.linalg.norm(phi))
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        R, V = np.eye(3) + K, np.eye(3) + 0.5 * K
    else:
        R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, V @ rho
    return T


def _setup(seed):
    sc = scenes.scene_wall_patch(64, seed, extent=(0.08, 0.06)).astype(np.float64)
    rng = np.random.default_rng(seed + 7)
    g = (rng.normal(size=(24, 32, 3)), rng.normal(size=(24, 32)), rng.normal(size=(24, 32)))
    w2c = scenes.perturbed_w2c(seed, 0.01, 0.5).astype(np.float64)
    return sc, w2c, g


def _loss(orc, sc, w2c, g):
    o = orc.render_fwd(sc, w2c, CAM, BG, dtype=np.float64)
    return float((g[0] * o["rgb"]).sum() + (g[1] * o["depth"]).sum() + (g[2] * o["sil"]).sum()), o["signature"]


def _fd(orc, f, sig0, h0=1e-6):
    h = h0
    for _ in range(3):
        lp, sp = f(h)
        lm, sm = f(-h)
        if sp == sig0 and sm == sig0:
            return (lp - lm) / (2 * h)
        h *= 0.1
    return None


def _check(an, fd, tol):
    an, fd = np.asarray(an), np.asarray(fd)
    rms = math.sqrt(float(np.mean(fd ** 2))) + 1e-300
    err = np.abs(an - fd)
    bound = tol * np.abs(fd) + tol * rms
    assert np.all(err <= bound), (np.max(err / (np.abs(fd) + rms)), an[np.argmax(err - bound)], fd[np.argmax(err - bound)])


@pytest.mark.parametrize("seed", [100, 101])
def test_adjoint_matches_finite_differences(orc, seed):
    sc, w2c, g = _setup(seed)
    L0, sig0 = _loss(orc, sc, w2c, g)
    grads = orc.render_bwd(sc, w2c, CAM, BG, *g, dtype=np.float64)
    o0 = orc.render_fwd(sc, w2c, CAM, BG, dtype=np.float64)
    assert o0["n_contrib"].mean() > 5  # the Gaussians overlap: compositing is exercised
    skipped = 0
    for name in ("mean", "log_scale", "quat", "opacity_logit", "rgb"):
        arr = getattr(sc, name)
        an, fd = [], []
        for idx in np.ndindex(arr.shape):
            orig = arr[idx]

            def f(h):
                arr[idx] = orig + h
                r = _loss(orc, sc, w2c, g)
                arr[idx] = orig
                return r

            v = _fd(orc, f, sig0)
            if v is None:
                skipped += 1
                continue
            an.append(grads[name][idx])
            fd.append(v)
        _check(an, fd, 1e-5)
    fd_pose = []
    for k in range(6):
        e = np.zeros(6)
        e[k] = 1.0
        v = _fd(orc, lambda h: _loss(orc, sc, se3_exp(h * e) @ w2c, g), sig0)
        assert v is not None
        fd_pose.append(v)
    _check(grads["pose"], fd_pose, 1e-5)
    assert skipped <= 10


def test_float32_adjoint_close_to_float64(orc):
    sc, w2c, g = _setup(102)
    g64 = orc.render_bwd(sc, w2c, CAM, BG, *g, dtype=np.float64)
    o32 = orc.render_fwd(sc.astype(np.float32), w2c, CAM, BG, dtype=np.float32)
    o64 = orc.render_fwd(sc, w2c, CAM, BG, dtype=np.float64)
    # same discrete decisions in both precisions on this scene
    assert np.array_equal(o32["n_contrib"], o64["n_contrib"])
    g32 = orc.render_bwd(sc.astype(np.float32), w2c, CAM, BG, *(a.astype(np.float32) for a in g), dtype=np.float32)
    for name in ("mean", "log_scale", "quat", "opacity_logit", "rgb", "pose"):
        ref = g64[name].ravel()
        rms = math.sqrt(float(np.mean(ref ** 2)))
        err = np.abs(g32[name].ravel() - ref)
        assert np.all(err <= 1e-4 * np.abs(ref) + 1e-4 * rms), name


def test_planted_mistake_is_caught_by_fd(orc):
    """A dropped term in the adjoint (here: the background term of dL/dalpha,
    emulated by differentiating with the wrong background) fails the check."""
    sc, w2c, g = _setup(103)
    L0, sig0 = _loss(orc, sc, w2c, g)
    wrong = orc.render_bwd(sc, w2c, CAM, np.zeros(3), *g, dtype=np.float64)
    arr = sc.opacity_logit
    an, fd = [], []
    for i in range(sc.n):
        orig = arr[i]

        def f(h):
            arr[i] = orig + h
            r = _loss(orc, sc, w2c, g)
            arr[i] = orig
            return r

        v = _fd(orc, f, sig0)
        if v is not None:
            an.append(wrong["opacity_logit"][i])
            fd.append(v)
    with pytest.raises(AssertionError):
        _check(an, fd, 1e-5)


def ad_transpose_apply(w2c, g):
    """Ad(w2c)^T g for a 6-vector g = (rho, phi): (R^T g_rho, R^T (g_phi - t x g_rho))."""
    R, t = np.asarray(w2c)[:3, :3], np.asarray(w2c)[:3, 3]
    g = np.asarray(g, float)
    return np.concatenate([R.T @ g[:3], R.T @ (g[3:] - np.cross(t, g[:3]))])


def test_relative_transform_gradient_is_adjoint_transpose(orc):
    """A map aligned by T_rel and seen through w2c_A is rendered with
    w2c_A exp(delta^) T_rel; its gradient w.r.t. delta equals
    Ad(w2c_A)^T applied to the camera-pose gradient at w2c_A T_rel."""
    sc, _, g = _setup(104)
    w2c_a = scenes.perturbed_w2c(20, 0.05, 4.0).astype(np.float64)
    T_rel = scenes.perturbed_w2c(21, 0.03, 2.0).astype(np.float64)
    w_eff = w2c_a @ T_rel
    L0, sig0 = _loss(orc, sc, w_eff, g)
    d_cam = orc.render_bwd(sc, w_eff, CAM, BG, *g, dtype=np.float64)["pose"]
    want = ad_transpose_apply(w2c_a, d_cam)
    fd = []
    for k in range(6):
        e = np.zeros(6)
        e[k] = 1.0
        v = _fd(orc, lambda h: _loss(orc, sc, w2c_a @ se3_exp(h * e) @ T_rel, g), sig0)
        assert v is not None
        fd.append(v)
    _check(want, fd, 1e-5)
