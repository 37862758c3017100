"""CUDA path vs the oracle for the consensus terms and pruning, through the C
ABI: the inter-agent loss of Eq. (optim) with its SSIM term and gradients,
the Mahalanobis Gauss-Newton system and step, and Algorithm 1 pruning
(mask and compaction bit-exact)."""
import numpy as np
import pytest

import oracle
from oracle import consensus as C
from paper_2412_09723_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_GRAD = 1e-3


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_09723_gb300 import binding

    binding.load()
    return torch.device("cuda:0")


def _t(a, dev, dtype=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype), device=dev)


def _assert_grad_close(got, ref, name):
    got, ref = np.asarray(got, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    rms = float(np.sqrt(np.mean(ref ** 2)))
    err = np.abs(got - ref)
    bound = RTOL_GRAD * np.abs(ref) + RTOL_GRAD * rms
    bad = err > bound
    assert not bad.any(), f"{name}: {bad.sum()} of {bad.size}; worst {np.max(err / (bound + 1e-30))}"


def _image_pair(seed, H, W):
    """Rendered-like images: a smooth field plus texture, and a shifted,
    noisy copy; depth in [1, 3] m."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W] / max(H, W)
    base = np.stack([0.5 + 0.4 * np.sin(6 * xx + c) * np.cos(5 * yy - c) for c in range(3)], -1)
    rgb = np.clip(base + rng.normal(0, 0.05, base.shape), 0, 1).astype(np.float32)
    t_rgb = np.clip(np.roll(base, 2, axis=1) + rng.normal(0, 0.05, base.shape), 0, 1).astype(np.float32)
    depth = (2 + 0.8 * np.sin(4 * xx) * np.cos(3 * yy)).astype(np.float32)
    t_depth = (depth + rng.normal(0, 0.02, depth.shape)).astype(np.float32)
    t_depth[::7, ::5] = depth[::7, ::5]  # exact ties: zero subgradient
    return rgb, depth, t_rgb, t_depth


@pytest.mark.parametrize("H,W", [(37, 53), (150, 200), (680, 1200)])
def test_consensus_loss_matches_oracle(dev, H, W):
    from paper_2412_09723_gb300 import binding as B

    rgb, depth, t_rgb, t_depth = _image_pair(H * 7 + W, H, W)
    L, S, g_rgb, g_depth = C.paper_loss(rgb, depth, t_rgb, t_depth)
    d_rgb = torch.zeros(H, W, 3, device=dev)
    d_depth = torch.zeros(H, W, device=dev)
    loss = torch.zeros(2, device=dev)
    ws = torch.empty(B.splat_loss_consensus_workspace_size(H, W), dtype=torch.uint8, device=dev)
    B.splat_loss_consensus(_t(rgb, dev), _t(depth, dev), _t(t_rgb, dev), _t(t_depth, dev), 0.8, 0.2, 0.1, d_rgb,
                           d_depth, loss, ws)
    torch.cuda.synchronize()
    got = loss.cpu().numpy().astype(np.float64)
    assert abs(got[0] - L) <= 2e-6 * max(1.0, abs(L)), (got[0], L)
    assert abs(got[1] - S) <= 2e-6, (got[1], S)
    _assert_grad_close(d_rgb.cpu().numpy(), g_rgb, "d_rgb")
    _assert_grad_close(d_depth.cpu().numpy(), g_depth, "d_depth")
    assert np.array_equal(d_depth.cpu().numpy() == 0, g_depth == 0)  # ties give exactly zero


def test_consensus_loss_identical_images(dev):
    """SSIM(C, C) = 1: the loss is the two L1 terms (zero here) and the SSIM
    gradient vanishes."""
    from paper_2412_09723_gb300 import binding as B

    rgb, depth, _, _ = _image_pair(3, 64, 80)
    d_rgb = torch.zeros(64, 80, 3, device=dev)
    d_depth = torch.zeros(64, 80, device=dev)
    loss = torch.zeros(2, device=dev)
    ws = torch.empty(B.splat_loss_consensus_workspace_size(64, 80), dtype=torch.uint8, device=dev)
    x, d = _t(rgb, dev), _t(depth, dev)
    B.splat_loss_consensus(x, d, x, d, 0.8, 0.2, 0.1, d_rgb, d_depth, loss, ws)
    torch.cuda.synchronize()
    assert abs(float(loss[1]) - 1.0) < 1e-5 and abs(float(loss[0])) < 1e-6
    assert float(d_rgb.abs().max()) < 1e-6


# ---------------------------------------------------------------------------
def _maha_case(seed, n=20000, m=6000):
    a, b, perm, T_true, _, T0, _ = scenes.workload_alignment(seed=seed, n=n, n_views=2)
    rng = np.random.default_rng(seed)
    lb = rng.choice(n, m, replace=False).astype(np.int32)
    pairs = np.stack([perm[lb].astype(np.int32), lb], 1)  # (A id, B id) of the same surface element
    weights = rng.integers(1, 40, m).astype(np.int32)
    return a, b, pairs, weights, T_true, T0


def _maha_ref(a, b, pairs, weights, T):
    x_k = a.mean[pairs[:, 0]].astype(np.float64)
    x_l = b.mean[pairs[:, 1]].astype(np.float64)
    cov_k = C.covariances(a.log_scale[pairs[:, 0]], a.quat[pairs[:, 0]])
    cov_l = C.covariances(b.log_scale[pairs[:, 1]], b.quat[pairs[:, 1]])
    return x_l, cov_l, x_k, cov_k


def test_mahalanobis_system_and_step_match_oracle(dev):
    from paper_2412_09723_gb300 import binding as B

    a, b, pairs, weights, T_true, T0 = _maha_case(5)
    pa = [_t(x, dev) for x in a.arrays()]
    pb = [_t(x, dev) for x in b.arrays()]
    ga, gb = B.gaussians_struct(*pa), B.gaussians_struct(*pb)
    pairs_t, w_t = _t(pairs, dev, np.int32), _t(weights, dev, np.int32)
    m_dev = torch.tensor([len(pairs)], dtype=torch.int64, device=dev)
    T = _t(T0, dev)
    sys = torch.zeros(28, dtype=torch.float64, device=dev)
    B.splat_mahalanobis_system(ga, gb, pairs_t, w_t, m_dev, T, sys)
    torch.cuda.synchronize()
    x_l, cov_l, x_k, cov_k = _maha_ref(a, b, pairs, weights, T0)
    # the oracle's residual is T x_k - x_l with k the transformed map: here B (l) is transformed onto A
    cost, g, H = C.mahalanobis_system(T0.astype(np.float64), x_l, cov_l, x_k, cov_k, weights)
    s = sys.cpu().numpy()
    iu = np.triu_indices(6)
    Hg = np.zeros((6, 6))
    Hg[iu] = s[:21]
    Hg = Hg + np.triu(Hg, 1).T
    np.testing.assert_allclose(Hg, H, rtol=2e-4, atol=2e-4 * np.abs(H).max())
    np.testing.assert_allclose(s[21:27], g, rtol=2e-4, atol=2e-4 * np.abs(g).max())
    assert abs(s[27] - cost) <= 2e-4 * cost
    delta = torch.zeros(6, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    B.splat_mahalanobis_step(sys, T, delta, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    d_ref = -np.linalg.solve(H, g)
    np.testing.assert_allclose(delta.cpu().numpy(), d_ref, rtol=1e-3, atol=1e-3 * np.abs(d_ref).max())
    np.testing.assert_allclose(T.cpu().numpy(), C.se3_exp(d_ref) @ T0.astype(np.float64), atol=2e-6)


def test_mahalanobis_distance_threshold_matches_oracle(dev):
    """A fifth of the pairs get wrong partners; with a correspondence
    distance the far ones are left out on both sides (the threshold is put in
    the widest gap between residuals, so float32 and float64 agree on it)."""
    from paper_2412_09723_gb300 import binding as B

    a, b, pairs, weights, T_true, T0 = _maha_case(8)
    rng = np.random.default_rng(8)
    bad = rng.choice(len(pairs), len(pairs) // 5, replace=False)
    pairs[bad, 0] = rng.integers(0, a.n, len(bad)).astype(np.int32)
    x_l, cov_l, x_k, cov_k = _maha_ref(a, b, pairs, weights, T0)
    T64 = T0.astype(np.float64)
    r = np.sort(np.linalg.norm(x_l @ T64[:3, :3].T + T64[:3, 3] - x_k, axis=1))
    lo, hi = np.searchsorted(r, 0.015), np.searchsorted(r, 0.05)
    j = lo + int(np.argmax(np.diff(r[lo:hi])))
    d = 0.5 * (r[j] + r[j + 1])
    assert r[j + 1] - r[j] > 1e-6
    cost, g, H = C.mahalanobis_system(T64, x_l, cov_l, x_k, cov_k, weights, max_dist=d)
    pa = [_t(x, dev) for x in a.arrays()]
    pb = [_t(x, dev) for x in b.arrays()]
    sys = torch.zeros(28, dtype=torch.float64, device=dev)
    m_dev = torch.tensor([len(pairs)], dtype=torch.int64, device=dev)
    B.splat_mahalanobis_system(B.gaussians_struct(*pa), B.gaussians_struct(*pb), _t(pairs, dev, np.int32),
                               _t(weights, dev, np.int32), m_dev, _t(T0, dev), sys, max_dist=float(d))
    torch.cuda.synchronize()
    s = sys.cpu().numpy()
    np.testing.assert_allclose(s[21:27], g, rtol=2e-4, atol=2e-4 * np.abs(g).max())
    assert abs(s[27] - cost) <= 2e-4 * cost


def test_mahalanobis_iterations_reduce_error(dev):
    """Gauss-Newton iterations from 1 cm / 0.5 degrees off: the transform
    moves to within the 2 mm jitter of B's means of T_true."""
    from paper_2412_09723_gb300 import align
    from paper_2412_09723_gb300 import binding as B

    a, b, pairs, weights, T_true, T0 = _maha_case(6)
    pa = [_t(x, dev) for x in a.arrays()]
    pb = [_t(x, dev) for x in b.arrays()]
    ga, gb = B.gaussians_struct(*pa), B.gaussians_struct(*pb)
    pairs_t, w_t = _t(pairs, dev, np.int32), _t(weights, dev, np.int32)
    m_dev = torch.tensor([len(pairs)], dtype=torch.int64, device=dev)
    T = _t(T0, dev)
    sys = torch.zeros(28, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    e0 = align.pose_error(T0, T_true)
    for _ in range(4):
        sys.zero_()
        B.splat_mahalanobis_system(ga, gb, pairs_t, w_t, m_dev, T, sys)
        B.splat_mahalanobis_step(sys, T, None, status)
    torch.cuda.synchronize()
    e1 = align.pose_error(T.cpu().numpy(), T_true)
    assert int(status.item()) == 0
    assert e1[0] < 0.1 * e0[0] and e1[1] < 0.1 * e0[1], (e0, e1)


def test_mahalanobis_system_step_matches_oracle_and_clears(dev):
    """The one-launch form: the pairs split over two calls (the first only
    accumulating, the second solving in its last CTA) give the oracle's step
    of the whole set; sys is left zero, and the next call solves afresh."""
    from paper_2412_09723_gb300 import binding as B

    a, b, pairs, weights, T_true, T0 = _maha_case(11)
    pa = [_t(x, dev) for x in a.arrays()]
    pb = [_t(x, dev) for x in b.arrays()]
    ga, gb = B.gaussians_struct(*pa), B.gaussians_struct(*pb)
    half = len(pairs) // 2
    parts = [(pairs[:half], weights[:half]), (pairs[half:], weights[half:])]
    T = _t(T0, dev)
    sys = torch.zeros(32, dtype=torch.float64, device=dev)
    delta = torch.zeros(6, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    x_l, cov_l, x_k, cov_k = _maha_ref(a, b, pairs, weights, T0)
    cost, g, H = C.mahalanobis_system(T0.astype(np.float64), x_l, cov_l, x_k, cov_k, weights)
    d_ref = -np.linalg.solve(H, g)
    for it in range(2):
        T.copy_(_t(T0, dev))
        (p0, w0), (p1, w1) = parts
        B.splat_mahalanobis_system(ga, gb, _t(p0, dev, np.int32), _t(w0, dev, np.int32),
                                   torch.tensor([len(p0)], dtype=torch.int64, device=dev), T, sys)
        B.splat_mahalanobis_system_step(ga, gb, _t(p1, dev, np.int32), _t(w1, dev, np.int32),
                                        torch.tensor([len(p1)], dtype=torch.int64, device=dev), T, sys, delta, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert not sys.any()  # left zero, counter included
        np.testing.assert_allclose(delta.cpu().numpy(), d_ref, rtol=1e-3, atol=1e-3 * np.abs(d_ref).max())
        np.testing.assert_allclose(T.cpu().numpy(), C.se3_exp(d_ref) @ T0.astype(np.float64), atol=2e-6)
    # no pairs at all: the solve reports the singular system, T unchanged
    T.copy_(_t(T0, dev))
    B.splat_mahalanobis_system_step(ga, gb, _t(pairs, dev, np.int32), None, torch.zeros(1, dtype=torch.int64, device=dev),
                                    T, sys, None, status)
    torch.cuda.synchronize()
    assert int(status.item()) == B.SPLAT_ENUMERIC and not sys.any()
    assert np.array_equal(T.cpu().numpy(), T0.astype(np.float32))


def test_mahalanobis_without_pairs_reports_numeric_status(dev):
    from paper_2412_09723_gb300 import binding as B

    a, b, pairs, weights, T_true, T0 = _maha_case(7, n=1000, m=100)
    pa = [_t(x, dev) for x in a.arrays()]
    pb = [_t(x, dev) for x in b.arrays()]
    m_dev = torch.zeros(1, dtype=torch.int64, device=dev)  # no valid pairs
    T = _t(T0, dev)
    sys = torch.zeros(28, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    B.splat_mahalanobis_system(B.gaussians_struct(*pa), B.gaussians_struct(*pb), _t(pairs, dev, np.int32), None,
                               m_dev, T, sys)
    B.splat_mahalanobis_step(sys, T, None, status)
    torch.cuda.synchronize()
    assert int(status.item()) == B.SPLAT_ENUMERIC
    assert np.array_equal(T.cpu().numpy(), T0.astype(np.float32))


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 777, 200000])
def test_prune_matches_oracle(dev, n):
    from paper_2412_09723_gb300 import binding as B

    rng = np.random.default_rng(n)
    sc = scenes.scene_room(max(n, 1), 9).subset(slice(0, n))
    sc.opacity_logit = rng.normal(-3.0, 2.5, n).astype(np.float32)
    sc.log_scale = rng.normal(-3.0, 1.2, (n, 3)).astype(np.float32)
    arrays = list(sc.arrays())
    moments = [rng.normal(size=a.shape).astype(np.float32) for a in arrays]
    mask_ref = C.prune_mask(sc.opacity_logit, sc.log_scale, oracle.exp_f32)
    kept_ref = C.prune(arrays + moments, mask_ref)
    src = [_t(a, dev) for a in arrays + moments]
    dst = [torch.full_like(t, float("nan")) for t in src]
    g = B.gaussians_struct(*src[:5])
    mask = torch.zeros(n, dtype=torch.uint8, device=dev)
    n_keep = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(B.splat_prune_workspace_size(n), dtype=torch.uint8, device=dev)
    B.splat_prune(g, C.TAU_O, C.TAU_S, C.TAU_E, list(zip(src, dst)), mask, n_keep, ws)
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy().astype(bool), mask_ref)
    k = int(n_keep.item())
    assert k == int((~mask_ref).sum())
    for got, ref in zip(dst, kept_ref):
        assert np.array_equal(got[:k].cpu().numpy(), ref)


def test_prune_opacity_only(dev):
    from paper_2412_09723_gb300 import binding as B

    rng = np.random.default_rng(3)
    n = 5000
    logit = rng.normal(-4.0, 2.0, n).astype(np.float32)
    ls = rng.normal(-1.0, 1.5, (n, 3)).astype(np.float32)
    mask_ref = C.prune_mask(logit, ls, oracle.exp_f32, tau_s=None)
    z3 = np.zeros((n, 3), np.float32)
    g = B.gaussians_struct(_t(z3, dev), _t(ls, dev), _t(np.tile([1, 0, 0, 0], (n, 1)), dev), _t(logit, dev),
                           _t(z3, dev))
    mask = torch.zeros(n, dtype=torch.uint8, device=dev)
    n_keep = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(B.splat_prune_workspace_size(n), dtype=torch.uint8, device=dev)
    B.splat_prune(g, C.TAU_O, 0.0, C.TAU_E, [], mask, n_keep, ws)
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy().astype(bool), mask_ref)
    assert int(n_keep.item()) == int((~mask_ref).sum())
