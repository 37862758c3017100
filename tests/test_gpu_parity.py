"""CUDA path vs the CPU oracle, through the C ABI, on the same seeded inputs.

Integer and bit-level outputs (projection, tile rects, sort keys, Gaussian
ids, tile ranges, contributor counts, maximum-weight ids, association pairs)
must match exactly; rendered colour / depth / silhouette / transmittance too
(both sides take the same IEEE operations in the same order; the stated
tolerance is 1e-4 absolute, and the check is bit for bit so that a change of
operation order cannot hide under it); gradients to
|g - g_ref| <= 1e-3 |g_ref| + 1e-3 rms(g_ref)."""
import numpy as np
import pytest

import oracle
from paper_2412_09723_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_GRAD = 1e-3
ATOL_IMG = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_09723_gb300 import binding

    binding.load()
    return torch.device("cuda:0")


def _params(sc, dev):
    return tuple(torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev) for a in sc.arrays())


def _w(w2c, dev):
    return torch.as_tensor(np.ascontiguousarray(w2c, np.float32), device=dev)


def _cases():
    small = scenes.workload_small_forward()
    ragged_cam = scenes.Camera(200, 150, 120.0, 120.0, 100.0, 75.0)
    ragged = (scenes.scene_room(20000, 5), scenes.perturbed_w2c(6, 0.1, 10.0), ragged_cam, np.float32([0.2, 0.3, 0.4]))
    return {"small_2k_128x96": small, "room_20k_200x150_ragged": ragged}


CASES = _cases()


def _full_vga():
    sc, w2c, _, cam, bg = scenes.workload_track_map()
    return sc, w2c, cam, bg


def _render_gpu(sc, w2c, cam, bg, dev, want_keys=True):
    from paper_2412_09723_gb300 import rasterizer as R

    p = _params(sc, dev)
    fb = R.FrameBuffers(sc.n, cam, dev, want_keys=want_keys)
    R.render_forward(p, _w(w2c, dev), cam, tuple(float(x) for x in bg), fb)
    torch.cuda.synchronize()
    return p, fb


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a


def _assert_grad_close(got, ref, name):
    got, ref = np.asarray(got, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    rms = float(np.sqrt(np.mean(ref ** 2))) if ref.size else 0.0
    err = np.abs(got - ref)
    bound = RTOL_GRAD * np.abs(ref) + RTOL_GRAD * rms
    bad = err > bound
    assert not bad.any(), f"{name}: {bad.sum()} of {bad.size} out of tolerance; worst {np.max(err / (bound + 1e-30))}"


# ---------------------------------------------------------------------------
def test_exp_bit_exact(dev):
    from paper_2412_09723_gb300 import binding as B

    bits = np.arange(0, 2 ** 32, 1031, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x)]
    x = np.concatenate([x, np.float32([0.0, -0.0, 88.0, 88.00001, -87.0, -87.00001, np.inf, -np.inf])])
    xt = torch.as_tensor(x, device=dev)
    yt = torch.empty_like(xt)
    B.splat_exp_f32(xt, yt)
    y = yt.cpu().numpy()
    ref = oracle.exp_f32(x)
    assert np.array_equal(_bits(y), _bits(ref))


@pytest.mark.parametrize("case", list(CASES))
def test_project_bit_exact(dev, case):
    sc, w2c, cam, bg = CASES[case]
    p, fb = _render_gpu(sc, w2c, cam, bg, dev)
    ref = oracle.project(sc, w2c, cam)
    got = {k: v.cpu().numpy() for k, v in fb.proj.items()}
    assert np.array_equal(_bits(got["xyzo"]), _bits(ref["xyzo"]))
    assert np.array_equal(_bits(got["conic"][:, :3]), _bits(ref["conic"][:, :3]))
    for k in ("radius", "rect", "tiles_touched"):
        assert np.array_equal(got[k], ref[k]), k


def test_project_off_screen_centres_bit_exact(dev):
    """Centres in a band around the image border, large anisotropic splats:
    many Gaussians reach into the image from outside (and many do not), so the
    projection's conservative centre cull is exercised on both sides of its
    bound; every field must equal the oracle's."""
    rng = np.random.default_rng(17)
    n = 20000
    cam = scenes.Camera(200, 150, 120.0, 120.0, 100.0, 75.0)
    z = rng.uniform(0.5, 4.0, n)
    u = rng.uniform(-150.0, 350.0, n)
    v = rng.uniform(-150.0, 300.0, n)
    mean = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], 1)
    ls = rng.normal(-2.3, 0.8, (n, 3))
    q = rng.normal(size=(n, 4))
    sc = scenes.Scene(mean.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                      rng.normal(0, 1, n).astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32))
    w2c = np.eye(4, dtype=np.float32)
    p, fb = _render_gpu(sc, w2c, cam, np.zeros(3, np.float32), dev)
    ref = oracle.project(sc, w2c, cam)
    got = {k: v.cpu().numpy() for k, v in fb.proj.items()}
    outside = (u < 0) | (u >= 200) | (v < 0) | (v >= 150)
    reaching = outside & (ref["radius"] > 0)
    assert reaching.sum() > 1000 and (outside & (ref["radius"] == 0)).sum() > 1000
    assert np.array_equal(_bits(got["xyzo"]), _bits(ref["xyzo"]))
    assert np.array_equal(_bits(got["conic"][:, :3]), _bits(ref["conic"][:, :3]))
    for k in ("radius", "rect", "tiles_touched"):
        assert np.array_equal(got[k], ref[k]), k


def _check_bins(fb, sc, w2c, cam):
    keys, vals, ranges = oracle.bin_sort(sc, w2c, cam)
    k = int(fb.k_dev.item())
    assert k == len(vals)
    assert int(fb.status.item()) == 0
    assert np.array_equal(fb.vals[:k].cpu().numpy().view(np.uint32), vals)
    assert np.array_equal(fb.keys[:k].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(fb.ranges.cpu().numpy().view(np.uint32), ranges)


def _cost_bucket(S):
    """1 + the exponent and three mantissa bits of S as a float32 (eighths of
    an octave), 0 for S = 0, at most 127."""
    S = np.asarray(S, np.float32)
    b = np.where(S > 0, ((S.view(np.uint32) >> 20).astype(np.int64) - (127 << 3)) + 1, 0)
    return np.minimum(b, 127)


def _check_schedule(sched, n_contrib, cam, ordered_by_cost=False):
    """The tile schedule after a forward render: the per-tile costs are the
    summed contributor counts of the tile's pixels (from the oracle's image),
    and the order written by the binning is a permutation of the tiles; with
    `ordered_by_cost` (the binning ran after the forward) the order takes the
    cost buckets heaviest first."""
    sched = sched.view(np.uint32)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    n_t = tx * ty
    assert sched.size == 1 + 2 * n_t
    pad = np.zeros((ty * 16, tx * 16), np.int64)
    pad[:cam.height, :cam.width] = n_contrib
    S = pad.reshape(ty, 16, tx, 16).sum(axis=(1, 3)).ravel()
    assert np.array_equal(sched[1 + n_t:].astype(np.int64), S)
    assert sched[0] == n_t
    order = sched[1:1 + n_t]
    assert np.array_equal(np.sort(order), np.arange(n_t, dtype=np.uint32))
    if ordered_by_cost:
        assert (np.diff(_cost_bucket(S[order])) <= 0).all()


def _check_image(fb, ref):
    if hasattr(fb, "schedule"):
        _check_schedule(fb.schedule.cpu().numpy(), ref["n_contrib"], fb.cam)
    got = {k: v.cpu().numpy() for k, v in fb.image.items()}
    for k in ("rgb", "depth", "sil", "t_final"):
        d = np.abs(got[k].astype(np.float64) - ref[k])
        assert d.max() <= ATOL_IMG, (k, d.max())
        assert np.array_equal(_bits(got[k]), _bits(ref[k])), (k, "not bit-exact", d.max())
    assert np.array_equal(got["n_contrib"], ref["n_contrib"])
    assert np.array_equal(got["max_id"], ref["max_id"])


@pytest.mark.parametrize("case", list(CASES))
def test_bin_sort_and_render_fwd(dev, case):
    from paper_2412_09723_gb300 import rasterizer as R

    sc, w2c, cam, bg = CASES[case]
    p, fb = _render_gpu(sc, w2c, cam, bg, dev)
    _check_bins(fb, sc, w2c, cam)
    ref = oracle.render_fwd(sc, w2c, cam, bg)
    _check_image(fb, ref)
    R.bin_sort(fb)  # the next binning orders the tiles by the costs this forward wrote
    torch.cuda.synchronize()
    _check_schedule(fb.schedule.cpu().numpy(), ref["n_contrib"], cam, ordered_by_cost=True)


def test_full_size_vga_forward(dev):
    sc, w2c, cam, bg = _full_vga()
    p, fb = _render_gpu(sc, w2c, cam, bg, dev)
    _check_bins(fb, sc, w2c, cam)
    _check_image(fb, oracle.render_fwd(sc, w2c, cam, bg))


def _bwd_gpu(p, fb, w2c, cam, bg, g, dev):
    from paper_2412_09723_gb300 import binding as B

    grads = [torch.zeros_like(t) for t in p]
    d_pose = torch.zeros(6, dtype=torch.float32, device=dev)
    d2d = torch.zeros(sc_n(p), 10, dtype=torch.float32, device=dev)
    gr, gd, gs = (torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev) for a in g)
    B.splat_render_bwd(B.gaussians_struct(*p), fb.cproj, fb.ccam, _w(w2c, dev), fb.vals, fb.ranges, fb.cimg, bg,
                       gr, gd, gs, B.CGaussiansGrad(*(B._p(t) for t in grads)), d_pose, d2d, fb.bwd_ws,
                       schedule=fb.schedule)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in grads], d_pose.cpu().numpy(), d2d.cpu().numpy()


def sc_n(p):
    return p[0].shape[0]


def _upstream(cam, seed):
    rng = np.random.default_rng(seed)
    H, W = cam.height, cam.width
    return (rng.normal(size=(H, W, 3)).astype(np.float32), rng.normal(size=(H, W)).astype(np.float32),
            rng.normal(size=(H, W)).astype(np.float32))


@pytest.mark.parametrize("case", list(CASES))
def test_render_bwd(dev, case):
    sc, w2c, cam, bg = CASES[case]
    p, fb = _render_gpu(sc, w2c, cam, bg, dev)
    g = _upstream(cam, 11)
    grads, d_pose, d2d = _bwd_gpu(p, fb, w2c, cam, bg, g, dev)
    ref = oracle.render_bwd(sc, w2c, cam, bg, *g)
    _assert_grad_close(d2d, ref["d2d"], "d2d")
    for name, got in zip(("mean", "log_scale", "quat", "opacity_logit", "rgb"), grads):
        _assert_grad_close(got, ref[name], name)
    _assert_grad_close(d_pose, ref["pose"], "pose")


def test_full_size_vga_backward(dev):
    sc, w2c, cam, bg = _full_vga()
    p, fb = _render_gpu(sc, w2c, cam, bg, dev, want_keys=False)
    g = _upstream(cam, 12)
    grads, d_pose, d2d = _bwd_gpu(p, fb, w2c, cam, bg, g, dev)
    ref = oracle.render_bwd(sc, w2c, cam, bg, *g)
    for name, got in zip(("mean", "log_scale", "quat", "opacity_logit", "rgb"), grads):
        _assert_grad_close(got, ref[name], name)
    _assert_grad_close(d_pose, ref["pose"], "pose")


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_empty_map(dev):
    sc = scenes.scene_uniform(0, 0)
    cam = scenes.Camera(40, 24, 50.0, 50.0, 20.0, 12.0)
    p, fb = _render_gpu(sc, np.eye(4, dtype=np.float32), cam, (0.1, 0.2, 0.3), dev)
    assert int(fb.k_dev.item()) == 0
    assert not fb.ranges.any()
    rgb = fb.image["rgb"].cpu().numpy()
    assert np.allclose(rgb, np.float32([0.1, 0.2, 0.3]))
    assert (fb.image["max_id"].cpu().numpy() == -1).all()


def test_all_behind_camera(dev):
    sc = scenes.scene_uniform(500, 1)
    sc.mean[:, 2] = -sc.mean[:, 2]
    cam = scenes.CAM_SMALL
    p, fb = _render_gpu(sc, np.eye(4, dtype=np.float32), cam, (0, 0, 0), dev)
    assert int(fb.k_dev.item()) == 0
    assert (fb.proj["radius"].cpu().numpy() == 0).all()
    assert (fb.image["t_final"].cpu().numpy() == 1).all()


def test_zero_opacity_background(dev):
    sc, w2c, cam, _ = scenes.workload_small_forward(seed=9)
    sc.opacity_logit[:] = -np.inf
    p, fb = _render_gpu(sc, w2c, cam, (0.25, 0.5, 0.75), dev)
    assert np.array_equal(fb.image["rgb"].cpu().numpy(), np.broadcast_to(np.float32([0.25, 0.5, 0.75]), (96, 128, 3)))
    assert (fb.image["t_final"].cpu().numpy() == 1).all() and (fb.image["max_id"].cpu().numpy() == -1).all()
    assert (fb.image["n_contrib"].cpu().numpy() == 0).all()


def test_capacity_overflow_is_reported(dev):
    from paper_2412_09723_gb300 import binding as B
    from paper_2412_09723_gb300 import rasterizer as R

    sc, w2c, cam, bg = scenes.workload_small_forward()
    p = _params(sc, dev)
    fb = R.FrameBuffers(sc.n, cam, dev, capacity=1000)
    R.project(B.gaussians_struct(*p), _w(w2c, dev), fb)
    fb.status.zero_()
    B.splat_bin_sort(fb.cproj, fb.n, fb.ccam, None, fb.vals, fb.capacity, fb.k_dev, fb.ranges, fb.status, fb.bin_ws)
    torch.cuda.synchronize()
    k_true = len(oracle.bin_sort(sc, w2c, cam)[1])
    assert int(fb.k_dev.item()) == k_true > 1000
    assert int(fb.status.item()) == B.SPLAT_ECAPACITY
    r = fb.ranges.cpu().numpy().view(np.uint32)
    assert r.max() <= 1000


def test_single_tile_image(dev):
    sc = scenes.scene_uniform(300, 4)
    cam = scenes.Camera(13, 9, 12.0, 12.0, 6.5, 4.5)
    p, fb = _render_gpu(sc, np.eye(4, dtype=np.float32), cam, (0, 0, 0), dev)
    _check_bins(fb, sc, np.eye(4, dtype=np.float32), cam)
    _check_image(fb, oracle.render_fwd(sc, np.eye(4, dtype=np.float32), cam, np.zeros(3, np.float32)))


# ---------------------------------------------------------------------------
# loss, Adam, pose step, association
# ---------------------------------------------------------------------------
def test_loss_l1(dev):
    from paper_2412_09723_gb300 import binding as B

    rng = np.random.default_rng(0)
    H, W = 37, 53
    a = [rng.uniform(size=s).astype(np.float32) for s in ((H, W, 3), (H, W), (H, W, 3), (H, W))]
    a[2][:3] = a[0][:3]  # exact ties -> zero subgradient
    t = [torch.as_tensor(x, device=dev) for x in a]
    gr, gd = torch.empty_like(t[0]), torch.empty_like(t[1])
    loss = torch.zeros(1, device=dev)
    B.splat_loss_l1(t[0], t[1], t[2], t[3], 1.0, 0.5, gr, gd, loss)
    L, rgr, rgd = oracle.loss_l1(a[0], a[1], a[2], a[3], 1.0, 0.5)
    assert np.array_equal(gr.cpu().numpy(), rgr) and np.array_equal(gd.cpu().numpy(), rgd)
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)


def test_adam(dev):
    from paper_2412_09723_gb300 import binding as B

    rng = np.random.default_rng(1)
    n = 10007
    p, g, m, v = (rng.normal(size=n).astype(np.float32) for _ in range(4))
    v = np.abs(v)
    tp, tg, tm, tv = (torch.as_tensor(x.copy(), device=dev) for x in (p, g, m, v))
    B.splat_adam(tp, tg, tm, tv, torch.tensor([3], dtype=torch.int32, device=dev), 1e-3)
    rp, rm, rv = oracle.adam(p, g, m, v, 3, 1e-3)
    np.testing.assert_allclose(tp.cpu().numpy(), rp, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(tm.cpu().numpy(), rm, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(tv.cpu().numpy(), rv, rtol=1e-6, atol=1e-7)


def test_pose_step_matches_oracle_adam_and_retraction(dev):
    """Five pose steps with gradients that change size and sign from step to
    step, so that the moments and bias corrections of steps t > 1 matter: the
    device moments equal the oracle's Adam (run on the 6-vector, the update of
    a zero parameter being the step delta itself), and the device pose the
    oracle's chain w2c_t = exp(delta_t^) w2c_(t-1) in float64 from the same
    start, within float32 rounding."""
    from oracle import consensus as C
    from paper_2412_09723_gb300 import binding as B

    w0 = scenes.perturbed_w2c(3, 0.2, 15.0)
    w = _w(w0, dev)
    m, v = torch.zeros(6, device=dev), torch.zeros(6, device=dev)
    lr_t, lr_r = 0.01, 0.002
    rng = np.random.default_rng(21)
    ref_w = w0.astype(np.float64)
    rm, rv = np.zeros(6, np.float32), np.zeros(6, np.float32)
    for t in range(1, 6):
        g = (rng.normal(size=6) * 10.0 ** rng.uniform(-2, 1, 6)).astype(np.float32)
        B.splat_pose_step(w, torch.as_tensor(g, device=dev), m, v, torch.tensor([t], dtype=torch.int32, device=dev),
                          lr_t, lr_r)
        d_t, rm[:3], rv[:3] = oracle.adam(np.zeros(3, np.float32), g[:3], rm[:3], rv[:3], t, lr_t)
        d_r, rm[3:], rv[3:] = oracle.adam(np.zeros(3, np.float32), g[3:], rm[3:], rv[3:], t, lr_r)
        ref_w = C.se3_exp(np.concatenate([d_t, d_r]).astype(np.float64)) @ ref_w
        torch.cuda.synchronize()
        np.testing.assert_allclose(m.cpu().numpy(), rm, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(v.cpu().numpy(), rv, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(w.cpu().numpy(), ref_w, atol=2e-6 * t)
    assert np.abs(ref_w - w0).max() > 1e-3  # the steps did move the pose


def test_assoc_two_maps(dev):
    from paper_2412_09723_gb300 import binding as B

    cam = scenes.Camera(160, 120, 130.0, 130.0, 80.0, 60.0)
    a = scenes.scene_room(30000, 7)
    b = scenes.scene_room(25000, 8)
    w2c = scenes.perturbed_w2c(9, 0.05, 3.0)
    ra = oracle.render_fwd(a, w2c, cam, np.zeros(3))
    rb = oracle.render_fwd(b, w2c, cam, np.zeros(3))
    ref_pairs, ref_counts = oracle.assoc(ra["max_id"], ra["t_final"], rb["max_id"], rb["t_final"], 0.5)
    t = [torch.as_tensor(x, device=dev) for x in (ra["max_id"], ra["t_final"], rb["max_id"], rb["t_final"])]
    npix = cam.npix
    cap = npix
    pairs = torch.zeros(cap, 2, dtype=torch.int32, device=dev)
    counts = torch.zeros(cap, dtype=torch.int32, device=dev)
    m_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(B.splat_assoc_workspace_size(npix), dtype=torch.uint8, device=dev)
    B.splat_assoc(t[0], t[1], t[2], t[3], a.n, b.n, 0.5, pairs, counts, cap, m_dev, status, ws)
    m = int(m_dev.item())
    assert m == len(ref_pairs) > 100
    assert np.array_equal(pairs[:m].cpu().numpy(), ref_pairs)
    assert np.array_equal(counts[:m].cpu().numpy(), ref_counts)
    assert int(status.item()) == 0
    # too small a capacity: status raised, the first pairs kept
    status.zero_()
    B.splat_assoc(t[0], t[1], t[2], t[3], a.n, b.n, 0.5, pairs, counts, 10, m_dev, status, ws)
    assert int(status.item()) == B.SPLAT_ECAPACITY and int(m_dev.item()) == m
    assert np.array_equal(pairs[:10].cpu().numpy(), ref_pairs[:10])


# ---------------------------------------------------------------------------
# autograd wrapper
# ---------------------------------------------------------------------------
def test_autograd_matches_oracle(dev):
    from paper_2412_09723_gb300 import rasterizer as R

    sc, w2c, cam, bg = CASES["room_20k_200x150_ragged"]
    p = [t.clone().requires_grad_(True) for t in _params(sc, dev)]
    delta = torch.zeros(6, device=dev, requires_grad=True)
    rgb, depth, sil, tfin, mid = R.render(*p, _w(w2c, dev), cam, tuple(float(x) for x in bg), delta)
    g = _upstream(cam, 13)
    gt = [torch.as_tensor(x, device=dev) for x in g]
    L = (rgb * gt[0]).sum() + (depth * gt[1]).sum() + (sil * gt[2]).sum()
    L.backward()
    ref = oracle.render_bwd(sc, w2c, cam, bg, *g)
    for name, t in zip(("mean", "log_scale", "quat", "opacity_logit", "rgb"), p):
        _assert_grad_close(t.grad.cpu().numpy(), ref[name], name)
    _assert_grad_close(delta.grad.cpu().numpy(), ref["pose"], "pose")


def test_deep_tiles_use_the_merge_path(dev):
    """More than 8192 duplicates in one tile: the per-tile sort falls back to
    chunked shared-memory sorts plus global merges; the order must not change."""
    rng = np.random.default_rng(3)
    n = 30000
    sc = scenes.Scene(
        mean=np.stack([rng.uniform(-0.05, 0.05, n), rng.uniform(-0.05, 0.05, n), rng.uniform(1.0, 3.0, n)],
                      axis=1).astype(np.float32),
        log_scale=np.full((n, 3), -4.0, np.float32), quat=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
        opacity_logit=rng.normal(-3.0, 0.5, n).astype(np.float32), rgb=rng.uniform(0, 1, (n, 3)).astype(np.float32))
    cam = scenes.Camera(40, 40, 60.0, 60.0, 20.0, 20.0)
    p, fb = _render_gpu(sc, np.eye(4, dtype=np.float32), cam, (0, 0, 0), dev)
    ranges = fb.ranges.cpu().numpy().view(np.uint32)
    assert (ranges[:, 1] - ranges[:, 0]).max() > 8192 * 2
    _check_bins(fb, sc, np.eye(4, dtype=np.float32), cam)
    _check_image(fb, oracle.render_fwd(sc, np.eye(4, dtype=np.float32), cam, np.zeros(3, np.float32)))


def test_many_tiles_take_the_scan_launch(dev):
    """More tiles than the scatter keeps in shared memory (8192): the tile
    prefix runs as its own launch and the scatter takes one global atomic per
    duplicate; bins and image must not change."""
    sc = scenes.scene_room(6000, 21)
    cam = scenes.Camera(2064, 1024, 900.0, 900.0, 1032.0, 512.0)
    w2c = scenes.perturbed_w2c(22, 0.05, 2.0)
    assert ((cam.width + 15) // 16) * ((cam.height + 15) // 16) > 8192
    p, fb = _render_gpu(sc, w2c, cam, (0, 0, 0), dev)
    assert int(fb.k_dev.item()) > 10000
    _check_bins(fb, sc, w2c, cam)
    _check_image(fb, oracle.render_fwd(sc, w2c, cam, np.zeros(3, np.float32)))


def _render_gpu_cap(sc, w2c, cam, bg, dev, capacity):
    from paper_2412_09723_gb300 import rasterizer as R

    p = _params(sc, dev)
    fb = R.FrameBuffers(sc.n, cam, dev, capacity=capacity, want_keys=True)
    R.render_forward(p, _w(w2c, dev), cam, tuple(float(x) for x in bg), fb)
    torch.cuda.synchronize()
    return p, fb


def test_bins_at_tight_capacity_and_one_deep_tile(dev):
    """The full 300k / 640x480 workload with a duplicate capacity close to K
    (as the agent sizes it), and a 640x480 frame whose centre tile holds about
    20000 keys (chunked shared-memory sorts and global merges): bins equal the
    oracle's."""
    sc, w2c, cam, bg = _full_vga()
    K = int(oracle.project(sc, w2c, cam)["tiles_touched"].sum())  # whole-rect count: an upper bound of K
    p, fb = _render_gpu_cap(sc, w2c, cam, bg, dev, int(K * 1.1))
    _check_bins(fb, sc, w2c, cam)
    rng = np.random.default_rng(8)
    n = 20000
    c = np.array([(16 * 20 + 8 - 320) / 525.0, (16 * 15 + 8 - 240) / 525.0])  # a tile centre at depth 1
    z = rng.uniform(1.0, 3.0, n)
    deep = scenes.Scene(
        mean=np.stack([c[0] * z + rng.normal(0, 1e-3, n), c[1] * z + rng.normal(0, 1e-3, n), z], 1).astype(np.float32),
        log_scale=np.full((n, 3), -6.0, np.float32), quat=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
        opacity_logit=rng.normal(0.0, 0.5, n).astype(np.float32), rgb=rng.uniform(0, 1, (n, 3)).astype(np.float32))
    eye = np.eye(4, dtype=np.float32)
    p, fb = _render_gpu_cap(deep, eye, cam, bg, dev, 4 * n)
    ranges = fb.ranges.cpu().numpy().view(np.uint32)
    assert (ranges[:, 1] - ranges[:, 0]).max() > 4 * 2048
    _check_bins(fb, deep, eye, cam)


@pytest.mark.parametrize("levels", [1, 40, 1500])
def test_depth_ties_break_by_id(dev, levels):
    """Depths drawn from `levels` exact values (1: one fronto-parallel plane,
    every tile one long run of equal depths; 40: runs of tens; 1500: short
    runs): equal depths must come in ascending id order in every tile."""
    rng = np.random.default_rng(levels)
    n = 6000
    z = (2.0 + 1e-3 * rng.integers(0, levels, n)).astype(np.float32)
    sc = scenes.Scene(
        mean=np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.2, 0.2, n), z], axis=1).astype(np.float32),
        log_scale=np.full((n, 3), -3.5, np.float32), quat=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
        opacity_logit=rng.normal(-2.0, 0.5, n).astype(np.float32), rgb=rng.uniform(0, 1, (n, 3)).astype(np.float32))
    cam = scenes.Camera(160, 112, 200.0, 200.0, 80.0, 56.0)
    w2c = np.eye(4, dtype=np.float32)
    p, fb = _render_gpu(sc, w2c, cam, (0, 0, 0), dev)
    ranges = fb.ranges.cpu().numpy().view(np.uint32)
    assert (ranges[:, 1] - ranges[:, 0]).max() > 256  # the radix path, not only the small bitonic one
    _check_bins(fb, sc, w2c, cam)
    _check_image(fb, oracle.render_fwd(sc, w2c, cam, np.zeros(3, np.float32)))


def test_adam_groups_matches_per_group_adam(dev):
    from paper_2412_09723_gb300 import binding as B

    rng = np.random.default_rng(2)
    sizes = [3001, 17, 4096, 1, 999]
    lrs = [1e-3, 5e-2, 1e-4, 2e-3, 7e-3]
    host = [[rng.normal(size=n).astype(np.float32) for _ in range(4)] for n in sizes]
    for h in host:
        h[3] = np.abs(h[3])
    dev_t = [[torch.as_tensor(a.copy(), device=dev) for a in h] for h in host]
    groups = B.AdamGroups([d[0] for d in dev_t], [d[1] for d in dev_t], [d[2] for d in dev_t], [d[3] for d in dev_t],
                          lrs)
    step = torch.tensor([4], dtype=torch.int32, device=dev)
    B.splat_adam_groups(groups, step, zero_grad=True)
    torch.cuda.synchronize()
    for h, d, lr in zip(host, dev_t, lrs):
        rp, rm, rv = oracle.adam(h[0], h[1], h[2], h[3], 4, lr)
        np.testing.assert_allclose(d[0].cpu().numpy(), rp, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(d[2].cpu().numpy(), rm, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(d[3].cpu().numpy(), rv, rtol=1e-6, atol=1e-7)
        assert not d[1].any()  # gradients cleared


def test_adam_groups_sparse_state(dev):
    """Most aligned runs of 4 elements have gradient and moments +0 (Gaussians
    never seen): their parameters stay bit for bit unchanged; runs with a -0,
    with only moments, or with only a gradient get the full update."""
    from paper_2412_09723_gb300 import binding as B

    rng = np.random.default_rng(9)
    n = 4096 + 3
    h = [rng.normal(size=n).astype(np.float32) for _ in range(4)]
    h[3] = np.abs(h[3])
    quiet = rng.random((n + 3) // 4) < 0.7
    mask = np.repeat(quiet, 4)[:n]
    for a in (h[1], h[2], h[3]):
        a[mask] = 0.0
    live = np.nonzero(~mask)[0]
    h[1][live[:40]] = 0.0  # moments only
    h[2][live[40:80]] = 0.0
    h[3][live[40:80]] = 0.0  # gradient only
    q = np.nonzero(quiet)[0][:5] * 4  # a -0 gradient in five otherwise quiet runs
    h[1][q] = np.float32(-0.0)
    d = [torch.as_tensor(a.copy(), device=dev) for a in h]
    groups = B.AdamGroups([d[0]], [d[1]], [d[2]], [d[3]], [3e-3])
    step = torch.tensor([7], dtype=torch.int32, device=dev)
    B.splat_adam_groups(groups, step, zero_grad=True)
    torch.cuda.synchronize()
    rp, rm, rv = oracle.adam(h[0], h[1], h[2], h[3], 7, 3e-3)
    got = [x.cpu().numpy() for x in d]
    np.testing.assert_allclose(got[0], rp, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(got[2], rm, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(got[3], rv, rtol=1e-6, atol=1e-7)
    skipped = mask.copy()
    skipped[q] = False
    assert np.array_equal(got[0][skipped].view(np.uint32), h[0][skipped].view(np.uint32))
    assert not got[1].any()
    assert not np.signbit(got[1]).any()  # the -0 gradients were consumed and cleared to +0


def test_assoc_deep_buckets_and_duplicates(dev):
    """Few distinct ids over many pixels (deep buckets -> merge path) and many
    repeated pairs; pairs and counts must equal the oracle's."""
    from paper_2412_09723_gb300 import binding as B

    rng = np.random.default_rng(5)
    H, W = 300, 400
    ia = rng.integers(0, 40, size=(H, W)).astype(np.int32)
    ib = rng.integers(0, 7, size=(H, W)).astype(np.int32)
    ia[:5] = -1
    ta = rng.uniform(0, 1, (H, W)).astype(np.float32)
    tb = rng.uniform(0, 1, (H, W)).astype(np.float32)
    ref_pairs, ref_counts = oracle.assoc(ia, ta, ib, tb, 0.7)
    t = [torch.as_tensor(x, device=dev) for x in (ia, ta, ib, tb)]
    npix = H * W
    pairs = torch.zeros(npix, 2, dtype=torch.int32, device=dev)
    counts = torch.zeros(npix, dtype=torch.int32, device=dev)
    m_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(B.splat_assoc_workspace_size(npix), dtype=torch.uint8, device=dev)
    B.splat_assoc(t[0], t[1], t[2], t[3], 40, 7, 0.7, pairs, counts, npix, m_dev, status, ws)
    m = int(m_dev.item())
    assert m == len(ref_pairs)
    assert np.array_equal(pairs[:m].cpu().numpy(), ref_pairs)
    assert np.array_equal(counts[:m].cpu().numpy(), ref_counts)


def test_distance_selection_parity(dev):
    """Candidate selection by distance (Sec. 3.4 step 1) inside the projection:
    projection, bins and image bit-exact, gradients within tolerance."""
    import dataclasses

    sc = scenes.scene_room(20000, 23)
    w2c = scenes.perturbed_w2c(24, 0.2, 15.0)
    W = w2c.astype(np.float64)
    r = np.sort(np.linalg.norm(sc.mean.astype(np.float64) @ W[:3, :3].T + W[:3, 3], axis=1))
    lo, hi = int(0.3 * len(r)), int(0.7 * len(r))
    j = lo + int(np.argmax(np.diff(r[lo:hi])))
    cam = dataclasses.replace(scenes.Camera(200, 150, 120.0, 120.0, 100.0, 75.0), max_dist=float(0.5 * (r[j] + r[j + 1])))
    bg = np.float32([0.1, 0.2, 0.3])
    p, fb = _render_gpu(sc, w2c, cam, bg, dev)
    ref = oracle.project(sc, w2c, cam)
    got = {k: v.cpu().numpy() for k, v in fb.proj.items()}
    for k in ("radius", "rect", "tiles_touched"):
        assert np.array_equal(got[k], ref[k]), k
    assert 0 < (ref["radius"] == 0).mean() < 1
    _check_bins(fb, sc, w2c, cam)
    _check_image(fb, oracle.render_fwd(sc, w2c, cam, bg))
    g = _upstream(cam, 12)
    grads, d_pose, d2d = _bwd_gpu(p, fb, w2c, cam, bg, g, dev)
    refg = oracle.render_bwd(sc, w2c, cam, bg, *g)
    for name, gg in zip(("mean", "log_scale", "quat", "opacity_logit", "rgb"), grads):
        _assert_grad_close(gg, refg[name], name)
    _assert_grad_close(d_pose, refg["pose"], "pose")


def _assoc_gpu(dev, ia, ta, ib, tb, n_a, n_b, t_max):
    from paper_2412_09723_gb300 import binding as B

    t = [torch.as_tensor(np.ascontiguousarray(x), device=dev) for x in (ia, ta, ib, tb)]
    npix = ia.size
    pairs = torch.zeros(npix, 2, dtype=torch.int32, device=dev)
    counts = torch.zeros(npix, dtype=torch.int32, device=dev)
    m_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(B.splat_assoc_workspace_size(npix), dtype=torch.uint8, device=dev)
    B.splat_assoc(t[0], t[1], t[2], t[3], n_a, n_b, t_max, pairs, counts, npix, m_dev, status, ws)
    torch.cuda.synchronize()
    m = int(m_dev.item())
    assert int(status.item()) == 0
    return pairs[:m].cpu().numpy(), counts[:m].cpu().numpy()


def test_assoc_runs_and_global_table(dev):
    """Long horizontal runs of one pair (merged per thread, split at chunk and
    CTA boundaries), and buckets with tens of thousands of distinct pairs (the
    global-memory hash table): pairs and pixel counts equal the oracle's."""
    rng = np.random.default_rng(9)
    H, W = 333, 517
    yy, xx = np.mgrid[0:H, 0:W]
    ia = ((yy // 3) * 1000 + xx // 13).astype(np.int32)   # runs of 13 along rows
    ib = ((yy // 5) * 700 + xx // 11).astype(np.int32)
    ia[rng.uniform(size=ia.shape) < 0.02] = -1
    ta = rng.uniform(0, 1, (H, W)).astype(np.float32)
    tb = rng.uniform(0, 0.6, (H, W)).astype(np.float32)
    ref = oracle.assoc(ia, ta, ib, tb, 0.8)
    got = _assoc_gpu(dev, ia, ta, ib, tb, int(ia.max()) + 1, int(ib.max()) + 1, 0.8)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # three ids of map A, each paired with ~40k distinct ids of map B
    ia2 = rng.integers(0, 3, (H, W)).astype(np.int32)
    ib2 = rng.integers(0, 60000, (H, W)).astype(np.int32)
    ref2 = oracle.assoc(ia2, ta, ib2, tb, 0.8)
    assert len(ref2[0]) > 3 * 2000
    got2 = _assoc_gpu(dev, ia2, ta, ib2, tb, 3, 60000, 0.8)
    assert np.array_equal(got2[0], ref2[0]) and np.array_equal(got2[1], ref2[1])


# ---------------------------------------------------------------------------
# fused entry points: forward render with the L1 terms, projection adjoint
# with the map's Adam step
# ---------------------------------------------------------------------------
def test_render_fwd_l1_matches_oracle_loss(dev):
    """splat_render_fwd_l1: the image bit for bit as splat_render_fwd, the L1
    gradients bit for bit as the oracle's on that image, the loss to 1e-5."""
    from paper_2412_09723_gb300 import binding as B
    from paper_2412_09723_gb300 import rasterizer as R

    sc, w2c, cam, bg = CASES["room_20k_200x150_ragged"]
    p, fb = _render_gpu(sc, w2c, cam, bg, dev)
    ref = oracle.render_fwd(sc, w2c, cam, bg)
    tgt = oracle.render_fwd(sc, scenes.perturbed_w2c(31, 0.01, 0.5, base=w2c), cam, bg)
    t_rgb, t_depth = (torch.as_tensor(tgt[k], device=dev) for k in ("rgb", "depth"))
    t_rgb[:2] = torch.as_tensor(ref["rgb"][:2], device=dev)  # exact ties: zero subgradient
    g_rgb, g_depth = torch.full_like(t_rgb, 7.0), torch.full_like(t_depth, 7.0)
    loss = torch.full((1,), 0.25, device=dev)
    fb2 = R.FrameBuffers(sc.n, cam, dev)
    R.project(B.gaussians_struct(*p), _w(w2c, dev), fb2)
    R.bin_sort(fb2)
    l1 = B.l1_struct(t_rgb, t_depth, 1.0, 0.5, g_rgb, g_depth, loss)
    B.splat_render_fwd_l1(fb2.cproj, p[4], sc.n, fb2.vals, fb2.ranges, fb2.ccam, tuple(float(x) for x in bg), fb2.cimg,
                          l1, schedule=fb2.schedule)
    torch.cuda.synchronize()
    _check_image(fb2, ref)
    L, rg, rd = oracle.loss_l1(ref["rgb"], ref["depth"], t_rgb.cpu().numpy(), t_depth.cpu().numpy(), 1.0, 0.5)
    assert np.array_equal(_bits(g_rgb.cpu().numpy()), _bits(rg))
    assert np.array_equal(_bits(g_depth.cpu().numpy()), _bits(rd))
    assert (rg[:2] == 0).all()
    assert float(loss.item()) == pytest.approx(0.25 + L, rel=1e-5)


@pytest.mark.parametrize("case", ["room_20k_200x150_ragged", "vga_300k"])
def test_render_fwd_bwd_one_launch_matches_oracle(dev, case):
    """splat_render_fwd_bwd: images, L1 gradients and loss as
    splat_render_fwd_l1, and the screen-space gradients it leaves in the
    workspace, carried to the parameters and the pose by splat_project_bwd,
    within the gradient rule of the oracle's adjoint of the same L1 loss;
    twice (the second call takes the tiles heaviest first, in the order the
    binning built from the first call's costs)."""
    from paper_2412_09723_gb300 import binding as B
    from paper_2412_09723_gb300 import rasterizer as R

    sc, w2c, cam, bg = _full_vga() if case == "vga_300k" else CASES[case]
    p = _params(sc, dev)
    ref = oracle.render_fwd(sc, w2c, cam, bg)
    tgt = oracle.render_fwd(sc, scenes.perturbed_w2c(31, 0.01, 0.5, base=w2c), cam, bg)
    t_rgb, t_depth = (torch.as_tensor(tgt[k], device=dev) for k in ("rgb", "depth"))
    L, rg, rd = oracle.loss_l1(ref["rgb"], ref["depth"], tgt["rgb"], tgt["depth"], 1.0, 0.5)
    want = oracle.render_bwd(sc, w2c, cam, bg, rg, rd)
    fb = R.FrameBuffers(sc.n, cam, dev)
    g_rgb, g_depth = torch.zeros_like(t_rgb), torch.zeros_like(t_depth)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    gs = B.gaussians_struct(*p)
    for it in range(2):
        loss = torch.zeros(1, device=dev)
        l1 = B.l1_struct(t_rgb, t_depth, 1.0, 0.5, g_rgb, g_depth, loss)
        R.project(gs, _w(w2c, dev), fb)
        R.bin_sort(fb)
        B.splat_render_fwd_bwd(fb.cproj, p[4], sc.n, fb.vals, fb.ranges, fb.ccam, tuple(float(x) for x in bg),
                               fb.cimg, l1, status, fb.bwd_ws, schedule=fb.schedule)
        grads = [torch.zeros_like(t) for t in p]
        d_pose = torch.zeros(6, dtype=torch.float32, device=dev)
        B.splat_project_bwd(gs, fb.cproj, fb.ccam, _w(w2c, dev), fb.bwd_ws, B.CGaussiansGrad(*(B._p(t) for t in grads)),
                            d_pose)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        _check_image(fb, ref)
        if it == 1:
            _check_schedule(fb.schedule.cpu().numpy(), ref["n_contrib"], cam, ordered_by_cost=False)
            order = fb.schedule.cpu().numpy().view(np.uint32)[1:1 + cam.n_tiles]
            prev = fb.schedule.cpu().numpy().view(np.uint32)[1 + cam.n_tiles:]  # equal costs: same frame
            assert (np.diff(_cost_bucket(prev[order])) <= 0).all()
        assert np.array_equal(_bits(g_rgb.cpu().numpy()), _bits(rg))
        assert np.array_equal(_bits(g_depth.cpu().numpy()), _bits(rd))
        assert float(loss.item()) == pytest.approx(L, rel=1e-5)
        for name, got in zip(("mean", "log_scale", "quat", "opacity_logit", "rgb"), grads):
            _assert_grad_close(got.cpu().numpy(), want[name], f"{case} step {it}: {name}")
        _assert_grad_close(d_pose.cpu().numpy(), want["pose"], f"{case} step {it}: pose")


def _fused_case(dev, seed, case="room_20k_200x150_ragged"):
    from paper_2412_09723_gb300 import binding as B

    if case == "room_700k_200x150_ragged":  # more Gaussians than one scan of the fused adjoint's warps covers
        _, w2c, cam, bg = CASES["room_20k_200x150_ragged"]
        sc = scenes.scene_room(700_000, 9)
    else:
        sc, w2c, cam, bg = CASES[case]
    p, fb = _render_gpu(sc, w2c, cam, bg, dev)
    g = _upstream(cam, seed)
    gr, gd, gs = (torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev) for a in g)
    B.splat_render_bwd(B.gaussians_struct(*p), fb.cproj, fb.ccam, _w(w2c, dev), fb.vals, fb.ranges, fb.cimg, bg,
                       gr, gd, gs, None, None, None, fb.bwd_ws)  # screen-space gradients only
    torch.cuda.synchronize()
    return sc, w2c, cam, bg, g, p, fb


LRS = (1e-4, 1e-3, 1e-3, 5e-2, 2.5e-3)


@pytest.mark.parametrize("case", ["room_20k_200x150_ragged", "room_700k_200x150_ragged"])
def test_project_bwd_adam_equals_adjoint_then_adam(dev, case):
    """The fused adjoint + Adam step (kept Gaussians by the adjoint, culled ones
    with gradient 0) moves the map and both moments exactly as
    splat_project_bwd into zeroed gradients followed by splat_adam_groups, and
    gives the same pose gradient (step 3, non-zero moments on half of the
    map, the rest of the moments zero: those elements stay untouched).  The
    700k map takes several rounds of the adjoint warps' batched radius scan,
    with partial queues carried from one round to the next."""
    from paper_2412_09723_gb300 import binding as B

    sc, w2c, cam, bg, g, p, fb = _fused_case(dev, 14, case)
    rng = np.random.default_rng(15)
    n = sc.n
    keep = torch.as_tensor(rng.random(n) < 0.5, device=dev)
    ms = [torch.as_tensor(rng.normal(0, 1e-3, tuple(t.shape)).astype(np.float32), device=dev) for t in p]
    vs = [torch.as_tensor(rng.uniform(1e-7, 1e-6, tuple(t.shape)).astype(np.float32), device=dev) for t in p]
    for t in ms + vs:
        t[~keep] = 0.0
    step = torch.tensor([3], dtype=torch.int32, device=dev)
    # unfused
    pa = [t.clone() for t in p]
    ma, va = [t.clone() for t in ms], [t.clone() for t in vs]
    grads = [torch.zeros_like(t) for t in p]
    pose_a = torch.zeros(6, device=dev)
    B.splat_project_bwd(B.gaussians_struct(*pa), fb.cproj, fb.ccam, _w(w2c, dev), fb.bwd_ws,
                        B.CGaussiansGrad(*(B._p(t) for t in grads)), pose_a)
    B.splat_adam_groups(B.AdamGroups(pa, grads, ma, va, list(LRS)), step, zero_grad=True)
    # fused
    pb = [t.clone() for t in p]
    mb, vb = [t.clone() for t in ms], [t.clone() for t in vs]
    pose_b = torch.zeros(6, device=dev)
    cmb, cvb = B.CGaussiansGrad(*(B._p(t) for t in mb)), B.CGaussiansGrad(*(B._p(t) for t in vb))
    B.splat_project_bwd_adam(B.gaussians_struct(*pb), fb.cproj, fb.ccam, _w(w2c, dev), fb.bwd_ws, cmb, cvb, LRS, step,
                             pose_b)
    torch.cuda.synchronize()
    for a, b in zip(pa + ma + va, pb + mb + vb):
        assert torch.equal(a, b)
    kept = fb.proj["radius"] != 0
    assert not torch.equal(pb[0][~kept & keep], p[0][~kept & keep])  # culled with moments: moved
    culled = fb.proj["radius"] == 0
    assert bool(culled.any()) and bool((~culled).any())
    assert torch.equal(pb[0][culled & ~keep], p[0][culled & ~keep])  # zero state, zero gradient: untouched
    np.testing.assert_allclose(pose_b.cpu().numpy(), pose_a.cpu().numpy(), rtol=1e-5,
                               atol=1e-5 * float(pose_a.abs().max()))


def test_pose_step_inside_the_fused_adjoint(dev):
    """splat_project_bwd_adam with a pose step: the last CTA takes the pose's
    Adam step and retraction from the whole d_pose, bit for bit as
    splat_pose_step does with that d_pose afterwards (two steps: non-zero
    moments in the second), and leaves its counter at zero."""
    from paper_2412_09723_gb300 import binding as B

    sc, w2c, cam, bg, g, p, fb = _fused_case(dev, 16)
    ms, vs = [torch.zeros_like(t) for t in p], [torch.zeros_like(t) for t in p]
    cm, cv = B.CGaussiansGrad(*(B._p(t) for t in ms)), B.CGaussiansGrad(*(B._p(t) for t in vs))
    w_in = _w(w2c, dev)
    w_a, w_b = w_in.clone(), w_in.clone()
    pm_a, pv_a = torch.zeros(6, device=dev), torch.zeros(6, device=dev)
    pm_b, pv_b = torch.zeros(6, device=dev), torch.zeros(6, device=dev)
    counter = torch.zeros(1, dtype=torch.int32, device=dev)
    for t in range(1, 3):
        step = torch.tensor([t], dtype=torch.int32, device=dev)
        d_pose = torch.zeros(6, device=dev)
        cpose = B.CPoseAdam(B._p(w_a), B._p(pm_a), B._p(pv_a), B._p(step), 2e-3, 4e-4, 0.9, 0.999, 1e-15,
                            B._p(counter))
        pa = [x.clone() for x in p]
        B.splat_project_bwd_adam(B.gaussians_struct(*pa), fb.cproj, fb.ccam, w_in, fb.bwd_ws, cm, cv, LRS, step,
                                 d_pose, pose=cpose)
        B.splat_pose_step(w_b, d_pose, pm_b, pv_b, step, 2e-3, 4e-4)
        torch.cuda.synchronize()
        assert float(d_pose.abs().max()) > 0
        assert torch.equal(w_a, w_b) and torch.equal(pm_a, pm_b) and torch.equal(pv_a, pv_b)
        assert int(counter.item()) == 0
    assert not torch.equal(w_a, w_in)


def _bits_of(mask):
    """A boolean per Gaussian packed into int32 words, bit i of word i // 32."""
    m = np.asarray(mask, bool)
    words = (m.size + 31) // 32
    b = np.zeros(words * 32, np.uint64)
    b[:m.size] = m
    return (b.reshape(words, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32).view(np.int32)


@pytest.mark.parametrize("entry,n", [("fused", 20_000), ("separate", 20_000), ("fused", 700_000)])
def test_seen_bitmap_changes_no_update(dev, entry, n):
    """With the seen bitmap the map's Adam step skips the culled Gaussians whose
    bit is clear (zero moments) and updates those whose bit is set, so map and
    moments equal the bitmap-free update bit for bit, step after step, over
    three steps from three poses (Gaussians seen at one pose and culled at the
    next keep moving), through splat_project_bwd_adam or through it with
    culled = 0 plus splat_adam_culled; the kept Gaussians' bits are set, and a
    clear bit always has zero moments.  Both updates take the same
    screen-space gradients (the render's atomics make their last bits vary
    from one render to the next).  The 700k map takes several rounds of the
    culled part's batched bit loads."""
    from paper_2412_09723_gb300 import binding as B
    from paper_2412_09723_gb300 import rasterizer as R

    sc, w2c0, cam, bg = CASES["room_20k_200x150_ragged"]
    if n != sc.n:
        sc = scenes.scene_room(n, 9)
    p0 = _params(sc, dev)
    state = []
    for use_seen in (False, True):
        p = [t.clone() for t in p0]
        m, v = [torch.zeros_like(t) for t in p], [torch.zeros_like(t) for t in p]
        seen = torch.zeros((sc.n + 31) // 32, dtype=torch.int32, device=dev) if use_seen else None
        state.append(dict(p=p, m=m, v=v, seen=seen, gs=B.gaussians_struct(*p),
                          cm=B.CGaussiansGrad(*(B._p(t) for t in m)), cv=B.CGaussiansGrad(*(B._p(t) for t in v))))
    a, b = state
    fb = R.FrameBuffers(sc.n, cam, dev)
    kept_any = torch.zeros(sc.n, dtype=torch.bool, device=dev)
    for t in range(3):
        w2c = scenes.perturbed_w2c(40 + t, 0.3, 25.0, base=w2c0)  # visibility changes from pose to pose
        R.project(a["gs"], _w(w2c, dev), fb)
        R.bin_sort(fb)
        B.splat_render_fwd(fb.cproj, a["p"][4], sc.n, fb.vals, fb.ranges, fb.ccam, tuple(float(x) for x in bg),
                           fb.cimg)
        gr, gd, gsil = (torch.as_tensor(np.ascontiguousarray(x, np.float32), device=dev) for x in _upstream(cam, t))
        B.splat_render_bwd(a["gs"], fb.cproj, fb.ccam, _w(w2c, dev), fb.vals, fb.ranges, fb.cimg, bg, gr, gd, gsil,
                           None, None, None, fb.bwd_ws)
        step = torch.tensor([t + 1], dtype=torch.int32, device=dev)
        for st in (b, a):  # b first: a's map, which the projection above read, moves last
            pose = torch.zeros(6, device=dev)
            B.splat_project_bwd_adam(st["gs"], fb.cproj, fb.ccam, _w(w2c, dev), fb.bwd_ws, st["cm"], st["cv"], LRS,
                                     step, pose, culled=entry == "fused", seen=st["seen"])
            if entry == "separate":
                B.splat_adam_culled(st["gs"], fb.proj["radius"], st["cm"], st["cv"], LRS, step, seen=st["seen"])
        kept_any |= fb.proj["radius"] != 0
        torch.cuda.synchronize()
        for x, y in zip(a["p"] + a["m"] + a["v"], b["p"] + b["m"] + b["v"]):
            assert torch.equal(x, y), f"step {t}"
    assert bool((kept_any & (fb.proj["radius"] == 0)).any())  # seen before, culled at the last pose
    assert np.array_equal(b["seen"].cpu().numpy(), _bits_of(kept_any.cpu().numpy()))
    nz = np.zeros(sc.n, bool)
    for x in b["m"] + b["v"]:
        nz |= (x.reshape(sc.n, -1) != 0).any(dim=1).cpu().numpy()
    assert not (nz & ~kept_any.cpu().numpy()).any()


def test_project_bwd_adam_matches_oracle(dev):
    """Against the oracle: the oracle's adjoint of the same per-pixel upstream
    gradients, then the oracle's Adam (step 2) with moments large against the
    gradient tolerance: every parameter's update within 1e-3 of the oracle's
    (relative to the largest update of its tensor) and the pose gradient by
    the gradient rule."""
    from paper_2412_09723_gb300 import binding as B

    sc, w2c, cam, bg, g, p, fb = _fused_case(dev, 16)
    ref = oracle.render_bwd(sc, w2c, cam, bg, *g)
    names = ("mean", "log_scale", "quat", "opacity_logit", "rgb")
    rng = np.random.default_rng(17)
    ms, vs = [], []
    for name in names:
        gr = ref[name]
        scale = float(np.abs(gr).max()) + 1e-30
        ms.append((rng.normal(0, 1, gr.shape) * scale).astype(np.float32))
        vs.append((rng.uniform(0.5, 2.0, gr.shape) * scale * scale).astype(np.float32))
    mb = [torch.as_tensor(x, device=dev) for x in ms]
    vb = [torch.as_tensor(x, device=dev) for x in vs]
    pb = [t.clone() for t in p]
    pose = torch.zeros(6, device=dev)
    step = torch.tensor([2], dtype=torch.int32, device=dev)
    cmb, cvb = B.CGaussiansGrad(*(B._p(t) for t in mb)), B.CGaussiansGrad(*(B._p(t) for t in vb))
    B.splat_project_bwd_adam(B.gaussians_struct(*pb), fb.cproj, fb.ccam, _w(w2c, dev), fb.bwd_ws, cmb, cvb, LRS, step,
                             pose)
    torch.cuda.synchronize()
    for k, name in enumerate(names):
        p0 = getattr(sc, name).astype(np.float32)
        rp, rm, rv = oracle.adam(p0, ref[name], ms[k], vs[k], 2, LRS[k])
        du_ref = rp.astype(np.float64) - p0
        du = pb[k].cpu().numpy().astype(np.float64) - p0
        assert np.abs(du - du_ref).max() <= 1e-3 * np.abs(du_ref).max(), name
        _assert_grad_close(mb[k].cpu().numpy(), rm, name + " m")
    _assert_grad_close(pose.cpu().numpy(), ref["pose"], "pose")
