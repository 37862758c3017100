"""The multi-threaded build of the oracle (the timed CPU baseline) against the
single-threaded parity build: the same forward results bit for bit, and the
same adjoint up to the grouping of its sums (per-thread buffers, filled in a
dynamic tile order, so the last bits vary from run to run): within the
gradient rule |g - g_ref| <= 1e-3 |g_ref| + 1e-3 rms(g_ref) per tensor."""
import numpy as np
import pytest

import oracle
from paper_2412_09723_gb300 import scenes


@pytest.fixture(scope="module")
def case():
    sc = scenes.scene_room(20000, 5)
    w2c = scenes.perturbed_w2c(6, 0.1, 10.0)
    cam = scenes.Camera(200, 150, 120.0, 120.0, 100.0, 75.0)
    bg = np.float32([0.2, 0.3, 0.4])
    g = np.random.default_rng(11)
    up = (g.normal(size=(150, 200, 3)).astype(np.float32), g.normal(size=(150, 200)).astype(np.float32),
          g.normal(size=(150, 200)).astype(np.float32))
    return sc, w2c, cam, bg, up


def test_parity_build_is_single_threaded():
    assert oracle.threads() == 1


def test_threaded_forward_equals_parity_build(case):
    sc, w2c, cam, bg, _ = case
    ref = oracle.render_fwd(sc, w2c, cam, bg)
    with oracle.parallel(4) as nth:
        assert nth == 4 and oracle.threads() == 4
        got = oracle.render_fwd(sc, w2c, cam, bg)
        band = oracle.render_fwd(sc, w2c, cam, bg, rows=(37, 101))
    assert oracle.threads() == 1
    for k in ("rgb", "depth", "sil", "t_final", "n_contrib", "max_id"):
        assert np.array_equal(got[k], ref[k]), k
        assert np.array_equal(band[k][37:101], ref[k][37:101]), k
    assert got["n_pairs"] == ref["n_pairs"]


def test_threaded_adjoint_matches_parity_build(case):
    sc, w2c, cam, bg, up = case
    ref = oracle.render_bwd(sc, w2c, cam, bg, *up)
    with oracle.parallel(4):
        got = oracle.render_bwd(sc, w2c, cam, bg, *up)
        band = oracle.render_bwd(sc, w2c, cam, bg, *up, rows=(37, 101))
    refb = oracle.render_bwd(sc, w2c, cam, bg, *up, rows=(37, 101))
    for r, x in ((ref, got), (refb, band)):
        for k in ("mean", "log_scale", "quat", "opacity_logit", "rgb", "pose", "d2d"):
            a, b = np.asarray(x[k], np.float64), np.asarray(r[k], np.float64)
            rms = float(np.sqrt(np.mean(b ** 2)))
            assert np.all(np.abs(a - b) <= 1e-3 * np.abs(b) + 1e-3 * rms), k
