"""Host arithmetic of bench.py's whole-step roofline (no GPU): the counts it
combines and which bound it picks."""
import pytest


def test_step_roofline_counts_and_bound():
    import bench

    r = bench.step_roofline(walked=1000, contributing=400, n_gaussians=10, duplicates=50, n_tiles=4, n_pix=100,
                            alu_peak_tops=1e-6, hbm_gbs=1.0)
    assert r["ops_alg"] == 2 * 9 * 1000 + (25 + 63) * 400
    assert r["bytes_alg"] == 2 * 56 * 10 + 24 * 50 + 8 * 4 + 72 * 100
    assert r["t_alu_ms"] == pytest.approx(1e3 * r["ops_alg"] / 1e6)
    assert r["t_hbm_ms"] == pytest.approx(1e3 * r["bytes_alg"] / 1e9)
    assert r["bound"] == "alu" and r["t_bound_ms"] == r["t_alu_ms"] and r["frac"] is None


def test_step_roofline_memory_bound_case():
    import bench

    r = bench.step_roofline(walked=1, contributing=1, n_gaussians=10**6, duplicates=10**6, n_tiles=1, n_pix=1,
                            alu_peak_tops=40.0, hbm_gbs=1.0)
    assert r["bound"] == "hbm" and r["t_bound_ms"] == r["t_hbm_ms"]
