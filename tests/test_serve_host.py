"""Host logic of the serving loop (no GPU): the Poisson request trace and the
latency statistics the bench reports."""
import numpy as np
import pytest

pytest.importorskip("torch")


def test_poisson_trace_rates_order_and_mapping_requests():
    from paper_2412_09723_gb300.serve import poisson_trace

    reqs = poisson_trace(n_agents=3, rate_hz=30.0, duration_s=200.0, frames_per_agent=8, map_every=5, seed=1)
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and [r.rid for r in reqs] == list(range(len(reqs)))
    for a in range(3):
        track = [r for r in reqs if r.agent == a and r.kind == "track"]
        maps = [r for r in reqs if r.agent == a and r.kind == "map"]
        # Poisson counts: mean rate x duration, standard deviation sqrt(6000) ~ 77
        assert abs(len(track) - 30.0 * 200.0) < 5 * np.sqrt(30.0 * 200.0)
        assert len(maps) == len(track) // 5
        # every 5th tracking frame carries a mapping request at the same time and frame
        for k, m in enumerate(maps):
            t = track[5 * k + 4]
            assert (m.arrival, m.frame) == (t.arrival, t.frame)
        assert all(r.frame == k % 8 for k, r in enumerate(track))
        gaps = np.diff([r.arrival for r in track])
        assert abs(gaps.mean() - 1 / 30.0) < 0.1 / 30.0  # exponential gaps with mean 1/rate


def test_latency_stats_percentiles():
    from paper_2412_09723_gb300.serve import Request, latency_stats

    reqs = []
    for i in range(100):
        r = Request(0, "track", 0, arrival=float(i))
        r.done = r.arrival + (i + 1) * 1e-3  # latencies 1 .. 100 ms
        reqs.append(r)
    st = latency_stats(reqs, makespan=100.0)
    assert st["requests"] == 100 and st["frames_per_s"] == pytest.approx(1.0)
    assert st["p50_ms"] == pytest.approx(50.5) and st["p99_ms"] == pytest.approx(99.0)
    assert st["mean_ms"] == pytest.approx(50.5)
