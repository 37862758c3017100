"""Serving loop: continuous batching gives every request the same result it
gets alone (within the gradient tolerance), also when the HBM budget forces
agents to give up their per-step buffers or to be swapped out and back in."""
import numpy as np
import pytest

from paper_2412_09723_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC = [dict(n=20000, seed=11, cam=scenes.Camera(320, 240, 262.5, 262.5, 160.0, 120.0)),
        dict(n=40000, seed=12, cam=scenes.Camera(400, 300, 300.0, 300.0, 200.0, 150.0)),
        dict(n=60000, seed=13, cam=scenes.Camera(320, 240, 262.5, 262.5, 160.0, 120.0))]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _server(dev, spec, budget=150 << 30, **kw):
    from paper_2412_09723_gb300.serve import Server, make_agents_workload

    srv = Server(dev, budget, **kw)
    make_agents_workload(srv, spec, frames_per_agent=3)
    srv.prepare()
    return srv


def _reqs(pattern):
    from paper_2412_09723_gb300.serve import Request

    return [Request(a, k, f, 0.0, rid=i) for i, (a, k, f) in enumerate(pattern)]


def _close(r1, r2):
    assert r1.loss == pytest.approx(r2.loss, rel=1e-5, abs=1e-7)
    np.testing.assert_allclose(r1.w2c, r2.w2c, atol=2e-6)


PATTERN = [(0, "track", 0), (1, "track", 0), (2, "map", 0), (0, "map", 1), (1, "track", 1), (2, "track", 1),
           (0, "track", 2), (2, "map", 2)]


def test_alone_equals_mix(dev):
    # agent 0's requests alone
    alone = _server(dev, SPEC[:1])
    ra = _reqs([p for p in PATTERN if p[0] == 0])
    alone.serve(ra, realtime=False)
    # the same requests in a mix with two other agents, batched
    mix = _server(dev, SPEC, max_batch=3, n_streams=2)
    rm = _reqs(PATTERN)
    mix.serve(rm, realtime=False)
    for a, b in zip(ra, [r for r in rm if r.agent == 0]):
        _close(a, b)
    # and the plain per-request path agrees with both
    plain = _server(dev, SPEC)
    rp = _reqs(PATTERN)
    plain.serve_plain(rp, realtime=False)
    for a, b in zip(rm, rp):
        _close(a, b)


@pytest.mark.parametrize("tier", ["releases", "swaps"])
def test_budget_forces_swaps_without_changing_results(dev, tier):
    """A budget of 1.2 footprints of the largest agent keeps every state
    resident but makes idle agents give up their per-step buffers; a budget
    below the largest footprint plus the other agents' states makes its
    admission swap states out to host memory.  Either way every request's
    result is the unbounded one."""
    from paper_2412_09723_gb300.serve import _agent_bytes

    big = _server(dev, SPEC)
    ref = _reqs(PATTERN)
    big.serve(ref, realtime=False)
    tiers = [_agent_bytes(s.agent) for s in big.slots]
    k = max(range(len(tiers)), key=lambda i: sum(tiers[i]))
    one = sum(tiers[k])
    others = sum(st for i, (st, _) in enumerate(tiers) if i != k)
    budget = int(one * 1.2) if tier == "releases" else int(one + 0.5 * others)
    small = _server(dev, SPEC, budget=budget, max_batch=3)
    got = _reqs(PATTERN)
    small.serve(got, realtime=False)
    assert getattr(small, tier) > 0
    for a, b in zip(ref, got):
        _close(a, b)
