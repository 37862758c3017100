"""The agent step (render, loss, backward, Adam, pose step, association) as
eager launches and as a captured CUDA graph."""
import numpy as np
import pytest

from paper_2412_09723_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _agent(dev, **cfg):
    from paper_2412_09723_gb300.agent import Agent, StepConfig

    sc, w2c, w2c_t, cam, bg = scenes.workload_track_map(n=60000)
    a = Agent(sc, w2c, cam, dev, cfg=StepConfig(**cfg))
    a.render_observation_from(w2c_t)
    a.size_capacity(1.5)
    return a


def test_graph_replay_equals_eager_step(dev):
    a = _agent(dev, map=False, track=False)
    b = _agent(dev, map=False, track=False)
    a.step()
    torch.cuda.synchronize()
    b.capture()  # runs one eager warm-up step, then captures
    b.replay()
    torch.cuda.synchronize()
    for k in ("rgb", "depth", "sil", "t_final", "n_contrib", "max_id"):
        assert torch.equal(a.fb.image[k], b.fb.image[k]), k
    assert float(a.loss.item()) == pytest.approx(float(b.loss.item()), rel=1e-5)
    for ga, gb in zip(a.grads, b.grads):
        ref = ga.double()
        rms = float(ref.pow(2).mean().sqrt())
        assert float((ga.double() - gb.double()).abs().max()) <= 1e-3 * rms + 1e-3 * float(ref.abs().max())
    assert int(a.m_dev.item()) == int(b.m_dev.item())
    assert torch.equal(a.pairs[: int(a.m_dev.item())], b.pairs[: int(b.m_dev.item())])


def test_tracking_reduces_pose_error(dev):
    """40 tracking + mapping steps from a pose 1 cm / 0.5 degree off the pose
    that rendered the target: the loss falls and the pose moves toward it."""
    from paper_2412_09723_gb300 import scenes as S

    sc, w2c, w2c_t, cam, bg = S.workload_track_map(n=60000)
    a = _agent(dev)
    target = torch.as_tensor(w2c_t, device=dev)
    e0 = float((a.w2c - target).abs().max())
    a.step()
    torch.cuda.synchronize()
    l0 = float(a.loss.item())
    for _ in range(39):
        a.step()
    torch.cuda.synchronize()
    l1 = float(a.loss.item())
    e1 = float((a.w2c - target).abs().max())
    assert a.status() == 0
    assert l1 < 0.7 * l0
    assert e1 < e0
