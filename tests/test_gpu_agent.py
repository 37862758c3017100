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


def test_one_launch_render_step_equals_two_launch_step(dev):
    """A step whose forward and screen-space backward share one launch
    (`fused`) gives the two-launch step's images bit for bit, its loss, its
    associations, and its parameter and pose gradients within the gradient
    rule; captured and replayed as well."""
    a = _agent(dev, map=False, track=False)
    b = _agent(dev, map=False, track=False, fused=True)
    for k in range(2):
        a.step()
        if k == 0:
            b.step()
        else:  # no map or pose update: the capture's warm-up step changes nothing
            b.capture()
            b.replay()
        torch.cuda.synchronize()
        for key in ("rgb", "depth", "sil", "t_final", "n_contrib", "max_id"):
            assert torch.equal(a.fb.image[key], b.fb.image[key]), key
        assert float(a.loss.item()) == pytest.approx(float(b.loss.item()), rel=1e-5)
        assert int(b.status()) == 0
        for ga, gb in zip([*a.grads, a.d_pose], [*b.grads, b.d_pose]):
            ref = ga.double()
            rms = float(ref.pow(2).mean().sqrt())
            assert float((ga.double() - gb.double()).abs().max()) <= 1e-3 * rms + 1e-3 * float(ref.abs().max())
        assert int(a.m_dev.item()) == int(b.m_dev.item())
        assert torch.equal(a.pairs[: int(a.m_dev.item())], b.pairs[: int(b.m_dev.item())])


def test_host_io_inside_the_captured_step(dev):
    """With pinned host buffers attached, the captured step copies its frame in
    and its loss and pose out: the same results as set_observation + step, and
    a new frame placed in the buffer is the one the next replay uses (no map
    or pose update, so that every frame renders the same map bit for bit)."""
    a = _agent(dev, map=False, track=False)
    b = _agent(dev, map=False, track=False)
    H, W = a.cam.height, a.cam.width
    rng = np.random.default_rng(4)
    frames = [(torch.as_tensor(rng.uniform(0, 1, (H, W, 3)).astype(np.float32)).pin_memory(),
               torch.as_tensor(rng.uniform(1, 3, (H, W)).astype(np.float32)).pin_memory()) for _ in range(2)]
    h_rgb = torch.empty(H, W, 3).pin_memory()
    h_depth = torch.empty(H, W).pin_memory()
    h_loss = torch.empty(1).pin_memory()
    h_pose = torch.empty(4, 4).pin_memory()
    b.attach_host_io(h_rgb, h_depth, h_loss, h_pose)
    h_rgb.copy_(frames[0][0])
    h_depth.copy_(frames[0][1])
    b.capture(keep_state=True)
    for rgb, depth in frames:
        a.set_observation(rgb.to(dev), depth.to(dev))
        a.step()
        h_rgb.copy_(rgb)
        h_depth.copy_(depth)
        b.replay()
        torch.cuda.synchronize()
        assert torch.equal(a.obs_rgb, b.obs_rgb) and torch.equal(a.obs_depth, b.obs_depth)
        for k in ("rgb", "depth", "t_final", "max_id"):
            assert torch.equal(a.fb.image[k], b.fb.image[k]), k
        assert float(h_loss[0]) == pytest.approx(float(a.loss.item()), rel=1e-5)
        np.testing.assert_allclose(h_pose.numpy(), a.w2c.cpu().numpy(), atol=1e-6)
    with pytest.raises(ValueError):
        b.attach_host_io(torch.empty(H, W, 3), h_depth)  # not pinned


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


def _agents(dev, sizes, cams, **cfg):
    from paper_2412_09723_gb300.agent import Agent, StepConfig

    out = []
    for i, (n, cam) in enumerate(zip(sizes, cams)):
        sc = scenes.scene_room(n, 30 + i)
        w2c = scenes.perturbed_w2c(40 + i, 0.05, 3.0)
        a = Agent(sc, w2c, cam, dev, cfg=StepConfig(**cfg))
        a.render_observation_from(scenes.perturbed_w2c(50 + i, 0.01, 0.5, base=w2c))
        a.size_capacity(1.5)
        out.append(a)
    return out


SIZES = (15000, 40000, 90000)
CAMS = (scenes.Camera(320, 240, 262.5, 262.5, 160.0, 120.0), scenes.Camera(400, 300, 300.0, 300.0, 200.0, 150.0),
        scenes.Camera(600, 340, 300.0, 300.0, 300.0, 170.0))


def test_batched_step_equals_single_agent_steps(dev):
    from paper_2412_09723_gb300.batch import MultiAgentBatch

    solo = _agents(dev, SIZES, CAMS, map=False, track=False)
    mine = _agents(dev, SIZES, CAMS, map=False, track=False)
    for a in solo:
        a.step()
    batch = MultiAgentBatch(mine, shape=(128, 4, 128, 7))
    batch.step()
    torch.cuda.synchronize()
    for a, b in zip(solo, mine):
        for k in ("rgb", "depth", "sil", "t_final", "n_contrib", "max_id"):
            assert torch.equal(a.fb.image[k], b.fb.image[k]), k
        for ga, gb in zip(a.grads, b.grads):
            ref = ga.double()
            tol = 1e-3 * float(ref.pow(2).mean().sqrt()) + 1e-3 * ref.abs()
            assert bool(((ga.double() - gb.double()).abs() <= tol).all())
        assert torch.allclose(a.d_pose, b.d_pose, rtol=1e-3, atol=1e-3 * float(a.d_pose.abs().max()))
    # the captured graph of the batch replays the same forward
    batch.capture()
    batch.replay()
    torch.cuda.synchronize()
    for a, b in zip(solo, mine):
        assert torch.equal(a.fb.image["max_id"], b.fb.image["max_id"])
    assert batch.status() == 0


def test_autotune_picks_a_candidate(dev, tmp_path):
    from paper_2412_09723_gb300.batch import MultiAgentBatch

    agents = _agents(dev, SIZES[:2], CAMS[:2])
    batch = MultiAgentBatch(agents)
    cands = [(128, 4, 128, 7), (256, 2, 256, 4)]
    entry = batch.autotune(candidates=cands, reps=2, cache_path=str(tmp_path / "tune.json"))
    assert tuple(entry["shape"]) in cands and len(entry["tried"]) == 2
    again = batch.autotune(candidates=cands, reps=2, cache_path=str(tmp_path / "tune.json"))
    assert again["shape"] == entry["shape"]


def test_agent_prune_matches_oracle_and_keeps_stepping(dev):
    """Algorithm 1 on a resident map after some mapping steps: the kept map
    and Adam moments are the oracle's compaction of the device state, the
    pruned map renders exactly as the oracle renders the same Gaussians, and
    the agent keeps stepping (and capturing) at the new size."""
    import oracle
    from oracle import consensus as C

    a = _agent(dev)
    rng = np.random.default_rng(4)
    with torch.no_grad():  # make every criterion bite on some Gaussians
        idx = torch.as_tensor(rng.choice(a.n, 3000, replace=False), device=dev)
        a.params[3][idx[:1000]] = -7.0                   # transparent
        a.params[1][idx[1000:2000], 0] = float(np.log(0.3))  # large
        a.params[1][idx[2000:], 1] = a.params[1][idx[2000:], 0] + 4.0  # elongated
    for _ in range(3):
        a.step()
    torch.cuda.synchronize()
    state = [t.cpu().numpy() for t in (*a.params, *a.m, *a.v)]
    mask = C.prune_mask(state[3], state[1], oracle.exp_f32)
    ref = C.prune(state, mask)
    k = a.prune()
    assert k == int((~mask).sum()) and k == a.n
    assert a.n < 60000 - 2500
    for got, want in zip((*a.params, *a.m, *a.v), ref):
        assert np.array_equal(got.cpu().numpy(), want)
    a.forward()
    torch.cuda.synchronize()
    scene = scenes.Scene(*(t.cpu().numpy() for t in a.params))
    refimg = oracle.render_fwd(scene, a.w2c.cpu().numpy(), a.cam, np.zeros(3, np.float32))
    for key in ("n_contrib", "max_id"):
        assert np.array_equal(a.fb.image[key].cpu().numpy(), refimg[key]), key
    a.size_capacity(1.5)
    a.capture()
    for _ in range(3):
        a.replay()
    torch.cuda.synchronize()
    assert a.status() == 0 and np.isfinite(float(a.loss.item()))
