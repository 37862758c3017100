"""The batched multi-agent step (one persistent forward and one persistent
backward launch over several agents' views, Sec. 3.6) against the CPU oracle
directly, through `MultiAgentBatch.step`.

- three small agents of uneven map sizes and frame shapes, whole frames: the
  images of the persistent forward launch equal the oracle's bit for bit, and
  every parameter gradient and the pose gradient of every agent (persistent
  backward launch, then the projection adjoint) are within the gradient rule
  of the oracle's adjoint of the same L1 loss;
- the three agents of the batched workload (150k, 400k and 900k Gaussians at
  1200x680) in row bands (a middle tile row and the ragged last tile row):
  each agent's observation equals its own render outside the bands, so that
  the L1 gradient vanishes there exactly, and the oracle differentiates the
  bands alone (the adjoint is linear in the upstream gradients, so the bands'
  gradients add up).

Gradient rule: |g - g_ref| <= 1e-3 |g_ref| + 1e-3 rms(g_ref) per tensor."""
import numpy as np
import pytest

import oracle
from paper_2412_09723_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_GRAD = 1e-3
NAMES = ("mean", "log_scale", "quat", "opacity_logit", "rgb")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_09723_gb300 import binding

    binding.load()
    return torch.device("cuda:0")


def _assert_grad_close(got, ref, name):
    got, ref = np.asarray(got, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    rms = float(np.sqrt(np.mean(ref ** 2))) if ref.size else 0.0
    err = np.abs(got - ref)
    bound = RTOL_GRAD * np.abs(ref) + RTOL_GRAD * rms
    bad = err > bound
    assert not bad.any(), f"{name}: {bad.sum()} of {bad.size} out of tolerance; worst {np.max(err / (bound + 1e-30))}"


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a


def _assert_image_rows(fb, ref, r0, r1, what):
    for k in ("rgb", "depth", "sil", "t_final", "n_contrib", "max_id"):
        got = fb.image[k].cpu().numpy()[r0:r1]
        assert np.array_equal(_bits(got), _bits(ref[k][r0:r1])), f"{what}: {k} rows {r0}..{r1}"


def _make_agents(dev, specs):
    from paper_2412_09723_gb300.agent import Agent, StepConfig

    cfg = dict(map=False, track=False, assoc=False)  # the step leaves the gradients and d_pose in place
    return [Agent(sc, w2c, cam, dev, cfg=StepConfig(**cfg)) for sc, w2c, cam in specs]


def _check_agent_grads(a, ref, what):
    for name, got in zip(NAMES, a.grads):
        _assert_grad_close(got.cpu().numpy(), ref[name], f"{what}: {name}")
    _assert_grad_close(a.d_pose.cpu().numpy(), ref["pose"], f"{what}: pose")


SMALL = ((15000, scenes.Camera(320, 240, 262.5, 262.5, 160.0, 120.0)),
         (40000, scenes.Camera(400, 300, 300.0, 300.0, 200.0, 150.0)),
         (90000, scenes.Camera(600, 340, 300.0, 300.0, 300.0, 170.0)))


@pytest.mark.parametrize("shape", [(256, 4, 64, 8), (64, 8, 256, 10)])
def test_batched_step_matches_oracle_whole_frames(dev, shape):
    from paper_2412_09723_gb300.batch import MultiAgentBatch

    specs, targets = [], []
    bg = np.zeros(3, np.float32)
    for i, (n, cam) in enumerate(SMALL):
        sc = scenes.scene_room(n, 60 + i)
        w2c = scenes.perturbed_w2c(70 + i, 0.05, 3.0)
        specs.append((sc, w2c, cam))
        targets.append(oracle.render_fwd(sc, scenes.perturbed_w2c(80 + i, 0.01, 0.5, base=w2c), cam, bg))
    agents = _make_agents(dev, specs)
    for a, t in zip(agents, targets):
        a.set_observation(torch.as_tensor(t["rgb"], device=dev), torch.as_tensor(t["depth"], device=dev))
        a.size_capacity(1.5)
    batch = MultiAgentBatch(agents, shape=shape)
    batch.step()
    torch.cuda.synchronize()
    assert batch.status() == 0
    for i, (a, (sc, w2c, cam), t) in enumerate(zip(agents, specs, targets)):
        ref = oracle.render_fwd(sc, w2c, cam, bg)
        _assert_image_rows(a.fb, ref, 0, cam.height, f"agent {i}")
        _, g_rgb, g_depth = oracle.loss_l1(ref["rgb"], ref["depth"], t["rgb"], t["depth"], 1.0, 0.5)
        _check_agent_grads(a, oracle.render_bwd(sc, w2c, cam, bg, g_rgb, g_depth), f"agent {i}")


BANDS = ((336, 352), (672, 680))  # a middle tile row; the ragged last tile row of a 680-row frame


def test_batched_step_matches_oracle_full_size_bands(dev):
    """150k / 400k / 900k Gaussians at 1200x680 in one batched step."""
    from paper_2412_09723_gb300.batch import MultiAgentBatch

    specs = scenes.workload_multi_agent()
    agents = _make_agents(dev, specs)
    bg = np.zeros(3, np.float32)
    band_targets = []
    for i, (a, (sc, w2c, cam)) in enumerate(zip(agents, specs)):
        a.size_capacity(1.5)
        a.forward()
        # outside the bands the observation is the agent's own render (zero L1
        # gradient); inside them, the oracle's render from a pose 1 cm / 0.5 deg away
        w2c_t = scenes.perturbed_w2c(700 + i, 0.01, 0.5, base=w2c)
        t_rgb = a.fb.image["rgb"].clone()
        t_depth = a.fb.image["depth"].clone()
        full = dict(rgb=np.zeros((cam.height, cam.width, 3), np.float32),
                    depth=np.zeros((cam.height, cam.width), np.float32))
        for r0, r1 in BANDS:
            t = oracle.render_fwd(sc, w2c_t, cam, bg, rows=(r0, r1))
            t_rgb[r0:r1] = torch.as_tensor(t["rgb"][r0:r1], device=dev)
            t_depth[r0:r1] = torch.as_tensor(t["depth"][r0:r1], device=dev)
            full["rgb"][r0:r1], full["depth"][r0:r1] = t["rgb"][r0:r1], t["depth"][r0:r1]
        a.set_observation(t_rgb, t_depth)
        band_targets.append(full)
    batch = MultiAgentBatch(agents)
    batch.step()
    torch.cuda.synchronize()
    assert batch.status() == 0
    for i, (a, (sc, w2c, cam), tgt) in enumerate(zip(agents, specs, band_targets)):
        # the oracle's render of the bands (zero elsewhere, like the band target)
        mine = dict(rgb=np.zeros_like(tgt["rgb"]), depth=np.zeros_like(tgt["depth"]))
        for r0, r1 in BANDS:
            ref = oracle.render_fwd(sc, w2c, cam, bg, rows=(r0, r1))
            _assert_image_rows(a.fb, ref, r0, r1, f"agent {i} ({sc.n} Gaussians)")
            mine["rgb"][r0:r1], mine["depth"][r0:r1] = ref["rgb"][r0:r1], ref["depth"][r0:r1]
        # full-frame means (the same scale as the step's loss), zero gradient outside the bands
        _, g_rgb, g_depth = oracle.loss_l1(mine["rgb"], mine["depth"], tgt["rgb"], tgt["depth"], 1.0, 0.5)
        total = None
        for r0, r1 in BANDS:
            part = oracle.render_bwd(sc, w2c, cam, bg, g_rgb, g_depth, rows=(r0, r1))
            total = part if total is None else {k: total[k] + part[k] for k in total}
        assert np.abs(total["pose"]).max() > 0
        _check_agent_grads(a, total, f"agent {i} ({sc.n} Gaussians)")
