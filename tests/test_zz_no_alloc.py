"""splat_bin_sort_static: binning and sorting for callers that cannot
allocate device memory (for instance a real-time loop whose memory was
reserved once at start-up), using the library's static scratch array.

Checked through the C ABI against splat_bin_sort with a caller workspace on
two calls in a row (different scenes, so the second call runs on scratch left
over by the first); the outputs are integer data and must be identical.  The
file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2412_09723_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(sc, w2c, cam, dev):
    from paper_2412_09723_gb300 import binding as B
    from paper_2412_09723_gb300 import rasterizer as R

    p = [torch.as_tensor(a, device=dev) for a in sc.arrays()]
    fb = R.FrameBuffers(sc.n, cam, dev, want_keys=True)
    R.project(B.gaussians_struct(*p), torch.as_tensor(w2c, device=dev), fb)
    R.bin_sort(fb)  # caller-workspace path; also sizes the capacity
    torch.cuda.synchronize()
    return fb


def _run_static(fb, dev):
    from paper_2412_09723_gb300 import binding as B

    keys = torch.full((fb.capacity,), -1, dtype=torch.int64, device=dev)
    vals = torch.full((fb.capacity,), -1, dtype=torch.int32, device=dev)
    ranges = torch.full_like(fb.ranges, -1)
    k_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    B.splat_bin_sort_static(fb.cproj, fb.n, fb.ccam, keys, vals, fb.capacity, k_dev, ranges, status)
    torch.cuda.synchronize()
    return keys, vals, ranges, int(k_dev.item()), int(status.item())


def test_static_scratch_matches_workspace_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    cases = [scenes.workload_small_forward()[:3],
             (scenes.scene_room(20000, 5), scenes.perturbed_w2c(6, 0.1, 10.0),
              scenes.Camera(200, 150, 120.0, 120.0, 100.0, 75.0))]
    for sc, w2c, cam in cases:
        fb = _setup(sc, w2c, cam, dev)
        k_ref = int(fb.k_dev.item())
        keys, vals, ranges, k, status = _run_static(fb, dev)
        assert status == 0 and k == k_ref > 0
        assert torch.equal(vals[:k], fb.vals[:k])
        assert torch.equal(keys[:k], fb.keys[:k])
        assert torch.equal(ranges, fb.ranges)


def test_static_scratch_call_allocates_nothing():
    """After a first call, a call with preallocated outputs changes neither
    torch's allocated bytes nor the device's free memory."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_09723_gb300 import binding as B

    dev = torch.device("cuda:0")
    sc, w2c, cam = scenes.workload_small_forward()[:3]
    fb = _setup(sc, w2c, cam, dev)
    keys = torch.zeros(fb.capacity, dtype=torch.int64, device=dev)
    vals = torch.zeros(fb.capacity, dtype=torch.int32, device=dev)
    ranges = torch.zeros_like(fb.ranges)
    k_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    call = lambda: B.splat_bin_sort_static(fb.cproj, fb.n, fb.ccam, keys, vals, fb.capacity, k_dev, ranges, status)
    call()
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0])
    call()
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0])
    assert after == before
    assert int(status.item()) == 0 and torch.equal(vals[: int(k_dev.item())], fb.vals[: int(fb.k_dev.item())])


def test_static_scratch_rejects_oversized_problems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_09723_gb300 import binding as B

    dev = torch.device("cuda:0")
    sc, w2c, cam = scenes.workload_small_forward()[:3]
    fb = _setup(sc, w2c, cam, dev)
    limit = B.splat_bin_sort_static_scratch_bytes()
    too_big = limit  # duplicates capacity whose scratch alone exceeds the array
    dummy = torch.zeros(1, dtype=torch.int32, device=dev)
    k_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(B.SplatError) as e:
        B.splat_bin_sort_static(fb.cproj, fb.n, fb.ccam, None, dummy, too_big, k_dev, fb.ranges, dummy)
    assert e.value.code == B.SPLAT_EINVAL
