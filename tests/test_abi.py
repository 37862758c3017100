"""The C-ABI library builds, loads without a GPU, and exports every function
include/splat.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "splat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(splat_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_five_calls():
    names = _declared()
    for n in ("splat_project", "splat_bin_sort", "splat_render_fwd", "splat_render_bwd", "splat_assoc"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2412_09723_gb300 import build

    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2412_09723_gb300 import binding

    assert sorted(binding.exported_symbols()) == _declared()


def test_binding_refuses_without_cuda():
    import pytest
    import torch

    from paper_2412_09723_gb300 import binding

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError):
        binding.load()
