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


# the binding's ctypes structures and the header's typedefs they mirror
_STRUCTS = {"CCamera": "splat_camera", "CGaussians": "splat_gaussians", "CGaussiansGrad": "splat_gaussians_grad",
            "CProjected": "splat_projected", "CImage": "splat_image", "CL1": "splat_l1",
            "CPoseAdam": "splat_pose_adam", "CView": "splat_view", "CColumn": "splat_column",
            "CBatchShape": "splat_batch_shape"}


def test_header_is_plain_c_and_the_binding_mirrors_its_structs(tmp_path):
    """include/splat.h compiles as C99 on its own (plain types and pointers
    only), and every ctypes structure of the binding has the size and field
    offsets of the C struct it mirrors, field by field by name."""
    import shutil
    import subprocess

    import pytest

    from paper_2412_09723_gb300 import binding as B

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "splat.h"', "int main(void) {"]
    want = []
    for cls, cname in _STRUCTS.items():
        py = getattr(B, cls)
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append(getattr(py, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want
