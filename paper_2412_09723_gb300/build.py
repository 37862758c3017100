"""Build the C-ABI CUDA library libsplat_gb300.so in-tree, for sm_103a only.

Every translation unit is compiled with --fmad=false (fused multiply-adds
only where the source writes them) and IEEE division / square root (nvcc's
defaults, never --use_fast_math), which the bit-exact parity of tile rects,
sort keys and maximum-weight ids relies on.

With SPLAT_FAST_EXP=1 in the environment a second library,
libsplat_gb300_fastexp.so, is built (and loaded by the binding) in which the
exponential is the hardware __expf instead of the project exponential: it
measures what the bit-exact exponential costs.  Its results are not the
oracle's bit for bit (only the image and gradient tolerances can hold), so it
is a measurement build, never the default.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
FAST_EXP = os.environ.get("SPLAT_FAST_EXP", "") == "1"
BUILD = os.path.join(HERE, "_build_fastexp" if FAST_EXP else "_build")
LIB = os.path.join(HERE, "libsplat_gb300_fastexp.so" if FAST_EXP else "libsplat_gb300.so")
SOURCES = ["api.cu", "project.cu", "binsort.cu", "render.cu", "assoc.cu", "profile.cu", "noalloc.cu", "consensus.cu"]
HEADERS = ["common.cuh", "internal.cuh", "segsort.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"] + (["-DSPLAT_FAST_EXP=1"] if FAST_EXP else [])


def nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsplat_gb300.so")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(os.path.dirname(HERE), "include", "splat.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (in parallel) and link; returns the path of the shared library."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
