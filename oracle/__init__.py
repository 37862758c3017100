"""Python access to the CPU oracle (oracle/splat_oracle.cpp).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline / reference leg of bench.py may import this module.  The product
package never imports it and shares no code with it.

Inputs are plain numpy arrays (a `scenes.Scene`-like object with .mean,
.log_scale, .quat, .opacity_logit, .rgb, and a camera with .width, .height,
.fx, .fy, .cx, .cy, .z_near and optionally .max_dist, the distance beyond
which Gaussians are not candidates); outputs are numpy arrays.  `dtype` selects the
float32 instantiation (bit-level parity; project exp) or the float64 one
(std::exp; finite-difference checks).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "splat_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libsplat_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libsplat_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None
_active = threading.local()

CFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
# the timed CPU baseline: the same source with its OpenMP loops switched on
CFLAGS_OMP = CFLAGS + ["-fopenmp"]


def _build_one(path, flags, force):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *flags, _SRC, "-o", tmp])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (float ops in source order, no contraction);
    single-threaded: this is the build every parity check uses."""
    return _build_one(_LIB, CFLAGS, force)


def build_omp(force: bool = False) -> str:
    """Compile the multi-threaded build of the same source (the timed CPU
    baseline; its forward results equal the parity build's, its adjoint sums
    are grouped per thread)."""
    return _build_one(_LIB_OMP, CFLAGS_OMP, force)


def lib():
    """The library the calls below use: the parity build, or the
    multi-threaded build inside a `parallel()` block."""
    L = getattr(_active, "lib", None)
    return L if L is not None else _parity_lib()


def _parity_lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            _declare(L)
            _lib = L
    return _lib


def _omp_lib():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            L = ctypes.CDLL(build_omp())
            _declare(L)
            _lib_omp = L
    return _lib_omp


@contextlib.contextmanager
def parallel(threads: int | None = None):
    """Run the oracle calls of the block on the multi-threaded build (for
    timing only; parity checks use the single-threaded build).  Yields the
    number of threads."""
    L = _omp_lib()
    if threads:
        L.oracle_set_threads(int(threads))
    prev = getattr(_active, "lib", None)
    _active.lib = L
    try:
        yield int(L.oracle_threads())
    finally:
        _active.lib = prev


def threads() -> int:
    """Threads of the library in use (1 for the parity build)."""
    return int(lib().oracle_threads())


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_F = ctypes.c_float


def _declare(L):
    L.oracle_threads.argtypes = []
    L.oracle_threads.restype = ctypes.c_int
    L.oracle_set_threads.argtypes = [ctypes.c_int]
    L.oracle_set_threads.restype = None
    L.oracle_exp_f32.argtypes = [_I64, _P, _P]
    L.oracle_exp_f32.restype = None
    for suf in ("f32", "f64"):
        getattr(L, f"oracle_project_{suf}").argtypes = [_I64] + [_P] * 13
        getattr(L, f"oracle_project_{suf}").restype = ctypes.c_int
        getattr(L, f"oracle_render_fwd_{suf}").argtypes = [_I64] + [_P] * 17 + [_I32, _I32]
        getattr(L, f"oracle_render_fwd_{suf}").restype = ctypes.c_int
        getattr(L, f"oracle_render_bwd_{suf}").argtypes = [_I64] + [_P] * 19 + [_I32, _I32]
        getattr(L, f"oracle_render_bwd_{suf}").restype = ctypes.c_int
    L.oracle_bin_f32.argtypes = [_I64] + [_P] * 7 + [_I64, _P, _P, _P]
    L.oracle_bin_f32.restype = _I64
    L.oracle_loss_l1_f32.argtypes = [_I64, _P, _P, _P, _P, _F, _F, _P, _P]
    L.oracle_loss_l1_f32.restype = ctypes.c_double
    L.oracle_adam_f32.argtypes = [_I64, _P, _P, _P, _P, _I32, _F, _F, _F, _F]
    L.oracle_adam_f32.restype = None
    L.oracle_assoc.argtypes = [_I64, _P, _P, _P, _P, _F, _I64, _P, _P]
    L.oracle_assoc.restype = _I64


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _suffix(dtype):
    dt = np.dtype(dtype)
    if dt == np.float32:
        return "f32"
    if dt == np.float64:
        return "f64"
    raise ValueError(f"oracle supports float32/float64, not {dt}")


def _scene_args(scene, dtype):
    return [_c(scene.mean, dtype), _c(scene.log_scale, dtype), _c(scene.quat, dtype),
            _c(scene.opacity_logit, dtype)]


def _cam_args(cam, dtype):
    ci = np.array([cam.width, cam.height], dtype=np.int32)
    cf = np.array([cam.fx, cam.fy, cam.cx, cam.cy, cam.z_near, getattr(cam, "max_dist", 0.0)], dtype=dtype)
    return ci, cf


def set_exact_tiles(on: bool):
    """Test switch: with False, every tile of a Gaussian's rect is a member
    (the images must be the same either way)."""
    L = lib()
    L.oracle_set_exact_tiles.argtypes = [ctypes.c_int]
    L.oracle_set_exact_tiles.restype = None
    L.oracle_set_exact_tiles(1 if on else 0)


def exp_f32(x):
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib().oracle_exp_f32(x.size, _ptr(x), _ptr(y))
    return y


def project(scene, w2c, cam, dtype=np.float32):
    """Per-Gaussian projection: xyzo [N,4] = (u, v, depth, opacity), conic [N,4]
    = (a, b, c, 0), cov [N,3], radius [N], rect [N,4] (tile xmin, ymin, xmax,
    ymax; half open), tiles_touched [N].  Culled Gaussians are all zero."""
    n = scene.n
    args = _scene_args(scene, dtype)
    w = _c(w2c, dtype)
    ci, cf = _cam_args(cam, dtype)
    out = dict(xyzo=np.zeros((n, 4), dtype), conic=np.zeros((n, 4), dtype), cov=np.zeros((n, 3), dtype),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               tiles_touched=np.zeros(n, np.int32))
    getattr(lib(), f"oracle_project_{_suffix(dtype)}")(
        n, *map(_ptr, args), _ptr(w), _ptr(ci), _ptr(cf), _ptr(out["xyzo"]), _ptr(out["conic"]),
        _ptr(out["cov"]), _ptr(out["radius"]), _ptr(out["rect"]), _ptr(out["tiles_touched"]))
    return out


def bin_sort(scene, w2c, cam):
    """Sorted (tile, depth) keys, Gaussian ids and per-tile [start, end) ranges."""
    args = _scene_args(scene, np.float32)
    w = _c(w2c, np.float32)
    ci, cf = _cam_args(cam, np.float32)
    ranges = np.zeros((cam.n_tiles, 2), np.uint32)
    L = lib()
    k = L.oracle_bin_f32(scene.n, *map(_ptr, args), _ptr(w), _ptr(ci), _ptr(cf), 0, None, None, _ptr(ranges))
    keys = np.zeros(max(k, 1), np.uint64)
    vals = np.zeros(max(k, 1), np.uint32)
    L.oracle_bin_f32(scene.n, *map(_ptr, args), _ptr(w), _ptr(ci), _ptr(cf), k, _ptr(keys), _ptr(vals), _ptr(ranges))
    return keys[:k], vals[:k], ranges


def render_fwd(scene, w2c, cam, bg, dtype=np.float32, rows=None, signature=None):
    """Forward render: rgb [H,W,3], depth, sil, t_final [H,W], n_contrib, max_id
    [H,W] int32, the hash of all discrete decisions (`signature`: by default
    in the parity build only; 0 when not taken) and the summed n_contrib.
    `rows` = (row0, row1) renders only that band (other pixels stay zero)."""
    if signature is None:
        signature = threads() == 1
    H, W = cam.height, cam.width
    args = _scene_args(scene, dtype) + [_c(scene.rgb, dtype)]
    w = _c(w2c, dtype)
    ci, cf = _cam_args(cam, dtype)
    b = _c(bg, dtype)
    out = dict(rgb=np.zeros((H, W, 3), dtype), depth=np.zeros((H, W), dtype), sil=np.zeros((H, W), dtype),
               t_final=np.zeros((H, W), dtype), n_contrib=np.zeros((H, W), np.int32),
               max_id=np.zeros((H, W), np.int32))
    sig = np.zeros(1, np.uint64)
    npairs = np.zeros(1, np.int64)
    getattr(lib(), f"oracle_render_fwd_{_suffix(dtype)}")(
        scene.n, *map(_ptr, args), _ptr(w), _ptr(ci), _ptr(cf), _ptr(b), _ptr(out["rgb"]),
        _ptr(out["depth"]), _ptr(out["sil"]), _ptr(out["t_final"]), _ptr(out["n_contrib"]),
        _ptr(out["max_id"]), _ptr(sig) if signature else None, _ptr(npairs), *(rows or (0, H)))
    out["signature"] = int(sig[0])
    out["n_pairs"] = int(npairs[0])
    return out


def render_bwd(scene, w2c, cam, bg, g_rgb, g_depth=None, g_sil=None, dtype=np.float32, rows=None):
    """Adjoint of render_fwd for upstream per-pixel gradients.  Returns the
    gradients of mean, log_scale, quat, opacity_logit, rgb, the 6-vector pose
    gradient (rho, phi) of the left perturbation exp(delta^) w2c, and the
    per-Gaussian screen-space gradients d2d [N,10] = (du, dv, dconic a, b, c,
    dopacity, drgb[3], ddepth).  `rows` = (row0, row1) differentiates only the
    pixels of that band."""
    n = scene.n
    args = _scene_args(scene, dtype) + [_c(scene.rgb, dtype)]
    w = _c(w2c, dtype)
    ci, cf = _cam_args(cam, dtype)
    b = _c(bg, dtype)
    gr = _c(g_rgb, dtype)
    gd = None if g_depth is None else _c(g_depth, dtype)
    gs = None if g_sil is None else _c(g_sil, dtype)
    out = dict(mean=np.zeros((n, 3), dtype), log_scale=np.zeros((n, 3), dtype), quat=np.zeros((n, 4), dtype),
               opacity_logit=np.zeros(n, dtype), rgb=np.zeros((n, 3), dtype), pose=np.zeros(6, dtype),
               d2d=np.zeros((n, 10), dtype))
    getattr(lib(), f"oracle_render_bwd_{_suffix(dtype)}")(
        n, *map(_ptr, args), _ptr(w), _ptr(ci), _ptr(cf), _ptr(b), _ptr(gr), _ptr(gd), _ptr(gs),
        _ptr(out["mean"]), _ptr(out["log_scale"]), _ptr(out["quat"]), _ptr(out["opacity_logit"]),
        _ptr(out["rgb"]), _ptr(out["pose"]), _ptr(out["d2d"]), *(rows or (0, cam.height)))
    return out


def loss_l1(rgb, depth, t_rgb, t_depth, w_rgb=1.0, w_depth=0.5):
    """L = w_rgb mean|C - C*| + w_depth mean|D - D*| and its image gradients."""
    rgb, depth, t_rgb, t_depth = (_c(a, np.float32) for a in (rgb, depth, t_rgb, t_depth))
    g_rgb = np.zeros_like(rgb)
    g_depth = np.zeros_like(depth)
    L = lib().oracle_loss_l1_f32(depth.size, _ptr(rgb), _ptr(depth), _ptr(t_rgb), _ptr(t_depth), w_rgb,
                                 w_depth, _ptr(g_rgb), _ptr(g_depth))
    return float(L), g_rgb, g_depth


def adam(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """In-place textbook Adam on float32 arrays; returns (param, m, v)."""
    param, grad, m, v = (_c(a, np.float32).copy() for a in (param, grad, m, v))
    lib().oracle_adam_f32(param.size, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), step, lr, beta1, beta2, eps)
    return param, m, v


def assoc(id_a, t_a, id_b, t_b, t_max=0.5):
    """Unique (id_a, id_b) pairs sorted ascending, with pixel counts."""
    id_a, id_b = _c(id_a, np.int32).ravel(), _c(id_b, np.int32).ravel()
    t_a, t_b = _c(t_a, np.float32).ravel(), _c(t_b, np.float32).ravel()
    L = lib()
    m = L.oracle_assoc(id_a.size, _ptr(id_a), _ptr(t_a), _ptr(id_b), _ptr(t_b), t_max, 0, None, None)
    pairs = np.zeros((max(m, 1), 2), np.int32)
    counts = np.zeros(max(m, 1), np.int32)
    L.oracle_assoc(id_a.size, _ptr(id_a), _ptr(t_a), _ptr(id_b), _ptr(t_b), t_max, m, _ptr(pairs), _ptr(counts))
    return pairs[:m], counts[:m]
