"""Thin Python binding of libsplat_gb300.so (include/splat.h).

Argument marshalling only: every function here passes torch CUDA tensors'
device pointers and sizes to the C ABI entry point of the same name and
raises on a non-zero return code.  There is no CPU path: without a CUDA
device or without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_c_i32, _c_i64, _c_f, _c_p, _c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t

SPLAT_OK, SPLAT_EINVAL, SPLAT_ECAPACITY, SPLAT_ECUDA, SPLAT_ETIMEOUT, SPLAT_ENUMERIC = 0, 1, 2, 3, 4, 8


class SplatError(RuntimeError):
    def __init__(self, name, code, msg):
        super().__init__(f"{name} failed with code {code}: {msg}")
        self.code = code


class CCamera(ctypes.Structure):
    _fields_ = [("width", _c_i32), ("height", _c_i32), ("fx", _c_f), ("fy", _c_f), ("cx", _c_f), ("cy", _c_f),
                ("z_near", _c_f), ("max_dist", _c_f)]


class CGaussians(ctypes.Structure):
    _fields_ = [("mean", _c_p), ("log_scale", _c_p), ("quat", _c_p), ("opacity_logit", _c_p), ("rgb", _c_p),
                ("n", _c_i64)]


class CGaussiansGrad(ctypes.Structure):
    _fields_ = [("mean", _c_p), ("log_scale", _c_p), ("quat", _c_p), ("opacity_logit", _c_p), ("rgb", _c_p)]


class CProjected(ctypes.Structure):
    _fields_ = [("xyzo", _c_p), ("conic", _c_p), ("radius", _c_p), ("rect", _c_p), ("tiles_touched", _c_p)]


class CImage(ctypes.Structure):
    _fields_ = [("rgb", _c_p), ("depth", _c_p), ("sil", _c_p), ("t_final", _c_p), ("n_contrib", _c_p),
                ("max_id", _c_p), ("n_used", _c_p)]


class CL1(ctypes.Structure):
    _fields_ = [("t_rgb", _c_p), ("t_depth", _c_p), ("w_rgb", _c_f), ("w_depth", _c_f), ("d_rgb", _c_p),
                ("d_depth", _c_p), ("loss", _c_p)]


class CPoseAdam(ctypes.Structure):
    _fields_ = [("w2c", _c_p), ("m", _c_p), ("v", _c_p), ("step", _c_p), ("lr_t", ctypes.c_float),
                ("lr_r", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("counter", _c_p)]


class CView(ctypes.Structure):
    _fields_ = [("proj", CProjected), ("rgb", _c_p), ("n", _c_i64), ("vals", _c_p), ("ranges", _c_p),
                ("cam", CCamera), ("bg", ctypes.c_float * 3), ("image", CImage), ("d_rgb", _c_p), ("d_depth", _c_p),
                ("d_sil", _c_p), ("grad2d", _c_p), ("l1", ctypes.POINTER(CL1)), ("schedule", _c_p)]


class CColumn(ctypes.Structure):
    _fields_ = [("src", _c_p), ("dst", _c_p), ("width", _c_i32)]


class CBatchShape(ctypes.Structure):
    _fields_ = [("fwd_batch", _c_i32), ("fwd_ctas_per_sm", _c_i32), ("bwd_batch", _c_i32),
                ("bwd_ctas_per_sm", _c_i32)]


SPLAT_MAX_VIEWS = 16

_SIGS = {
    "splat_abi_version": ([], _c_i32),
    "splat_last_error": ([], ctypes.c_char_p),
    "splat_kernel_launches": ([], ctypes.c_uint64),
    "splat_profile_enable": ([ctypes.c_int], ctypes.c_int),
    "splat_profile_select": ([ctypes.c_char_p], ctypes.c_int),
    "splat_profile_read": ([_c_p, _c_sz, _c_p, _c_p, _c_i32, _c_p], ctypes.c_int),
    "splat_project": ([_c_p, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_bin_sort_workspace_size": ([_c_i64, _c_i64, _c_i32], _c_sz),
    "splat_bin_sort": ([_c_p, _c_i64, _c_p, _c_p, _c_p, _c_i64, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p], ctypes.c_int),
    "splat_bin_sort_static_scratch_bytes": ([], _c_sz),
    "splat_bin_sort_static": ([_c_p, _c_i64, _c_p, _c_p, _c_p, _c_i64, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_render_fwd": ([_c_p, _c_p, _c_i64, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_render_fwd_l1": ([_c_p, _c_p, _c_i64, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_tile_schedule_size": ([_c_i32], _c_sz),
    "splat_tile_schedule_order": ([_c_p, _c_i32, _c_p], ctypes.c_int),
    "splat_render_fwd_bwd_workspace_size": ([_c_i64, _c_i32], _c_sz),
    "splat_render_fwd_bwd": ([_c_p, _c_p, _c_i64, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p],
                             ctypes.c_int),
    "splat_render_bwd_workspace_size": ([_c_i64], _c_sz),
    "splat_render_bwd": ([_c_p] * 16 + [_c_sz, _c_p], ctypes.c_int),
    "splat_project_bwd": ([_c_p] * 8 + [_c_p], ctypes.c_int),
    "splat_project_bwd_adam": ([_c_p] * 8 + [_c_f, _c_f, _c_f, _c_p, _c_p, _c_i32, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_adam_culled": ([_c_p] * 5 + [_c_f, _c_f, _c_f, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_batch_workspace_size": ([], _c_sz),
    "splat_render_fwd_batch": ([_c_p, _c_i32, _c_p, _c_p, _c_sz, _c_p], ctypes.c_int),
    "splat_render_bwd_batch": ([_c_p, _c_i32, _c_p, _c_p, _c_sz, _c_p], ctypes.c_int),
    "splat_loss_l1": ([_c_p, _c_p, _c_p, _c_p, _c_i64, _c_f, _c_f, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_adam": ([_c_p, _c_p, _c_p, _c_p, _c_i64, _c_p, _c_f, _c_f, _c_f, _c_f, _c_p], ctypes.c_int),
    "splat_adam_groups": ([_c_i32, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_f, _c_f, _c_f, _c_i32, _c_p],
                          ctypes.c_int),
    "splat_pose_step": ([_c_p, _c_p, _c_p, _c_p, _c_p, _c_f, _c_f, _c_f, _c_f, _c_f, _c_p], ctypes.c_int),
    "splat_assoc_workspace_size": ([_c_i64], _c_sz),
    "splat_assoc": ([_c_p, _c_p, _c_p, _c_p, _c_i64, _c_i64, _c_i64, _c_f, _c_p, _c_p, _c_i64, _c_p, _c_p, _c_p,
                     _c_sz, _c_p], ctypes.c_int),
    "splat_pose_compose": ([_c_i32, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_pose_rel_grad": ([_c_i32, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_loss_consensus_workspace_size": ([_c_i32, _c_i32], _c_sz),
    "splat_loss_consensus": ([_c_p, _c_p, _c_p, _c_p, _c_i32, _c_i32, _c_f, _c_f, _c_f, _c_p, _c_p, _c_p, _c_p,
                              _c_sz, _c_p], ctypes.c_int),
    "splat_mahalanobis_system": ([_c_p, _c_p, _c_p, _c_p, _c_p, _c_i64, _c_p, _c_f, _c_p, _c_p], ctypes.c_int),
    "splat_mahalanobis_step": ([_c_p, _c_p, _c_p, _c_p, _c_p], ctypes.c_int),
    "splat_mahalanobis_system_step": ([_c_p, _c_p, _c_p, _c_p, _c_p, _c_i64, _c_p, _c_f, _c_p, _c_p, _c_p, _c_p],
                                      ctypes.c_int),
    "splat_prune_workspace_size": ([_c_i64], _c_sz),
    "splat_prune": ([_c_p, _c_f, _c_f, _c_f, _c_p, _c_i32, _c_p, _c_p, _c_p, _c_sz, _c_p], ctypes.c_int),
    "splat_exp_f32": ([_c_p, _c_p, _c_i64, _c_p], ctypes.c_int),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(require_cuda: bool = True):
    """Load (building first if stale) the CUDA library.  Raises when no CUDA
    device is present and `require_cuda` is set."""
    global _lib
    if require_cuda and not torch.cuda.is_available():
        raise RuntimeError("libsplat_gb300 needs a CUDA device (GB300, sm_103a); there is no CPU fallback")
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _p(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("splat: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("splat: expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(name, rc):
    if rc != SPLAT_OK:
        msg = load().splat_last_error().decode()
        raise SplatError(name, rc, msg)


def camera_struct(cam) -> CCamera:
    return CCamera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, cam.z_near, getattr(cam, "max_dist", 0.0))


def gaussians_struct(mean, log_scale, quat, opacity_logit, rgb) -> CGaussians:
    return CGaussians(_p(mean), _p(log_scale), _p(quat), _p(opacity_logit), _p(rgb), mean.shape[0])


def projected_struct(proj) -> CProjected:
    return CProjected(_p(proj["xyzo"]), _p(proj["conic"]), _p(proj["radius"]), _p(proj["rect"]),
                      _p(proj["tiles_touched"]))


def image_struct(img) -> CImage:
    return CImage(_p(img["rgb"]), _p(img["depth"]), _p(img["sil"]), _p(img["t_final"]), _p(img["n_contrib"]),
                  _p(img["max_id"]), _p(img.get("n_used")))


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def splat_abi_version() -> int:
    return int(load().splat_abi_version())


def splat_kernel_launches() -> int:
    return int(load().splat_kernel_launches())


def splat_profile_enable(on: bool):
    _check("splat_profile_enable", load().splat_profile_enable(1 if on else 0))


def splat_profile_select(kernel: str | None):
    _check("splat_profile_select", load().splat_profile_select(None if kernel is None else kernel.encode()))


def splat_profile_read(max_kernels: int = 64) -> dict:
    """{kernel name: (timed launches, total ms)} since the last read."""
    names = ctypes.create_string_buffer(8192)
    launches = (ctypes.c_int64 * max_kernels)()
    ms = (ctypes.c_double * max_kernels)()
    nk = ctypes.c_int32(0)
    _check("splat_profile_read", load().splat_profile_read(names, 8192, launches, ms, max_kernels, ctypes.byref(nk)))
    keys = [k for k in names.value.decode().split("\n") if k]
    return {k: (int(launches[i]), float(ms[i])) for i, k in enumerate(keys[:max_kernels])}


def splat_project(gaussians: CGaussians, cam: CCamera, w2c, proj: CProjected, stream=None):
    _check("splat_project", load().splat_project(ctypes.byref(gaussians), ctypes.byref(cam), _p(w2c),
                                                 ctypes.byref(proj), _stream(stream)))


def splat_bin_sort_workspace_size(n, capacity, n_tiles) -> int:
    return int(load().splat_bin_sort_workspace_size(n, capacity, n_tiles))


def splat_bin_sort(proj: CProjected, n, cam: CCamera, keys, vals, capacity, k_dev, ranges, status, ws, stream=None,
                   schedule=None):
    _check("splat_bin_sort", load().splat_bin_sort(
        ctypes.byref(proj), n, ctypes.byref(cam), _p(keys), _p(vals), capacity, _p(k_dev), _p(ranges),
        _p(schedule), _p(status), _p(ws), ws.numel() * ws.element_size(), _stream(stream)))


def splat_bin_sort_static_scratch_bytes() -> int:
    return int(load().splat_bin_sort_static_scratch_bytes())


def splat_bin_sort_static(proj: CProjected, n, cam: CCamera, keys, vals, capacity, k_dev, ranges, status,
                          stream=None):
    """splat_bin_sort with the library's static scratch array instead of a workspace."""
    _check("splat_bin_sort_static", load().splat_bin_sort_static(
        ctypes.byref(proj), n, ctypes.byref(cam), _p(keys), _p(vals), capacity, _p(k_dev), _p(ranges), _p(status),
        _stream(stream)))


def splat_render_fwd(proj: CProjected, rgb, n, vals, ranges, cam: CCamera, bg, image: CImage, stream=None):
    bgc = (ctypes.c_float * 3)(*[float(x) for x in bg])
    _check("splat_render_fwd", load().splat_render_fwd(
        ctypes.byref(proj), _p(rgb), n, _p(vals), _p(ranges), ctypes.byref(cam), bgc, ctypes.byref(image),
        _stream(stream)))


def l1_struct(t_rgb, t_depth, w_rgb, w_depth, d_rgb, d_depth, loss) -> CL1:
    return CL1(_p(t_rgb), _p(t_depth), w_rgb, w_depth, _p(d_rgb), _p(d_depth), _p(loss))


def splat_render_fwd_l1(proj: CProjected, rgb, n, vals, ranges, cam: CCamera, bg, image: CImage, l1,
                        stream=None, schedule=None):
    bgc = (ctypes.c_float * 3)(*[float(x) for x in bg])
    _check("splat_render_fwd_l1", load().splat_render_fwd_l1(
        ctypes.byref(proj), _p(rgb), n, _p(vals), _p(ranges), ctypes.byref(cam), bgc, ctypes.byref(image),
        None if l1 is None else ctypes.byref(l1), _p(schedule), _stream(stream)))



def splat_tile_schedule_size(n_tiles) -> int:
    return int(load(require_cuda=False).splat_tile_schedule_size(n_tiles))


def splat_tile_schedule_order(schedule, n_tiles, stream=None):
    _check("splat_tile_schedule_order", load().splat_tile_schedule_order(_p(schedule), n_tiles, _stream(stream)))


def splat_render_fwd_bwd_workspace_size(n, n_tiles) -> int:
    return int(load(require_cuda=False).splat_render_fwd_bwd_workspace_size(n, n_tiles))


def splat_render_fwd_bwd(proj: CProjected, rgb, n, vals, ranges, cam: CCamera, bg, image: CImage, l1: CL1, status,
                         ws, stream=None, schedule=None):
    """Forward render with the L1 terms and the screen-space backward in one
    launch; the screen-space gradients are left at the start of `ws`."""
    bgc = (ctypes.c_float * 3)(*[float(x) for x in bg])
    _check("splat_render_fwd_bwd", load().splat_render_fwd_bwd(
        ctypes.byref(proj), _p(rgb), n, _p(vals), _p(ranges), ctypes.byref(cam), bgc, ctypes.byref(image),
        ctypes.byref(l1), _p(schedule), _p(status), _p(ws), ws.numel() * ws.element_size(), _stream(stream)))


def splat_render_bwd_workspace_size(n) -> int:
    return int(load().splat_render_bwd_workspace_size(n))


def splat_render_bwd(gaussians: CGaussians, proj: CProjected, cam: CCamera, w2c, vals, ranges, image: CImage, bg,
                     d_rgb, d_depth, d_sil, grads: CGaussiansGrad, d_pose, d2d, ws, stream=None, schedule=None):
    bgc = (ctypes.c_float * 3)(*[float(x) for x in bg])
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check("splat_render_bwd", load().splat_render_bwd(
        ctypes.byref(gaussians), ctypes.byref(proj), ctypes.byref(cam), _p(w2c), _p(vals), _p(ranges),
        _p(schedule), ctypes.byref(image), bgc, _p(d_rgb), _p(d_depth), _p(d_sil), None if grads is None else ctypes.byref(grads),
        _p(d_pose), _p(d2d), _p(ws), wsb, _stream(stream)))


def splat_project_bwd(gaussians: CGaussians, proj: CProjected, cam: CCamera, w2c, grad2d, grads: CGaussiansGrad,
                      d_pose, d2d=None, stream=None):
    _check("splat_project_bwd", load().splat_project_bwd(
        ctypes.byref(gaussians), ctypes.byref(proj), ctypes.byref(cam), _p(w2c), _p(grad2d),
        None if grads is None else ctypes.byref(grads), _p(d_pose), _p(d2d), _stream(stream)))


def splat_project_bwd_adam(gaussians: CGaussians, proj: CProjected, cam: CCamera, w2c, grad2d, m: CGaussiansGrad,
                           v: CGaussiansGrad, lr, step, d_pose, beta1=0.9, beta2=0.999, eps=1e-15, stream=None,
                           culled=True, seen=None, pose=None):
    """`gaussians`' arrays are updated in place; `lr`: 5 step sizes (mean,
    log_scale, quat, opacity_logit, rgb); `step`: device int32[1] (t >= 1);
    `culled`: also step the culled Gaussians (else splat_adam_culled does);
    `seen`: the optional bitmap of Gaussians whose moments may be nonzero;
    `pose`: an optional CPoseAdam (the pose's Adam step in the same launch)."""
    lrc = (ctypes.c_float * 5)(*[float(x) for x in lr])
    _check("splat_project_bwd_adam", load().splat_project_bwd_adam(
        ctypes.byref(gaussians), ctypes.byref(proj), ctypes.byref(cam), _p(w2c), _p(grad2d), ctypes.byref(m),
        ctypes.byref(v), lrc, beta1, beta2, eps, _p(step), _p(seen), 1 if culled else 0, _p(d_pose),
        None if pose is None else ctypes.byref(pose), _stream(stream)))


def splat_adam_culled(gaussians: CGaussians, radius, m: CGaussiansGrad, v: CGaussiansGrad, lr, step, beta1=0.9,
                      beta2=0.999, eps=1e-15, stream=None, seen=None):
    """The culled Gaussians' zero-gradient Adam step (see the header)."""
    lrc = (ctypes.c_float * 5)(*[float(x) for x in lr])
    _check("splat_adam_culled", load().splat_adam_culled(
        ctypes.byref(gaussians), _p(radius), ctypes.byref(m), ctypes.byref(v), lrc, beta1, beta2, eps, _p(step),
        _p(seen), _stream(stream)))


def splat_batch_workspace_size() -> int:
    return int(load().splat_batch_workspace_size())


def splat_render_fwd_batch(views, shape: CBatchShape | None, ws, stream=None):
    """`views`: ctypes array of CView."""
    _check("splat_render_fwd_batch", load().splat_render_fwd_batch(
        views, len(views), None if shape is None else ctypes.byref(shape), _p(ws), ws.numel() * ws.element_size(),
        _stream(stream)))


def splat_render_bwd_batch(views, shape: CBatchShape | None, ws, stream=None):
    _check("splat_render_bwd_batch", load().splat_render_bwd_batch(
        views, len(views), None if shape is None else ctypes.byref(shape), _p(ws), ws.numel() * ws.element_size(),
        _stream(stream)))


def splat_loss_l1(rgb, depth, target_rgb, target_depth, w_rgb, w_depth, d_rgb, d_depth, loss, stream=None):
    _check("splat_loss_l1", load().splat_loss_l1(
        _p(rgb), _p(depth), _p(target_rgb), _p(target_depth), depth.numel(), w_rgb, w_depth, _p(d_rgb), _p(d_depth),
        _p(loss), _stream(stream)))


def splat_adam(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """`step`: device int32[1] tensor holding the Adam step t >= 1."""
    _check("splat_adam", load().splat_adam(_p(param), _p(grad), _p(m), _p(v), param.numel(), _p(step), lr, beta1,
                                           beta2, eps, _stream(stream)))


class AdamGroups:
    """Host-side argument block of splat_adam_groups for fixed tensors."""

    def __init__(self, params, grads, m, v, lr):
        n = len(params)
        P = ctypes.c_void_p * n
        self.n = n
        self.params = P(*(_p(t) for t in params))
        self.grads = P(*(_p(t) for t in grads))
        self.m = P(*(_p(t) for t in m))
        self.v = P(*(_p(t) for t in v))
        self.sizes = (ctypes.c_int64 * n)(*(t.numel() for t in params))
        self.lr = (ctypes.c_float * n)(*lr)


def splat_adam_groups(groups: AdamGroups, step, beta1=0.9, beta2=0.999, eps=1e-15, zero_grad=True, stream=None):
    """One Adam step over all groups (`step`: device int32[1] holding t >= 1)."""
    _check("splat_adam_groups", load().splat_adam_groups(
        groups.n, groups.params, groups.grads, groups.m, groups.v, groups.sizes, groups.lr, _p(step), beta1, beta2,
        eps, 1 if zero_grad else 0, _stream(stream)))


def splat_pose_step(w2c, d_pose, m, v, step, lr_t, lr_r, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """`step`: device int32[1] tensor holding the Adam step t >= 1."""
    _check("splat_pose_step", load().splat_pose_step(_p(w2c), _p(d_pose), _p(m), _p(v), _p(step), lr_t, lr_r,
                                                     beta1, beta2, eps, _stream(stream)))


def splat_assoc_workspace_size(npix) -> int:
    return int(load().splat_assoc_workspace_size(npix))


def splat_assoc(id_a, t_a, id_b, t_b, n_a, n_b, t_max, pairs, counts, capacity, m_dev, status, ws, stream=None):
    _check("splat_assoc", load().splat_assoc(
        _p(id_a), _p(t_a), _p(id_b), _p(t_b), id_a.numel(), n_a, n_b, t_max, _p(pairs), _p(counts), capacity,
        _p(m_dev), _p(status), _p(ws), ws.numel() * ws.element_size(), _stream(stream)))


def splat_pose_compose(a, b, out, stream=None):
    """out[k] = a[k] @ b for a [n,4,4], b [4,4] (device float32)."""
    _check("splat_pose_compose", load().splat_pose_compose(a.shape[0], _p(a), _p(b), _p(out), _stream(stream)))


def splat_pose_rel_grad(w2c, d_cam, d_rel, stream=None):
    """d_rel = sum_k Ad(w2c[k])^T d_cam[k]."""
    _check("splat_pose_rel_grad", load().splat_pose_rel_grad(w2c.shape[0], _p(w2c), _p(d_cam), _p(d_rel),
                                                             _stream(stream)))


def splat_loss_consensus_workspace_size(height, width) -> int:
    return int(load().splat_loss_consensus_workspace_size(height, width))


def splat_loss_consensus(rgb, depth, target_rgb, target_depth, w_l1, w_ssim, w_geom, d_rgb, d_depth, loss, ws,
                         stream=None):
    """`loss`: device float32[2] (loss, SSIM), added to."""
    H, W = depth.shape
    _check("splat_loss_consensus", load().splat_loss_consensus(
        _p(rgb), _p(depth), _p(target_rgb), _p(target_depth), H, W, w_l1, w_ssim, w_geom, _p(d_rgb), _p(d_depth),
        _p(loss), _p(ws), ws.numel() * ws.element_size(), _stream(stream)))


def splat_mahalanobis_system(map_a: CGaussians, map_b: CGaussians, pairs, weights, m_dev, T, sys, max_dist=0.0,
                             stream=None):
    """`pairs`: device int32[capacity, 2]; `sys`: device float64[28], added to."""
    _check("splat_mahalanobis_system", load().splat_mahalanobis_system(
        ctypes.byref(map_a), ctypes.byref(map_b), _p(pairs), _p(weights), _p(m_dev), pairs.shape[0], _p(T),
        max_dist, _p(sys), _stream(stream)))


def splat_mahalanobis_step(sys, T, delta, status, stream=None):
    _check("splat_mahalanobis_step", load().splat_mahalanobis_step(_p(sys), _p(T), _p(delta), _p(status),
                                                                    _stream(stream)))


def splat_mahalanobis_system_step(map_a: CGaussians, map_b: CGaussians, pairs, weights, m_dev, T, sys, delta, status,
                                  max_dist=0.0, stream=None):
    """`sys`: device float64[32], zero before the first call and left zero by
    every call; T updated in place."""
    _check("splat_mahalanobis_system_step", load().splat_mahalanobis_system_step(
        ctypes.byref(map_a), ctypes.byref(map_b), _p(pairs), _p(weights), _p(m_dev), pairs.shape[0], _p(T),
        max_dist, _p(sys), _p(delta), _p(status), _stream(stream)))


def splat_prune_workspace_size(n) -> int:
    return int(load().splat_prune_workspace_size(n))


def splat_prune(g: CGaussians, tau_o, tau_s, tau_e, columns, mask, n_keep_dev, ws, stream=None):
    """`columns`: list of (src, dst) float32 device tensors of shape [n, width]
    (or [n])."""
    cols = (CColumn * max(1, len(columns)))()
    for i, (src, dst) in enumerate(columns):
        width = 1 if src.dim() == 1 else src.shape[1]
        cols[i] = CColumn(_p(src), _p(dst), width)
    _check("splat_prune", load().splat_prune(
        ctypes.byref(g), tau_o, tau_s, tau_e, cols, len(columns), _p(mask), _p(n_keep_dev), _p(ws),
        ws.numel() * ws.element_size(), _stream(stream)))


def splat_exp_f32(x, y, stream=None):
    _check("splat_exp_f32", load().splat_exp_f32(_p(x), _p(y), x.numel(), _stream(stream)))
