"""Differentiable RGB-D Gaussian rasterizer on the C ABI (torch tensors in,
torch tensors out) and its torch.autograd.Function.

The pipeline per view is splat_project -> splat_bin_sort -> splat_render_fwd
and, for gradients, splat_render_bwd (screen-space adjoint + projection
adjoint + pose gradient).  Buffers are owned by a `FrameBuffers` object and
reused across calls; the duplicate capacity grows when the device reports an
overflow (one host read of the duplicate count per forward in this eager
path; the batched / graph path keeps fixed capacities instead).
"""
from __future__ import annotations

import torch

from . import binding as B
from .scenes import Camera

PARAM_NAMES = ("mean", "log_scale", "quat", "opacity_logit", "rgb")


def _f32(x, device):
    return torch.as_tensor(x, dtype=torch.float32, device=device).contiguous()


class FrameBuffers:
    """Device buffers of one view: projection, sorted lists, image, workspaces."""

    def __init__(self, n: int, cam: Camera, device, capacity: int | None = None, want_keys: bool = False,
                 want_used: bool = False, status=None):
        """`status`: a device int32[1] to use as the sticky capacity status
        (kept by an owner that outlives the buffers), or None for a new one."""
        self.n, self.cam, self.device = n, cam, device
        H, W = cam.height, cam.width
        f, i = dict(dtype=torch.float32, device=device), dict(dtype=torch.int32, device=device)
        self.proj = dict(xyzo=torch.zeros(n, 4, **f), conic=torch.zeros(n, 4, **f), radius=torch.zeros(n, **i),
                         rect=torch.zeros(n, 4, **i), tiles_touched=torch.zeros(n, **i))
        self.image = dict(rgb=torch.zeros(H, W, 3, **f), depth=torch.zeros(H, W, **f), sil=torch.zeros(H, W, **f),
                          t_final=torch.zeros(H, W, **f), n_contrib=torch.zeros(H, W, **i),
                          max_id=torch.zeros(H, W, **i))
        if want_used:
            self.image["n_used"] = torch.zeros(H, W, **i)
        self.ranges = torch.zeros(cam.n_tiles, 2, dtype=torch.int32, device=device)
        # the tile schedule: per-tile costs (written by the forward) and the order built from them
        self.schedule = torch.zeros(B.splat_tile_schedule_size(cam.n_tiles) // 4, dtype=torch.int32, device=device)
        self.k_dev = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device) if status is None else status
        self.want_keys = want_keys
        self.capacity = 0
        self._alloc(capacity if capacity else max(1024, 16 * n))
        # the backward's workspace, large enough for the one-launch forward + backward too
        self.bwd_ws = torch.empty(max(1, B.splat_render_bwd_workspace_size(n),
                                      B.splat_render_fwd_bwd_workspace_size(n, cam.n_tiles)),
                                  dtype=torch.uint8, device=device)
        self.cproj = B.projected_struct(self.proj)
        self.cimg = B.image_struct(self.image)
        self.ccam = B.camera_struct(cam)

    def _alloc(self, capacity: int):
        capacity = int(min(capacity, 0x7FFFFFFF))
        self.capacity = capacity
        self.vals = torch.zeros(capacity, dtype=torch.int32, device=self.device)
        self.keys = torch.zeros(capacity, dtype=torch.int64, device=self.device) if self.want_keys else None
        nbytes = B.splat_bin_sort_workspace_size(self.n, capacity, self.cam.n_tiles)
        self.bin_ws = torch.empty(max(1, nbytes), dtype=torch.uint8, device=self.device)

    def ensure_capacity(self, k: int):
        if k > self.capacity:
            self._alloc(int(k * 1.25) + 1024)


def project(g: B.CGaussians, w2c, fb: FrameBuffers, stream=None):
    B.splat_project(g, fb.ccam, w2c, fb.cproj, stream)


def bin_sort(fb: FrameBuffers, stream=None, sync_check: bool = True, order: bool = True):
    """Bin and sort.  With `sync_check`, clear the status, read K back and
    retry on overflow; without it the call stays asynchronous and the sticky
    status word reports an overflow later.  With `order`, the tile schedule's
    order is rebuilt here (else the caller builds it elsewhere)."""
    sched = fb.schedule if order else None
    if sync_check:
        fb.status.zero_()
    B.splat_bin_sort(fb.cproj, fb.n, fb.ccam, fb.keys, fb.vals, fb.capacity, fb.k_dev, fb.ranges, fb.status,
                     fb.bin_ws, stream, schedule=sched)
    if sync_check:
        k = int(fb.k_dev.item())
        if k > fb.capacity:
            fb.ensure_capacity(k)
            fb.status.zero_()
            B.splat_bin_sort(fb.cproj, fb.n, fb.ccam, fb.keys, fb.vals, fb.capacity, fb.k_dev, fb.ranges, fb.status,
                             fb.bin_ws, stream, schedule=sched)
        return k
    return None


def render_forward(params, w2c, cam: Camera, bg=(0.0, 0.0, 0.0), fb: FrameBuffers | None = None, stream=None):
    """Render colour, depth, silhouette, final transmittance, contributor count
    and maximum-weight id of one view.  `params` = (mean, log_scale, quat,
    opacity_logit, rgb) CUDA float32 tensors."""
    mean = params[0]
    n = mean.shape[0]
    if fb is None:
        fb = FrameBuffers(n, cam, mean.device)
    g = B.gaussians_struct(*params)
    project(g, w2c, fb, stream)
    bin_sort(fb, stream)
    B.splat_render_fwd_l1(fb.cproj, params[4], n, fb.vals, fb.ranges, fb.ccam, bg, fb.cimg, None, stream,
                          schedule=fb.schedule)
    return fb


class SplatRender(torch.autograd.Function):
    """Differentiable render of one view.

    Inputs: mean [N,3], log_scale [N,3], quat [N,4], opacity_logit [N],
    rgb [N,3], delta [6] (tangent of the left perturbation exp(delta^) w2c,
    gradients are exact at delta = 0; pass zeros and retract outside), then
    the non-differentiable w2c [4,4], camera, background.
    Outputs: rgb [H,W,3], depth [H,W], silhouette [H,W], t_final [H,W],
    max_id [H,W] (int32).  The gradient of t_final is folded into that of the
    silhouette (T_final = 1 - S).
    """

    @staticmethod
    def forward(ctx, mean, log_scale, quat, opacity_logit, rgb, delta, w2c, cam, bg):
        params = tuple(t.detach().contiguous() for t in (mean, log_scale, quat, opacity_logit, rgb))
        w = w2c.detach().contiguous()
        fb = render_forward(params, w, cam, bg)
        img = fb.image
        ctx.fb, ctx.cam, ctx.bg = fb, cam, bg
        ctx.save_for_backward(*params, w)
        ctx.mark_non_differentiable(img["t_final"], img["max_id"])
        return (img["rgb"].clone(), img["depth"].clone(), img["sil"].clone(), img["t_final"].clone(),
                img["max_id"].clone())

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_sil, g_tfinal, g_id):
        mean, log_scale, quat, opacity_logit, rgb, w = ctx.saved_tensors
        fb = ctx.fb
        dev = mean.device
        g_rgb = torch.zeros_like(fb.image["rgb"]) if g_rgb is None else g_rgb.contiguous()
        g_depth = None if g_depth is None else g_depth.contiguous()
        if g_tfinal is not None:
            g_sil = (-g_tfinal if g_sil is None else g_sil - g_tfinal)
        g_sil = None if g_sil is None else g_sil.contiguous()
        grads = [torch.zeros_like(t) for t in (mean, log_scale, quat, opacity_logit, rgb)]
        d_pose = torch.zeros(6, dtype=torch.float32, device=dev)
        cg = B.gaussians_struct(mean, log_scale, quat, opacity_logit, rgb)
        cgr = B.CGaussiansGrad(*(B._p(t) for t in grads))
        B.splat_render_bwd(cg, fb.cproj, fb.ccam, w, fb.vals, fb.ranges, fb.cimg, ctx.bg, g_rgb, g_depth, g_sil, cgr,
                           d_pose, None, fb.bwd_ws, schedule=fb.schedule)
        return (*grads, d_pose, None, None, None)


def render(mean, log_scale, quat, opacity_logit, rgb, w2c, cam: Camera, bg=(0.0, 0.0, 0.0), delta=None):
    """Differentiable render (see SplatRender)."""
    if delta is None:
        delta = torch.zeros(6, dtype=torch.float32, device=mean.device)
    return SplatRender.apply(mean, log_scale, quat, opacity_logit, rgb, delta, w2c, cam, tuple(bg))
