"""Inter-agent association and alignment (Sec. 3.5 steps 2-4).

Agent B's map is brought into agent A's frame by a relative transform T_rel
(B world -> A world).  B is rendered from A's keyframe poses w2c_k composed
with T_rel, w2c_eff = w2c_k T_rel, all views forward and backward in one
persistent launch each.

* Association (step 2): the per-pixel maximum-weight Gaussians of A's and B's
  renders of each keyframe are paired (`associate`).
* Alignment (step 3): Gauss-Newton on the Mahalanobis objective over the
  associated pairs of all keyframes, T_rel <- exp(delta^) T_rel
  (`mahalanobis`).
* Optimisation (step 4): the loss of Eq. (optim) (L1 colour, SSIM and L1
  depth with the paper's weights 0.8 / 0.2 / 0.1) between B's and A's renders
  is differentiated to every view's camera pose; since
  w2c_k exp(d^) T_rel = exp((Ad_{w2c_k} d)^) w2c_k T_rel, the gradient with
  respect to T_rel is sum_k Ad(w2c_k)^T d_cam_k, and an Adam step with the
  retraction T_rel <- exp(delta^) T_rel follows (`step`).
"""
from __future__ import annotations

import torch

from . import binding as B
from .rasterizer import FrameBuffers, bin_sort, project
from .scenes import Camera


class Alignment:
    def __init__(self, map_b, keyframes, targets, cam: Camera, T_rel0, device, loss="paper",
                 weights=(0.8, 0.2, 0.1), lr=(1e-3, 4e-4), shape=(256, 4, 64, 8), capacity=None, want_keys=False,
                 map_a=None):
        """map_b: Scene of B's map (B's world); keyframes: list of A's w2c
        (4x4); targets: list of dicts with A's renders ("rgb", "depth",
        "max_id", "t_final") of the keyframes (device tensors); loss: "paper"
        (Eq. (optim) with `weights` = (L1, SSIM, geometry)) or "l1" (L1 colour
        and depth with weights[0], weights[2]); map_a: A's map (Scene or
        device tensors), needed by `mahalanobis`."""
        n_views = len(keyframes)
        if not 1 <= n_views <= B.SPLAT_MAX_VIEWS:
            raise ValueError(f"1..{B.SPLAT_MAX_VIEWS} keyframes")
        self.device = device
        self.cam = cam
        self.params = [torch.as_tensor(a, dtype=torch.float32, device=device).contiguous() for a in map_b.arrays()]
        self.n = self.params[0].shape[0]
        self.grads = [torch.zeros_like(p) for p in self.params]  # map gradients (accumulated, not applied)
        self.cg = B.gaussians_struct(*self.params)
        self.cgr = B.CGaussiansGrad(*(B._p(t) for t in self.grads))
        self.w2c_a = torch.as_tensor([list(k.reshape(-1)) for k in keyframes], dtype=torch.float32,
                                     device=device).reshape(n_views, 4, 4).contiguous()
        self.w2c_eff = torch.zeros_like(self.w2c_a)
        self.T = torch.as_tensor(T_rel0, dtype=torch.float32, device=device).contiguous().clone()
        self.d_cam = torch.zeros(n_views, 6, dtype=torch.float32, device=device)
        self.d_rel = torch.zeros(6, dtype=torch.float32, device=device)
        self.m6 = torch.zeros(6, dtype=torch.float32, device=device)
        self.v6 = torch.zeros(6, dtype=torch.float32, device=device)
        self.t_dev = torch.zeros(1, dtype=torch.int32, device=device)
        self.loss = torch.zeros(2, dtype=torch.float32, device=device)  # loss, SSIM
        self.lr = lr
        if loss not in ("paper", "l1"):
            raise ValueError("loss must be 'paper' or 'l1'")
        self.loss_kind = loss
        self.w = tuple(weights)
        self.loss_ws = torch.empty(max(16, B.splat_loss_consensus_workspace_size(cam.height, cam.width)),
                                   dtype=torch.uint8, device=device)
        self.map_a = None
        if map_a is not None:
            arrs = map_a.arrays() if hasattr(map_a, "arrays") else map_a
            self.map_a = [torch.as_tensor(a, dtype=torch.float32, device=device).contiguous() for a in arrs]
            self.cga = B.gaussians_struct(*self.map_a)
        self.sys = torch.zeros(32, dtype=torch.float64, device=device)  # 28 sums + a counter, left zero by every solve
        self.delta = torch.zeros(6, dtype=torch.float64, device=device)
        self.maha_status = torch.zeros(1, dtype=torch.int32, device=device)
        self.targets = targets
        self.fbs = [FrameBuffers(self.n, cam, device, capacity=capacity, want_keys=want_keys) for _ in range(n_views)]
        H, W = cam.height, cam.width
        self.g_rgb = [torch.zeros(H, W, 3, device=device) for _ in range(n_views)]
        self.g_depth = [torch.zeros(H, W, device=device) for _ in range(n_views)]
        self.views = (B.CView * n_views)()
        for k, fb in enumerate(self.fbs):
            self._fill_view(k)
        self.shape = B.CBatchShape(*shape)
        self.ws = torch.zeros(max(256, B.splat_batch_workspace_size()), dtype=torch.uint8, device=device)
        npix = cam.npix
        self.pairs = torch.zeros(npix, 2, dtype=torch.int32, device=device)
        self.counts = torch.zeros(npix, dtype=torch.int32, device=device)
        self.m_dev = torch.zeros(1, dtype=torch.int64, device=device)
        self.assoc_status = torch.zeros(1, dtype=torch.int32, device=device)
        self.assoc_ws = torch.empty(B.splat_assoc_workspace_size(npix), dtype=torch.uint8, device=device)
        self.graph = None
        self.steps_done = 0

    def _fill_view(self, k):
        fb = self.fbs[k]
        v = self.views[k]
        v.proj = fb.cproj
        v.rgb = B._p(self.params[4])
        v.n = self.n
        v.vals = B._p(fb.vals)
        v.ranges = B._p(fb.ranges)
        v.cam = fb.ccam
        v.bg[0] = v.bg[1] = v.bg[2] = 0.0
        v.image = fb.cimg
        v.d_rgb = B._p(self.g_rgb[k])
        v.d_depth = B._p(self.g_depth[k])
        v.d_sil = None
        v.grad2d = B._p(fb.bwd_ws)
        v.schedule = B._p(fb.schedule)

    def size_capacity(self, headroom=1.5):
        """One host read per view to size the duplicate buffers."""
        B.splat_pose_compose(self.w2c_a, self.T, self.w2c_eff)
        for k, fb in enumerate(self.fbs):
            project(self.cg, self.w2c_eff[k], fb)
            kdup = bin_sort(fb, sync_check=True)
            if kdup * headroom > fb.capacity:
                fb._alloc(int(kdup * headroom) + 1024)
                self._fill_view(k)

    def render(self, s=None):
        """Render B's map from every keyframe through the current T_rel."""
        s = torch.cuda.current_stream() if s is None else s
        B.splat_pose_compose(self.w2c_a, self.T, self.w2c_eff, s)
        for k, fb in enumerate(self.fbs):
            project(self.cg, self.w2c_eff[k], fb, s)
            bin_sort(fb, s, sync_check=False)
        B.splat_render_fwd_batch(self.views, self.shape, self.ws, s)

    def step(self, s=None):
        """One alignment iteration: render all views, loss, backward to T_rel,
        Adam + retraction of T_rel."""
        s = torch.cuda.current_stream() if s is None else s
        self.render(s)
        with torch.cuda.stream(s):
            self.loss.zero_()
            self.d_cam.zero_()
            for g in self.grads:
                g.zero_()
        for k, fb in enumerate(self.fbs):
            t = self.targets[k]
            if self.loss_kind == "paper":
                B.splat_loss_consensus(fb.image["rgb"], fb.image["depth"], t["rgb"], t["depth"], self.w[0], self.w[1],
                                       self.w[2], self.g_rgb[k], self.g_depth[k], self.loss, self.loss_ws, s)
            else:
                B.splat_loss_l1(fb.image["rgb"], fb.image["depth"], t["rgb"], t["depth"], self.w[0], self.w[2],
                                self.g_rgb[k], self.g_depth[k], self.loss, s)
        B.splat_render_bwd_batch(self.views, self.shape, self.ws, s)
        for k, fb in enumerate(self.fbs):
            B.splat_project_bwd(self.cg, fb.cproj, fb.ccam, self.w2c_eff[k], fb.bwd_ws, self.cgr, self.d_cam[k],
                                None, s)
        B.splat_pose_rel_grad(self.w2c_a, self.d_cam, self.d_rel, s)
        with torch.cuda.stream(s):
            self.t_dev.add_(1)
        B.splat_pose_step(self.T, self.d_rel, self.m6, self.v6, self.t_dev, self.lr[0], self.lr[1], stream=s)

    def capture(self):
        """Capture one alignment step into a CUDA graph (after a warm-up step
        on a side stream); returns the number of library launches per step."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        snap = [self.T.clone(), self.m6.clone(), self.v6.clone(), self.t_dev.clone()]
        with torch.cuda.stream(s):
            self.step(s)
        torch.cuda.current_stream().wait_stream(s)
        for dst, src in zip((self.T, self.m6, self.v6, self.t_dev), snap):
            dst.copy_(src)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        n0 = B.splat_kernel_launches()
        with torch.cuda.graph(g):
            self.step()
        self.launches_per_step = B.splat_kernel_launches() - n0
        self.graph = g
        return self.launches_per_step

    def replay(self):
        self.graph.replay()
        self.steps_done += 1

    def reset(self, T_rel0):
        """Restart the optimisation from T_rel0."""
        self.T.copy_(torch.as_tensor(T_rel0, dtype=torch.float32))
        self.maha_status.zero_()
        self.m6.zero_()
        self.v6.zero_()
        self.t_dev.zero_()

    def error(self, T_true):
        """(translation metres, rotation degrees) of T_rel T_true^-1."""
        return pose_error(self.T.double().cpu().numpy(), T_true)

    def mahalanobis(self, iters=3, views=None, t_max=0.5, weighted=True, max_dist=0.02, s=None):
        """Gauss-Newton iterations of the Mahalanobis alignment over the pairs
        associated in every keyframe (re-rendered and re-associated at each
        iteration).  Pairs are weighted by their pixel counts unless
        `weighted` is False; pairs farther apart than `max_dist` (the G-ICP
        correspondence distance of Sec. 4.1) are left out."""
        if self.map_a is None:
            raise ValueError("the Mahalanobis alignment needs map_a")
        s = torch.cuda.current_stream() if s is None else s
        views = range(len(self.fbs)) if views is None else views
        views = list(views)
        for _ in range(iters):
            self.render(s)
            for i, k in enumerate(views):
                self.associate(k, t_max, s)
                w = self.counts if weighted else None
                if i + 1 < len(views):  # accumulate; the last view's call also solves, steps and clears sys
                    B.splat_mahalanobis_system(self.cga, self.cg, self.pairs, w, self.m_dev, self.T, self.sys,
                                               max_dist, s)
                else:
                    B.splat_mahalanobis_system_step(self.cga, self.cg, self.pairs, w, self.m_dev, self.T, self.sys,
                                                    self.delta, self.maha_status, max_dist, s)

    def associate(self, k, t_max=0.5, s=None):
        """Distinct (A id, B id) pairs of keyframe k with pixel counts (device
        tensors; M in m_dev)."""
        s = torch.cuda.current_stream() if s is None else s
        fb = self.fbs[k]
        t = self.targets[k]
        with torch.cuda.stream(s):
            self.assoc_status.zero_()
        B.splat_assoc(t["max_id"], t["t_final"], fb.image["max_id"], fb.image["t_final"], t.get("n_a", self.n),
                      self.n, t_max, self.pairs, self.counts, self.pairs.shape[0], self.m_dev, self.assoc_status,
                      self.assoc_ws, s)

    def status(self) -> int:
        st = int(self.assoc_status.item()) | int(self.maha_status.item())
        for fb in self.fbs:
            st |= int(fb.status.item())
        return st


def pose_error(T, T_true):
    """(translation metres, rotation degrees) of T T_true^-1."""
    import math

    import numpy as np

    E = np.asarray(T, np.float64) @ np.linalg.inv(np.asarray(T_true, np.float64))
    c = float(np.clip((np.trace(E[:3, :3]) - 1.0) / 2.0, -1.0, 1.0))
    return float(np.linalg.norm(E[:3, 3])), math.degrees(math.acos(c))


def render_targets(map_a, keyframes, cam: Camera, device, bg=(0.0, 0.0, 0.0)):
    """Agent A's own renders of its keyframes (the alignment targets):
    list of dicts of device tensors rgb, depth, max_id, t_final and n_a."""
    from .rasterizer import render_forward

    params = [torch.as_tensor(a, dtype=torch.float32, device=device).contiguous() for a in map_a.arrays()]
    fb = FrameBuffers(params[0].shape[0], cam, device)
    out = []
    for w2c in keyframes:
        render_forward(params, torch.as_tensor(w2c, dtype=torch.float32, device=device).contiguous(), cam, bg, fb)
        out.append(dict(rgb=fb.image["rgb"].clone(), depth=fb.image["depth"].clone(),
                        max_id=fb.image["max_id"].clone(), t_final=fb.image["t_final"].clone(), n_a=fb.n))
    return out
