"""One agent's resident state and its tracking + mapping step.

An agent keeps its Gaussian map, the map's Adam moments, its camera pose
(world-to-camera, device float[16]) with the pose's Adam moments, the current
RGB-D observation and every work buffer on the device.  One step is the whole
hot path of the method for one frame:

  splat_project -> splat_bin_sort -> splat_render_fwd      (render, Sec. 3.3)
     with the L1 terms of Eq. optim (L1 colour + w_depth L1 depth) and their
     image gradients taken in the same pass, and the screen-space adjoint of
     the render in the same launch (splat_render_fwd_bwd; or two launches:
     splat_render_fwd_l1, splat_render_bwd)
  -> splat_project_bwd_adam (projection adjoint to every Gaussian parameter
     and the pose, with the map's Adam step in the same launch: mapping,
     Sec. 3.4 step 4; tracking-only steps use splat_project_bwd)
  -> splat_pose_step (render-driven tracking)
  -> splat_assoc of the rendered maximum-weight ids against the observation's
     ids (render-based association, Sec. 3.5 step 2).

`step()` issues only stream-ordered launches (no host synchronisation unless
asked for), so it can run back to back, be timed with events, or be captured.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import binding as B
from .rasterizer import FrameBuffers, bin_sort, project
from .scenes import Camera

# SplaTAM-style learning rates (the optimiser the paper follows, Sec. 3.4).
DEFAULT_LR = dict(mean=1e-4, log_scale=1e-3, quat=1e-3, opacity_logit=5e-2, rgb=2.5e-3)
DEFAULT_POSE_LR = (2e-3, 4e-4)  # translation, rotation


@dataclasses.dataclass
class StepConfig:
    w_rgb: float = 1.0
    w_depth: float = 0.5
    lr: dict = dataclasses.field(default_factory=lambda: dict(DEFAULT_LR))
    pose_lr: tuple = DEFAULT_POSE_LR
    track: bool = True
    map: bool = True
    assoc: bool = True
    t_max: float = 0.5
    bg: tuple = (0.0, 0.0, 0.0)
    # where the culled Gaussians' zero-gradient Adam step runs: inside the
    # fused projection adjoint's launch ("adjoint"), or on the side stream
    # beside the forward render ("forward": it needs only the projection's
    # radii and fills the render's tail) or beside the backward ("backward")
    culled_at: str = "adjoint"
    # the forward render and the screen-space backward in one launch
    # (splat_render_fwd_bwd), else two (splat_render_fwd_l1, splat_render_bwd).
    # One launch takes as long as the two at 300k / 640x480, and the
    # association then waits for both renders instead of overlapping the
    # backward, so two launches are the default.
    fused: bool = False
    # with mapping and tracking on, the pose's Adam step taken by the last CTA
    # of the fused projection adjoint + Adam launch, else its own one-warp
    # launch after it; the launch of its own is the faster step (0.257 vs
    # 0.261 ms at 300k / 640x480, measured), so it is the default
    pose_in_adjoint: bool = False
    # keep per-parameter gradient arrays, filled by steps without mapping;
    # without them such a step forms the pose gradient alone (a mapping step
    # never needs them: its Adam step is fused into the projection adjoint)
    grads: bool = True


class Agent:
    """Resident map + optimiser state + buffers of one agent."""

    def __init__(self, scene, w2c, cam: Camera, device, cfg: StepConfig | None = None, capacity: int | None = None,
                 want_used: bool = False, state=None, side=None):
        """`scene`: the map (numpy arrays, copied in synchronously), or None
        with `state`: the pinned host tensors of a swapped-out agent's
        _state() (map, moments, pose, pose moments, step, seen bitmap), copied in
        asynchronously on the current stream, like every allocation and fill
        here, so that a swap-in needs no host synchronisation.  `side`: a
        stream to reuse for the side work (a new one by default)."""
        self.cfg = cfg or StepConfig()
        self.cam = cam
        self.device = device
        if state is not None:
            def dev(t):
                d = torch.empty(t.shape, dtype=t.dtype, device=device)
                d.copy_(t, non_blocking=True)
                return d
            self.params = [dev(t) for t in state[:5]]
            self.m = [dev(t) for t in state[5:10]]
            self.v = [dev(t) for t in state[10:15]]
            self.w2c = dev(state[15])
        else:
            self.params = [torch.as_tensor(a, dtype=torch.float32, device=device).contiguous() for a in scene.arrays()]
            self.m = [torch.zeros_like(p) for p in self.params]
            self.v = [torch.zeros_like(p) for p in self.params]
            self.w2c = torch.as_tensor(w2c, dtype=torch.float32, device=device).contiguous().clone()
        self.n = self.params[0].shape[0]
        # per-step accumulators in one block, cleared by one launch: d_pose [6], loss [1], association status [1]
        self._acc = torch.zeros(8, dtype=torch.float32, device=device)
        self.d_pose = self._acc[0:6]
        self.loss = self._acc[6:7]
        self.assoc_status = self._acc[7:8].view(torch.int32)
        self.pose_m = torch.zeros(6, dtype=torch.float32, device=device)
        self.pose_v = torch.zeros(6, dtype=torch.float32, device=device)
        self.t_dev = torch.zeros(1, dtype=torch.int32, device=device)  # Adam step, advanced on the device
        self.bin_status = torch.zeros(1, dtype=torch.int32, device=device)  # sticky capacity status of the binning
        self._pose_counter = torch.zeros(1, dtype=torch.int32, device=device)  # last-CTA ticket of the pose step
        # bit i: Gaussian i's moments may be nonzero (a clear bit promises zero
        # moments, so the map's Adam step skips the Gaussian while it is culled)
        if state is not None:
            self.seen = dev(state[19])
        else:
            self.seen = torch.zeros((self.n + 31) // 32, dtype=torch.int32, device=device)
        if state is not None:
            for dst, src in zip((self.pose_m, self.pose_v, self.t_dev), state[16:19]):
                dst.copy_(src, non_blocking=True)
        self.side = side if side is not None else torch.cuda.Stream(device=device)  # association, beside the backward
        self.host_in = None  # pinned (rgb, depth) the step copies its observation from, or None
        self.host_out = None  # pinned (loss, w2c) the step writes its results to, or None
        self.cg = B.gaussians_struct(*self.params)
        self.steps_done = 0
        self.graph = None
        self.want_used = want_used
        self._make_adam()
        self.make_scratch(capacity)

    # -- per-step buffers ---------------------------------------------------------
    SCRATCH = ("grads", "cgr", "fb", "obs_rgb", "obs_depth", "obs_id", "obs_tfinal", "g_rgb", "g_depth", "pairs",
               "counts", "m_dev", "assoc_ws", "cl1")

    def make_scratch(self, capacity: int | None = None):
        """Allocate the per-step buffers: frame buffers (projection, sorted
        lists, image, workspaces), observation and image-gradient buffers,
        association buffers and, when kept, the gradient arrays.  Everything
        else (map, moments, pose, accumulators) is the agent's state.  The
        allocations and fills are stream-ordered on the current stream."""
        device, cam = self.device, self.cam
        self.grads = [torch.zeros_like(p) for p in self.params] if self.cfg.grads else None
        self.cgr = B.CGaussiansGrad(*(B._p(t) for t in self.grads)) if self.grads is not None else None
        self.grads_clean = True  # host-side: the gradient buffers hold zeros
        self.fb = FrameBuffers(self.n, cam, device, capacity=capacity, want_used=self.want_used, status=self.bin_status)
        H, W = cam.height, cam.width
        self.obs_rgb = torch.zeros(H, W, 3, dtype=torch.float32, device=device)
        self.obs_depth = torch.zeros(H, W, dtype=torch.float32, device=device)
        self.obs_id = torch.full((H, W), -1, dtype=torch.int32, device=device)
        self.obs_tfinal = torch.ones(H, W, dtype=torch.float32, device=device)
        self.g_rgb = torch.zeros(H, W, 3, dtype=torch.float32, device=device)
        self.g_depth = torch.zeros(H, W, dtype=torch.float32, device=device)
        npix = cam.npix
        self.assoc_cap = npix
        self.pairs = torch.zeros(npix, 2, dtype=torch.int32, device=device)
        self.counts = torch.zeros(npix, dtype=torch.int32, device=device)
        self.m_dev = torch.zeros(1, dtype=torch.int64, device=device)
        self.assoc_ws = torch.empty(max(1, B.splat_assoc_workspace_size(npix)), dtype=torch.uint8, device=device)
        self._make_l1()

    @property
    def has_scratch(self) -> bool:
        return self.fb is not None

    def release_scratch(self):
        """Drop the per-step buffers (the state stays) and any captured graph.
        Returns the dropped tensors: the caller keeps them alive until no
        launched work can still use them.  The duplicate capacity is kept for
        make_scratch."""
        held = [getattr(self, k) for k in self.SCRATCH]
        self.capacity = self.fb.capacity
        for k in self.SCRATCH:
            setattr(self, k, None)
        self.graph = None
        return held

    def state_tensors(self):
        """The device tensors of the agent's state (what stays resident
        without the per-step buffers)."""
        return [*self._state(), self._acc, self.bin_status]

    def scratch_tensors(self):
        out = []
        if self.grads is not None:
            out += self.grads
        for k in ("obs_rgb", "obs_depth", "obs_id", "obs_tfinal", "g_rgb", "g_depth", "pairs", "counts", "m_dev",
                  "assoc_ws"):
            out.append(getattr(self, k))
        fb = self.fb
        out += list(fb.proj.values()) + list(fb.image.values())
        out += [t for t in (fb.ranges, fb.schedule, fb.k_dev, fb.vals, fb.keys, fb.bin_ws, fb.bwd_ws)
                if t is not None]
        return out

    def _make_adam(self):
        names = ("mean", "log_scale", "quat", "opacity_logit", "rgb")
        self.lrs = [self.cfg.lr[k] for k in names]
        # the pose's Adam step, taken inside the fused projection adjoint + Adam launch
        self.cpose = B.CPoseAdam(B._p(self.w2c), B._p(self.pose_m), B._p(self.pose_v), B._p(self.t_dev),
                                 self.cfg.pose_lr[0], self.cfg.pose_lr[1], 0.9, 0.999, 1e-15, B._p(self._pose_counter))
        self.cm = B.CGaussiansGrad(*(B._p(t) for t in self.m))
        self.cv = B.CGaussiansGrad(*(B._p(t) for t in self.v))

    def _make_l1(self):
        """The L1 loss descriptor the forward render fills (observation as
        target, gradient images, loss accumulator)."""
        self.cl1 = B.l1_struct(self.obs_rgb, self.obs_depth, self.cfg.w_rgb, self.cfg.w_depth, self.g_rgb,
                               self.g_depth, self.loss)

    # -- observation ---------------------------------------------------------
    def set_observation(self, rgb, depth, ids=None, t_final=None, stream=None):
        """Copy an RGB-D frame (and optionally its id / transmittance images)
        into the resident observation buffers (stream-ordered)."""
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            self.obs_rgb.copy_(rgb, non_blocking=True)
            self.obs_depth.copy_(depth, non_blocking=True)
            if ids is not None:
                self.obs_id.copy_(ids, non_blocking=True)
            if t_final is not None:
                self.obs_tfinal.copy_(t_final, non_blocking=True)

    def attach_host_io(self, rgb=None, depth=None, loss=None, w2c=None):
        """Pinned host buffers that the step itself reads its observation from
        (rgb [H, W, 3], depth [H, W]) and writes its loss [1] and pose [4, 4]
        to, every step and also inside a captured graph: put the next frame in
        `rgb` / `depth` before a step, read `loss` / `w2c` after synchronising.
        The frame's copy runs on the side stream and overlaps the projection,
        binning; the forward render, which takes the loss, waits for it.  Calling it
        with no arguments detaches the buffers.  A graph captured before must
        be captured again."""
        H, W = self.cam.height, self.cam.width
        want = ((rgb, (H, W, 3)), (depth, (H, W)), (loss, (1,)), (w2c, (4, 4)))
        for t, shape in want:
            if t is None:
                continue
            if t.device.type != "cpu" or not t.is_pinned() or t.dtype != torch.float32 or tuple(t.shape) != shape:
                raise ValueError(f"host buffers must be pinned float32 CPU tensors of shape {shape}")
        if (rgb is None) != (depth is None) or (loss is None) != (w2c is None):
            raise ValueError("attach rgb with depth, and loss with w2c")
        self.host_in = (rgb, depth) if rgb is not None else None
        self.host_out = (loss, w2c) if loss is not None else None
        self.graph = None

    def render_observation_from(self, w2c_obs, stream=None):
        """Render the map from `w2c_obs` into the observation buffers (used to
        make synthetic targets)."""
        fb = FrameBuffers(self.n, self.cam, self.device, capacity=self.fb.capacity)
        B.splat_project(self.cg, fb.ccam, torch.as_tensor(w2c_obs, dtype=torch.float32, device=self.device), fb.cproj,
                        stream)
        bin_sort(fb, stream)
        B.splat_render_fwd(fb.cproj, self.params[4], self.n, fb.vals, fb.ranges, fb.ccam, self.cfg.bg, fb.cimg, stream)
        self.set_observation(fb.image["rgb"], fb.image["depth"], fb.image["max_id"], fb.image["t_final"], stream)
        return fb

    # -- the step ------------------------------------------------------------
    def size_capacity(self, headroom: float = 1.5, stream=None):
        """Project + count duplicates once (host read) and size the duplicate
        buffers with headroom, so that later steps need no host read."""
        project(self.cg, self.w2c, self.fb, stream)
        k = bin_sort(self.fb, stream, sync_check=True)
        if k * headroom > self.fb.capacity:
            self.fb._alloc(int(k * headroom) + 1024)
        return k

    def forward(self, stream=None, sync_check: bool = False):
        fb = self.fb
        project(self.cg, self.w2c, fb, stream)
        bin_sort(fb, stream, sync_check=sync_check)
        B.splat_render_fwd_l1(fb.cproj, self.params[4], self.n, fb.vals, fb.ranges, fb.ccam, self.cfg.bg, fb.cimg,
                              None, stream, schedule=fb.schedule)

    # The step in phases, so that a multi-agent batch can interleave them.
    def phase_clear(self, s):
        """Start a step: zero its accumulators (d_pose, loss, association
        status) and, when a previous step left them filled, the parameter
        gradients; advance the device Adam step count; build the tile
        schedule's order from the costs the previous forward wrote (off the
        projection and binning's stream: the binning then leaves it alone)."""
        with torch.cuda.stream(s):
            self._acc.zero_()
            self.t_dev.add_(1)
            if not self.grads_clean and self.grads is not None:  # the fused adjoint + Adam never fills them
                for g in self.grads:
                    g.zero_()
        B.splat_tile_schedule_order(self.fb.schedule, self.cam.n_tiles, s)
        self.grads_clean = True
        self.steps_done += 1

    def phase_pre(self, s, sync_check: bool = False):
        """Projection and binning (the schedule's order comes from phase_clear)."""
        project(self.cg, self.w2c, self.fb, s)
        bin_sort(self.fb, s, sync_check=sync_check, order=False)

    def phase_render(self, s):
        """Forward render with the L1 loss terms and their image gradients
        (needs phase_clear before it, and the observation in place)."""
        fb = self.fb
        B.splat_render_fwd_l1(fb.cproj, self.params[4], self.n, fb.vals, fb.ranges, fb.ccam, self.cfg.bg, fb.cimg,
                              self.cl1, s, schedule=fb.schedule)

    def phase_render_backward(self, s):
        """Forward render with the L1 terms and the screen-space adjoint in
        one launch (the gradients left in the backward workspace)."""
        fb = self.fb
        B.splat_render_fwd_bwd(fb.cproj, self.params[4], self.n, fb.vals, fb.ranges, fb.ccam, self.cfg.bg, fb.cimg,
                               self.cl1, fb.status, fb.bwd_ws, s, schedule=fb.schedule)

    def phase_loss(self, s):
        """Clear, then the L1 terms as a separate pass over a rendered image
        (the unfused form of phase_clear + the loss part of phase_render)."""
        cfg, fb = self.cfg, self.fb
        self.phase_clear(s)
        B.splat_loss_l1(fb.image["rgb"], fb.image["depth"], self.obs_rgb, self.obs_depth, cfg.w_rgb, cfg.w_depth,
                        self.g_rgb, self.g_depth, self.loss, s)

    def phase_backward(self, s):
        """Screen-space adjoint of the render (left in the backward workspace)."""
        fb = self.fb
        B.splat_render_bwd(self.cg, fb.cproj, fb.ccam, self.w2c, fb.vals, fb.ranges, fb.cimg, self.cfg.bg,
                           self.g_rgb, self.g_depth, None, None, None, None, fb.bwd_ws, s, schedule=fb.schedule)

    def phase_project_backward(self, s):
        """Projection adjoint of the screen-space gradients in the backward
        workspace: with mapping on, fused with the map's Adam step (the map
        moves, no gradient array is written); otherwise into the gradient
        arrays.  Either way the pose gradient goes to d_pose."""
        fb = self.fb
        if self.cfg.map:
            B.splat_project_bwd_adam(self.cg, fb.cproj, fb.ccam, self.w2c, fb.bwd_ws, self.cm, self.cv, self.lrs,
                                     self.t_dev, self.d_pose, stream=s, culled=self.cfg.culled_at == "adjoint",
                                     seen=self.seen, pose=self.cpose if self._pose_in_adjoint() else None)
        else:
            self.grads_clean = self.grads is None
            B.splat_project_bwd(self.cg, fb.cproj, fb.ccam, self.w2c, fb.bwd_ws, self.cgr, self.d_pose, None, s)

    def phase_adam_culled(self, s):
        """With mapping on and `culled_at` not "adjoint": the culled Gaussians'
        zero-gradient Adam step (needs only the projection's radii)."""
        if self.cfg.map and self.cfg.culled_at != "adjoint":
            B.splat_adam_culled(self.cg, self.fb.proj["radius"], self.cm, self.cv, self.lrs, self.t_dev, stream=s,
                                seen=self.seen)

    def _pose_in_adjoint(self) -> bool:
        return self.cfg.map and self.cfg.track and self.cfg.pose_in_adjoint

    def phase_update(self, s, assoc: bool = True, pose_stream=None):
        """The pose step (on `pose_stream` when given, after the projection
        adjoint on s), then the association when `assoc`.  The map's Adam
        step is part of phase_project_backward, and so is the pose step when
        mapping is on."""
        cfg = self.cfg
        if cfg.track and not self._pose_in_adjoint():
            ps = s
            if pose_stream is not None:
                pose_stream.wait_stream(s)
                ps = pose_stream
            B.splat_pose_step(self.w2c, self.d_pose, self.pose_m, self.pose_v, self.t_dev, cfg.pose_lr[0],
                              cfg.pose_lr[1], stream=ps)
        if assoc:
            self.phase_assoc(s)

    def phase_assoc(self, s):
        """Association of the rendered ids with the observation's (needs the
        forward render and the accumulators cleared in phase_clear)."""
        cfg, fb = self.cfg, self.fb
        if cfg.assoc:  # the status word was cleared with the other accumulators in phase_clear
            B.splat_assoc(fb.image["max_id"], fb.image["t_final"], self.obs_id, self.obs_tfinal, self.n, self.n,
                          cfg.t_max, self.pairs, self.counts, self.assoc_cap, self.m_dev, self.assoc_status,
                          self.assoc_ws, s)

    def step(self, stream=None, sync_check: bool = False):
        """One step.  The accumulators are cleared (and the frame copied in,
        with host buffers attached) on a side stream while the map is projected
        and binned; the forward render takes the loss, before the
        screen-space backward (or in the same launch: `fused`).  The
        association depends only on the forward render, so it runs on the side
        stream forked after it, overlapping the backward render (two launches)
        or the projection adjoint (one); the pose step follows it there, beside
        the map's Adam; the side stream is joined at the end."""
        s = torch.cuda.current_stream() if stream is None else stream
        self.side.wait_stream(s)
        self.phase_clear(self.side)
        if self.host_in is not None:
            with torch.cuda.stream(self.side):
                self.obs_rgb.copy_(self.host_in[0], non_blocking=True)
                self.obs_depth.copy_(self.host_in[1], non_blocking=True)
        self.phase_pre(s, sync_check)
        s.wait_stream(self.side)
        if self.cfg.culled_at == "forward":
            self.side.wait_stream(s)
            self.phase_adam_culled(self.side)  # beside the forward render
        if self.cfg.fused:  # the association follows the one render launch, beside the projection adjoint
            self.phase_render_backward(s)
            if self.cfg.assoc or self.cfg.culled_at == "backward":
                self.side.wait_stream(s)
                if self.cfg.culled_at == "backward":
                    self.phase_adam_culled(self.side)
                self.phase_assoc(self.side)
        else:
            self.phase_render(s)
            if self.cfg.assoc or self.cfg.culled_at == "backward":
                self.side.wait_stream(s)
                if self.cfg.culled_at == "backward":
                    self.phase_adam_culled(self.side)  # beside the backward render
                self.phase_assoc(self.side)
            self.phase_backward(s)
        self.phase_project_backward(s)
        self.phase_update(s, assoc=False, pose_stream=self.side)
        s.wait_stream(self.side)
        if self.host_out is not None:
            with torch.cuda.stream(s):
                self.host_out[0].copy_(self.loss, non_blocking=True)
                self.host_out[1].copy_(self.w2c, non_blocking=True)

    def view(self):
        """C descriptor of this agent's view for the batched render calls."""
        fb = self.fb
        v = B.CView()
        v.proj = fb.cproj
        v.rgb = B._p(self.params[4])
        v.n = self.n
        v.vals = B._p(fb.vals)
        v.ranges = B._p(fb.ranges)
        v.cam = fb.ccam
        v.bg[0], v.bg[1], v.bg[2] = self.cfg.bg
        v.image = fb.cimg
        v.d_rgb = B._p(self.g_rgb)
        v.d_depth = B._p(self.g_depth)
        v.d_sil = None
        v.grad2d = B._p(fb.bwd_ws)
        v.l1 = ctypes.pointer(self.cl1)
        v.schedule = B._p(fb.schedule)
        return v

    # -- pruning -----------------------------------------------------------------
    def prune(self, tau_o: float = 0.005, tau_s: float = 0.25, tau_e: float = 10.0, stream=None) -> int:
        """Gaussian splat pruning (Algorithm 1) of the resident map: Gaussians
        with opacity below tau_o, or (tau_s > 0) largest scale above tau_s or
        above tau_e times the sum of the other two, are removed from the map
        and from both Adam moments, keeping the order of the rest.  The map
        shrinks to the kept Gaussians (one host read of the count); gradient
        and frame buffers are re-made at the new size and a captured graph or
        snapshot is dropped.  Returns the number kept."""
        s = torch.cuda.current_stream() if stream is None else stream
        n = self.n
        ws = torch.empty(max(16, B.splat_prune_workspace_size(n)), dtype=torch.uint8, device=self.device)
        n_keep = torch.zeros(1, dtype=torch.int64, device=self.device)
        B.splat_prune(self.cg, tau_o, tau_s, tau_e, [], None, n_keep, ws, s)  # count only
        s.synchronize()
        k = int(n_keep.item())
        if k == n:
            return k
        src = [*self.params, *self.m, *self.v]
        dst = [torch.empty((k,) + tuple(t.shape[1:]), dtype=t.dtype, device=self.device) for t in src]
        B.splat_prune(self.cg, tau_o, tau_s, tau_e, list(zip(src, dst)), None, n_keep, ws, s)
        s.synchronize()
        self.params, self.m, self.v = dst[:5], dst[5:10], dst[10:]
        self.n = k
        self.seen = self._seen_from_moments()
        self.cg = B.gaussians_struct(*self.params)
        self.make_scratch(self.fb.capacity)
        self._make_adam()
        self.graph = None
        self._snap = None
        return k

    def _seen_from_moments(self):
        """The seen bitmap rebuilt from the moments: bit i set when any of
        Gaussian i's 28 moment elements is nonzero (host-side torch ops; used
        after the map is compacted)."""
        nz = torch.zeros(self.n, dtype=torch.bool, device=self.device)
        for t in (*self.m, *self.v):
            nz |= (t.reshape(self.n, -1) != 0).any(dim=1)
        words = (self.n + 31) // 32
        bits = torch.zeros(words * 32, dtype=torch.int64, device=self.device)
        bits[:self.n] = nz.to(torch.int64)
        w = (bits.view(words, 32) << torch.arange(32, device=self.device)).sum(dim=1)
        return torch.where(w >= 2 ** 31, w - 2 ** 32, w).to(torch.int32).contiguous()

    # -- episodes ---------------------------------------------------------------
    def _state(self):
        return [*self.params, *self.m, *self.v, self.w2c, self.pose_m, self.pose_v, self.t_dev, self.seen]

    def snapshot(self):
        """Keep a device copy of the map, optimiser state and pose."""
        self._snap = [t.clone() for t in self._state()]

    def restore(self, stream=None):
        """Return the map, optimiser state and pose to the last snapshot
        (device-to-device copies into the same buffers, so captured graphs
        stay valid)."""
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            for dst, src in zip(self._state(), self._snap):
                dst.copy_(src, non_blocking=True)

    # -- CUDA graph -------------------------------------------------------------
    def capture(self, keep_state: bool = False):
        """Capture one step into a CUDA graph.  All buffers are fixed (size the
        duplicate capacity first); replaying the graph performs exactly the
        kernels of `step()` with no host work.  The capture is preceded by one
        eager warm-up step; with `keep_state` the map, optimiser state and pose
        are put back after it, so that capturing changes nothing.  Returns the
        number of library kernel launches one replay performs."""
        saved = [t.clone() for t in self._state()] if keep_state else None
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # warm-up on the capture stream's side
            self.step(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        if saved is not None:
            for dst, src in zip(self._state(), saved):
                dst.copy_(src)
            torch.cuda.synchronize()
            del saved
            self.steps_done -= 1
            self.grads_clean = False  # the graph clears the gradients itself, whatever ran before it
        g = torch.cuda.CUDAGraph()
        n0 = B.splat_kernel_launches()
        with torch.cuda.graph(g):
            self.step()
        self.launches_per_step = B.splat_kernel_launches() - n0
        self.graph = g
        if keep_state:  # one replay (the first launch of a graph is the slow one), then the state put back
            saved = [t.clone() for t in self._state()]
            g.replay()
            torch.cuda.synchronize()
            for dst, src in zip(self._state(), saved):
                dst.copy_(src)
            torch.cuda.synchronize()
            del saved
        return self.launches_per_step

    def replay(self):
        self.graph.replay()
        self.steps_done += 1

    def status(self) -> int:
        """Sticky device status of the last steps (host read)."""
        return int(self.bin_status.item()) | int(self.assoc_status.item())
