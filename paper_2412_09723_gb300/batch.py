"""Several agents stepped together (batched differentiable rendering across
agents, Sec. 3.6 of the paper: intra-agent work is independent per agent).

One batched step:
  per agent, on its own stream:  accumulators cleared, projection, binning
  all agents, ONE persistent launch:  forward render with each agent's L1 loss
                                      terms (splat_render_fwd_batch)
  all agents, ONE persistent launch:  backward render  (splat_render_bwd_batch)
  per agent, on its own stream:  projection adjoint with the map's Adam step
  per agent, on a side stream forked after the forward:  association
  (overlapping the backward launch), then the pose step; joined at the end
The whole step is captured into one CUDA graph (the per-agent streams are
forked from and joined back into the capture stream), so a replay is a single
host call.  The persistent launches' execution shape (shared-memory batch of
Gaussians and CTAs per SM) is chosen by `autotune`, which times graph replays
of each candidate on the actual agents and caches the winner.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import binding as B


def shape_of(t):
    return B.CBatchShape(*t)


DEFAULT_SHAPE = (256, 4, 64, 8)
CANDIDATES = [(fb, fc, bb, bc) for fb in (128, 256) for fc in (4, 8) for bb in (64, 128) for bc in (6, 8, 10)]


class MultiAgentBatch:
    def __init__(self, agents, shape=DEFAULT_SHAPE):
        if not 1 <= len(agents) <= B.SPLAT_MAX_VIEWS:
            raise ValueError(f"1..{B.SPLAT_MAX_VIEWS} agents per batch")
        self.agents = agents
        self.device = agents[0].device
        self.views = (B.CView * len(agents))(*[a.view() for a in agents])
        self.shape_t = tuple(shape)
        self.shape = shape_of(self.shape_t)
        self.ws = torch.zeros(max(256, B.splat_batch_workspace_size()), dtype=torch.uint8, device=self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in agents]
        self.graph = None

    # -- one batched step ---------------------------------------------------------
    def _fork(self, s, fn):
        for a, st in zip(self.agents, self.streams):
            st.wait_stream(s)
            fn(a, st)
        for st in self.streams:
            s.wait_stream(st)

    def step(self, stream=None):
        s = torch.cuda.current_stream() if stream is None else stream
        self._fork(s, lambda a, st: (a.phase_clear(st), a.phase_pre(st)))
        B.splat_render_fwd_batch(self.views, self.shape, self.ws, s)
        for a in self.agents:  # associations overlap the backward launch and the updates
            a.side.wait_stream(s)
            a.phase_assoc(a.side)
        B.splat_render_bwd_batch(self.views, self.shape, self.ws, s)
        self._fork(s, lambda a, st: (a.phase_project_backward(st), a.phase_update(st, assoc=False, pose_stream=a.side)))
        for a in self.agents:
            s.wait_stream(a.side)

    def capture(self):
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step(stream=s)
        torch.cuda.current_stream().wait_stream(s)
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
        for a in self.agents:
            a.steps_done += 1

    def status(self) -> int:
        st = 0
        for a in self.agents:
            st |= a.status()
        return st

    def snapshot(self):
        for a in self.agents:
            a.snapshot()

    def restore(self):
        for a in self.agents:
            a.restore()

    # -- autotuner ----------------------------------------------------------------
    def signature(self) -> str:
        parts = [torch.cuda.get_device_name(self.device)]
        for a in self.agents:
            parts.append(f"{a.n}@{a.cam.width}x{a.cam.height}")
        return "|".join(parts)

    def autotune(self, candidates=CANDIDATES, reps: int = 5, cache_path: str | None = None, verbose=False):
        """Time `reps` graph replays of each candidate shape (state restored
        before each candidate, so every candidate sees the same scenes) and
        keep the fastest.  The choice is cached per signature in JSON."""
        cache_path = cache_path or os.environ.get(
            "SPLAT_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "splat_gb300", "autotune.json"))
        sig = self.signature()
        cache = {}
        if os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if sig in cache:
            self.set_shape(tuple(cache[sig]["shape"]))
            return cache[sig]
        self.snapshot()
        results = []
        for cand in candidates:
            self.set_shape(cand)
            self.capture()
            best = float("inf")
            for _ in range(reps):
                self.restore()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                self.replay()
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            results.append((best, cand))
            if verbose:
                print(f"autotune {cand}: {best:.3f} ms")
        self.restore()
        best_ms, best_shape = min(results)
        self.set_shape(best_shape)
        self.graph = None
        entry = {"shape": list(best_shape), "ms": best_ms,
                 "tried": [{"shape": list(c), "ms": t} for t, c in results], "when": time.time()}
        cache[sig] = entry
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
        return entry

    def set_shape(self, shape):
        self.shape_t = tuple(shape)
        self.shape = shape_of(self.shape_t)
