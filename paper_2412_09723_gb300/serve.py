"""Serving loop: asynchronous per-agent tracking and mapping requests over
resident agents, with continuous batching (the asynchronous, parallel intra-
and inter-agent processing of Sec. 3.2 / 3.6, on one GPU).

* Residency, in two tiers.  An agent's state (map, Adam moments, pose) and
  its per-step buffers (frame buffers, observation and gradient images,
  association buffers: most of its footprint) are charged against an HBM
  budget separately.  When a request needs room, idle agents first give up
  their per-step buffers (nothing is copied: they are re-made, uninitialised
  work space, when the agent is next stepped), and only then are idle agents'
  states swapped out to pinned host memory -- in both tiers agents with no
  request waiting go first, least recently used first.  Nothing blocks the
  loop: released buffers are kept alive until the agent's last step has
  finished on the device; a swap-out's copies run on a copy stream after that
  step and its memory is uncharged when they are done; a swap-in, or the
  re-made buffers of a resident state, are allocated and filled on the same
  stream, and the agent's next step waits for that stream on the device, so
  the request is batched at once.  Mapping steps take the map's Adam step
  inside the projection adjoint and tracking steps form the pose gradient
  alone, so no agent holds per-parameter gradient arrays.
* Continuous batching.  At every tick the loop admits the requests that have
  arrived, takes up to `max_batch` ready requests of distinct agents (oldest
  first; an agent has at most one request in flight, so its state advances in
  order) and launches them as ONE batched step on a free stream: the frames are
  copied in from pinned host memory, every agent is projected and binned on its
  own stream, all of them are rendered forward and backward in one persistent
  launch each, and the loss, pose and Adam updates follow per agent.  Up to
  `n_streams` batches are in flight at once, so requests that arrive while
  others run are admitted as stream slots and memory free up, and their work
  overlaps on the device.  Completion is detected with CUDA events.  A batch
  of one request replays the agent's own captured single-agent step (one
  graph launch, captured and warmed when the agent becomes resident, without
  changing its state).  Python's cyclic garbage collector is off while the
  loop serves, so no collection pause lands inside a request.
* Plain mode serves the same requests one at a time in arrival order with the
  single-agent launches and a synchronisation per request.

A request is one fwd + bwd + update step: "track" updates the pose, "map"
updates the Gaussian map.  Its result is the loss of the step and the pose
after it.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import statistics
import time

import numpy as np
import torch

from . import binding as B
from .agent import Agent, StepConfig


@dataclasses.dataclass
class Request:
    agent: int
    kind: str  # "track" or "map"
    frame: int  # index of the agent's observation frame
    arrival: float  # seconds (trace time)
    rid: int = 0
    start: float = 0.0
    done: float = 0.0
    loss: float = float("nan")
    w2c: np.ndarray | None = None


class _AgentSlot:
    """Host-side record of an agent: its map when swapped out, its frames."""

    def __init__(self, aid, scene, w2c, cam, frames, cfg):
        self.aid = aid
        self.scene = scene
        self.w2c = np.asarray(w2c, np.float32)
        self.cam = cam
        self.frames = frames  # list of (rgb pinned [H,W,3], depth pinned [H,W])
        self.cfg = cfg
        self.agent: Agent | None = None
        self.host_state = None  # swapped-out device state
        self.capacity = None
        self.bytes = 0
        self.footprint = 0  # device bytes when resident (last measured)
        self.last_used = 0.0
        self.busy = False
        # pinned result buffers (an agent has at most one request in flight)
        self.out_loss = torch.empty(1, dtype=torch.float32, pin_memory=True)
        self.out_w2c = torch.empty(4, 4, dtype=torch.float32, pin_memory=True)
        self.graphs = {}  # request kind -> captured single-agent step of the resident agent
        self.state_bytes = 0  # device bytes of the state / of the per-step buffers (last measured)
        self.scratch_bytes = 0
        self.loading = None  # copy-stream event of a swap-in that may still run
        self.last_event = None  # completion event of the agent's last launched step
        self.evicting = None  # (agent, event): a swap-out whose copies may still run
        self.evict_bytes = 0
        self.side = None  # the agent's side stream, kept across swaps


def _bytes(tensors) -> int:
    """Device bytes of distinct storages among `tensors`."""
    seen = set()
    total = 0
    for t in tensors:
        if isinstance(t, torch.Tensor) and t.is_cuda:
            st = t.untyped_storage()
            if st.data_ptr() not in seen:
                seen.add(st.data_ptr())
                total += st.nbytes()
    return total


def _agent_bytes(a: Agent) -> tuple[int, int]:
    """(state bytes, per-step buffer bytes) of a resident agent."""
    return _bytes(a.state_tensors()), (_bytes(a.scratch_tensors()) if a.has_scratch else 0)


class Server:
    def __init__(self, device, hbm_budget_bytes: int, max_batch: int = 8, n_streams: int = 2,
                 shape=(256, 4, 64, 8), single_graphs: bool = True):
        self.device = device
        self.single_graphs = single_graphs  # a lone request replays its agent's captured step
        self.budget = int(hbm_budget_bytes)
        self.max_batch = min(max_batch, B.SPLAT_MAX_VIEWS)
        self.n_streams = n_streams
        self.shape = B.CBatchShape(*shape)
        self.slots: list[_AgentSlot] = []
        self.used = 0
        self.swaps = 0
        self.batch_ws = [torch.zeros(256, dtype=torch.uint8, device=device) for _ in range(n_streams)]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self.agent_streams = [[torch.cuda.Stream(device=device) for _ in range(self.max_batch)]
                              for _ in range(n_streams)]
        self.copy_stream = torch.cuda.Stream(device=device)  # swaps in and out
        self.releasing = []  # (tensors, event, bytes): per-step buffers given up, alive until the event
        self.releases = 0

    def reset(self, budget: int | None = None):
        """Drop every agent's device state (they restart from their initial
        maps and poses at the next prepare())."""
        torch.cuda.synchronize()
        for slot in self.slots:
            slot.agent = None
            slot.graphs = {}
            slot.host_state = None
            slot.bytes = 0
            slot.busy = False
            slot.last_used = 0.0
            slot.loading = slot.last_event = slot.evicting = None
            slot.evict_bytes = 0
        self.releasing = []
        self.releases = 0
        self.used = 0
        self.swaps = 0
        if budget is not None:
            self.budget = int(budget)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    # -- agents and residency -------------------------------------------------
    def add_agent(self, scene, w2c, cam, frames, cfg: StepConfig | None = None) -> int:
        slot = _AgentSlot(len(self.slots), scene, w2c, cam, frames, cfg or StepConfig(grads=False))
        self.slots.append(slot)
        return slot.aid

    def _poll_swaps(self):
        """Release the memory (and the budget) of swap-outs whose copies are
        done and of given-up per-step buffers whose last step is done, and
        forget swap-ins that have landed."""
        keep = []
        for held, ev, nbytes in self.releasing:
            if ev is None or ev.query():
                self.used -= nbytes
            else:
                keep.append((held, ev, nbytes))
        self.releasing = keep
        for slot in self.slots:
            if slot.evicting is not None and slot.evicting[1].query():
                slot.evicting = None
                self.used -= slot.evict_bytes
                slot.evict_bytes = 0
            if slot.loading is not None and slot.loading.query():
                slot.loading = None

    def _start_swap_out(self, slot: _AgentSlot):
        """Copy the agent's state to pinned host memory on the copy stream,
        after its last step; its device memory stays charged until then."""
        a = slot.agent
        cs = self.copy_stream
        if slot.last_event is not None:
            cs.wait_event(slot.last_event)
        if slot.loading is not None:
            cs.wait_event(slot.loading)
        state = a._state()
        if slot.host_state is None:  # pinned host copies, allocated once per agent and reused
            slot.host_state = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in state]
        with torch.cuda.stream(cs):
            for dst, src in zip(slot.host_state, state):
                dst.copy_(src, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(cs)
        slot.evicting = (a, ev)  # the agent (and its memory) lives until the copies are done
        slot.evict_bytes = slot.bytes
        slot.capacity = a.fb.capacity if a.has_scratch else a.capacity
        slot.agent = None
        slot.graphs = {}
        slot.bytes = 0
        slot.loading = None
        self.swaps += 1

    def _start_swap_in(self, slot: _AgentSlot, now: float):
        """Allocate the agent and copy its state in on the copy stream (after
        its own swap-out's copies, on the same stream); nothing waits on the
        host.  A first residency builds the agent from its scene instead."""
        cs = self.copy_stream
        cfg = dataclasses.replace(slot.cfg)
        if slot.side is None:
            slot.side = torch.cuda.Stream(device=self.device)
        if slot.host_state is not None:
            with torch.cuda.stream(cs):
                a = Agent(None, None, slot.cam, self.device, cfg=cfg, capacity=slot.capacity,
                          state=slot.host_state, side=slot.side)
            ev = torch.cuda.Event()
            ev.record(cs)
            slot.loading = ev
        else:
            a = Agent(slot.scene, slot.w2c, slot.cam, self.device, cfg=cfg, capacity=slot.capacity, side=slot.side)
            if slot.capacity is None:
                slot.capacity = a.fb.capacity
        slot.agent = a
        if not slot.footprint:
            slot.state_bytes, slot.scratch_bytes = _agent_bytes(a)
            slot.footprint = slot.state_bytes + slot.scratch_bytes
        slot.bytes = slot.footprint
        self.used += slot.bytes
        slot.last_used = now

    def _release_scratch(self, slot: _AgentSlot):
        """Give up an idle agent's per-step buffers; they stay alive (and
        charged) until its last launched step is done."""
        held = slot.agent.release_scratch()
        self.releasing.append((held, slot.last_event, slot.scratch_bytes))
        self.releases += 1
        slot.bytes -= slot.scratch_bytes
        slot.graphs = {}

    def _remake_scratch(self, slot: _AgentSlot, now: float):
        """Re-make the per-step buffers of a resident state on the copy
        stream (the next step waits for it)."""
        cs = self.copy_stream
        if slot.loading is not None:
            cs.wait_event(slot.loading)
        with torch.cuda.stream(cs):
            slot.agent.make_scratch(slot.agent.capacity)
        ev = torch.cuda.Event()
        ev.record(cs)
        slot.loading = ev
        slot.bytes += slot.scratch_bytes
        self.used += slot.scratch_bytes
        slot.last_used = now

    def _make_room(self, need: int, waiting, keep=None) -> bool:
        """Free memory of idle residents until `need` bytes fit the budget
        once it is released: first their per-step buffers, then -- only when
        the resident states and `need` alone exceed the budget -- their states
        (swap-outs); in each tier agents with no request waiting first, least
        recently used first; `keep` (the slot being admitted) is spared.
        True when the bytes fit now."""
        if self.used + need <= self.budget:
            return True
        freeing = (sum(sl.evict_bytes for sl in self.slots if sl.evicting is not None)
                   + sum(b for _, _, b in self.releasing))
        order = lambda x: (x.aid in waiting, x.last_used)  # noqa: E731
        idle = [sl for sl in self.slots if sl.agent is not None and not sl.busy and sl is not keep]
        for sl in sorted((sl for sl in idle if sl.agent.has_scratch), key=order):
            if self.used - freeing + need <= self.budget:
                return False
            freeing += sl.scratch_bytes
            self._release_scratch(sl)
        # states go only when the resident states alone leave no room: else
        # the per-step buffers of the agents at work free up when they finish
        states = sum(sl.state_bytes for sl in self.slots if sl.agent is not None)
        if states + need <= self.budget:
            return False
        for sl in sorted(idle, key=order):
            if self.used - freeing + need <= self.budget:
                break
            freeing += sl.bytes
            self._start_swap_out(sl)
        return False

    def _admit(self, slot: _AgentSlot, now: float, waiting=()) -> bool:
        """Make the agent resident (or loading) if the budget allows now;
        otherwise start making room and report False."""
        if slot.agent is not None:
            if slot.agent.has_scratch:
                return True
            if not self._make_room(slot.scratch_bytes, waiting, keep=slot):
                return False
            self._remake_scratch(slot, now)
            return True
        need = slot.footprint
        if need and need > self.budget:
            raise RuntimeError(f"agent {slot.aid} alone exceeds the HBM budget")
        if need and not self._make_room(need, waiting):
            return False
        self._start_swap_in(slot, now)
        if not need and self.used > self.budget:  # first residency, size learnt now: make room after the fact
            self._make_room(0, waiting, keep=slot)
        return True

    def prepare(self, size_capacity: bool = True):
        """Size every agent's duplicate buffers (one host read each, before
        serving), bringing agents in one after another and swapping earlier
        ones out when the budget requires; the agents resident at the end are
        the last ones that fit."""
        for slot in self.slots:
            while not self._admit(slot, 0.0):
                torch.cuda.synchronize()
                self._poll_swaps()
            torch.cuda.synchronize()
            self._poll_swaps()
            if size_capacity:
                slot.agent.size_capacity(1.5)
                slot.capacity = slot.agent.fb.capacity
                self.used -= slot.bytes
                slot.state_bytes, slot.scratch_bytes = _agent_bytes(slot.agent)
                slot.bytes = slot.footprint = slot.state_bytes + slot.scratch_bytes
                self.used += slot.bytes
            torch.cuda.synchronize()
        if self.single_graphs:  # the agents resident now get their single-request graphs
            for slot in self.slots:
                if slot.agent is not None and slot.agent.has_scratch:
                    self._capture(slot)

    def _capture(self, slot: _AgentSlot):
        """One captured step per request kind, taken without changing the
        agent's state."""
        a = slot.agent
        for kind in ("track", "map"):
            a.cfg.track = kind == "track"
            a.cfg.map = kind == "map"
            a.capture(keep_state=True)
            slot.graphs[kind] = a.graph
        a.graph = None

    # -- one batched step ---------------------------------------------------------
    def _launch(self, reqs, si):
        s = self.streams[si]
        for r in reqs:  # agents still being copied in: the step waits for the copy stream on the device
            if self.slots[r.agent].loading is not None:
                s.wait_event(self.slots[r.agent].loading)
        if len(reqs) == 1 and self.slots[reqs[0].agent].graphs:
            return self._launch_graph(reqs[0], s)
        agents = [self.slots[r.agent].agent for r in reqs]
        views = (B.CView * len(agents))(*[a.view() for a in agents])
        ast = self.agent_streams[si]
        with torch.cuda.stream(s):
            for r, a in zip(reqs, agents):
                rgb, depth = self.slots[r.agent].frames[r.frame]
                a.obs_rgb.copy_(rgb, non_blocking=True)
                a.obs_depth.copy_(depth, non_blocking=True)
        for a, st in zip(agents, ast):
            st.wait_stream(s)
            a.phase_clear(st)
            a.phase_pre(st)
        for st in ast[:len(agents)]:
            s.wait_stream(st)
        B.splat_render_fwd_batch(views, self.shape, self.batch_ws[si], s)
        B.splat_render_bwd_batch(views, self.shape, self.batch_ws[si], s)
        for r, a, st in zip(reqs, agents, ast):
            st.wait_stream(s)
            a.cfg.track = r.kind == "track"
            a.cfg.map = r.kind == "map"
            a.phase_project_backward(st)
            a.phase_update(st)
        for st in ast[:len(agents)]:
            s.wait_stream(st)
        outs = []
        with torch.cuda.stream(s):
            for r, a in zip(reqs, agents):
                slot = self.slots[r.agent]
                slot.out_loss.copy_(a.loss, non_blocking=True)
                slot.out_w2c.copy_(a.w2c, non_blocking=True)
                outs.append((slot.out_loss, slot.out_w2c))
        ev = torch.cuda.Event()
        ev.record(s)
        return ev, outs

    def _launch_graph(self, r, s):
        """A lone request: its frame is copied in and the agent's captured step
        for the request kind is replayed on stream s."""
        slot = self.slots[r.agent]
        a = slot.agent
        rgb, depth = slot.frames[r.frame]
        with torch.cuda.stream(s):
            a.obs_rgb.copy_(rgb, non_blocking=True)
            a.obs_depth.copy_(depth, non_blocking=True)
            slot.graphs[r.kind].replay()
            slot.out_loss.copy_(a.loss, non_blocking=True)
            slot.out_w2c.copy_(a.w2c, non_blocking=True)
        a.steps_done += 1
        a.grads_clean = False
        ev = torch.cuda.Event()
        ev.record(s)
        return ev, [(slot.out_loss, slot.out_w2c)]

    def _mark_launched(self, reqs, ev):
        for r in reqs:
            self.slots[r.agent].last_event = ev

    def _finish(self, reqs, outs, now):
        for r, (loss, w2c) in zip(reqs, outs):
            r.done = now
            r.loss = float(loss.item())
            r.w2c = w2c.numpy().copy()
            slot = self.slots[r.agent]
            slot.busy = False
            slot.last_used = now

    # -- the loop -------------------------------------------------------------------
    def serve(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times in seconds from the start).  With
        `realtime`, a request becomes visible at its arrival time on the host
        clock; otherwise all are submitted at time 0 (saturation), and their
        arrival is set to 0."""
        if not realtime:
            for r in requests:
                r.arrival = 0.0
        with _no_gc():
            return self._serve(requests, realtime)

    def _serve(self, requests, realtime):
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        ready = collections.deque()
        in_flight = {}  # stream index -> (event, reqs, outs)
        t0 = time.perf_counter()
        n_done = 0
        total = len(pending)
        while n_done < total:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                ready.append(pending.popleft())
            self._poll_swaps()
            # completions
            for si in list(in_flight):
                ev, reqs, outs = in_flight[si]
                if ev.query():
                    self._finish(reqs, outs, time.perf_counter() - t0)
                    n_done += len(reqs)
                    del in_flight[si]
            # admissions: free stream slots take the oldest ready requests of idle, resident agents
            free = [si for si in range(self.n_streams) if si not in in_flight]
            waiting = {r.agent for r in ready}
            while free and ready:
                batch, seen, keep = [], set(), collections.deque()
                # requests of resident agents first; swap agents in only when none is left
                failed = set()
                for resident_only in (True, False):
                    if batch:
                        break
                    while ready and len(batch) < self.max_batch:
                        r = ready.popleft()
                        slot = self.slots[r.agent]
                        if (r.agent in seen or r.agent in failed or slot.busy
                                or (resident_only and slot.agent is None)):
                            keep.append(r)
                            continue
                        if not self._admit(slot, now, waiting):
                            failed.add(r.agent)
                            keep.append(r)
                            continue
                        seen.add(r.agent)
                        slot.busy = True  # from here on it cannot be swapped out for another batch member
                        batch.append(r)
                    ready.extendleft(reversed(keep))
                    keep = collections.deque()
                if not batch:
                    break
                si = free.pop(0)
                for r in batch:
                    r.start = now
                ev, outs = self._launch(batch, si)
                self._mark_launched(batch, ev)
                in_flight[si] = (ev, batch, outs)
            if not in_flight and not ready and pending and realtime:
                time.sleep(max(0.0, min(0.0005, pending[0].arrival - (time.perf_counter() - t0))))
            elif not in_flight and ready:  # waiting for memory: swap-outs in flight
                time.sleep(0.00005)
        torch.cuda.synchronize()
        self._poll_swaps()
        status = 0
        for slot in self.slots:
            if slot.agent is not None:
                status |= slot.agent.status()
        if status:
            raise RuntimeError(f"device status {status} while serving")
        return time.perf_counter() - t0

    def serve_plain(self, requests, realtime: bool = True):
        """The per-request path: one request at a time in arrival order
        (without `realtime`, all are submitted at time 0)."""
        order = sorted(requests, key=lambda r: (r.arrival, r.rid))
        if not realtime:
            for r in order:
                r.arrival = 0.0
        with _no_gc():
            return self._serve_plain(order, realtime)

    def _serve_plain(self, order, realtime):
        t0 = time.perf_counter()
        s = torch.cuda.current_stream()
        for r in order:
            now = time.perf_counter() - t0
            if realtime and r.arrival > now:
                time.sleep(r.arrival - now)
            slot = self.slots[r.agent]
            while not self._admit(slot, time.perf_counter() - t0):
                self.copy_stream.synchronize()  # the swap-outs that make room
                self._poll_swaps()
            if slot.loading is not None:
                s.wait_event(slot.loading)
            a = slot.agent
            r.start = time.perf_counter() - t0
            rgb, depth = slot.frames[r.frame]
            a.obs_rgb.copy_(rgb, non_blocking=True)
            a.obs_depth.copy_(depth, non_blocking=True)
            a.cfg.track = r.kind == "track"
            a.cfg.map = r.kind == "map"
            a.step(stream=s)
            r.loss = float(a.loss.item())  # synchronises
            r.w2c = a.w2c.cpu().numpy()
            r.done = time.perf_counter() - t0
            slot.last_used = r.done
        return time.perf_counter() - t0


class _no_gc:
    """The Python collector stays off while requests are served (a collection
    of the host's object graph can take tens of milliseconds)."""

    def __enter__(self):
        gc.collect()
        self.was = gc.isenabled()
        gc.disable()

    def __exit__(self, *exc):
        if self.was:
            gc.enable()


def latency_stats(requests, makespan):
    lat = [1e3 * (r.done - r.arrival) for r in requests]
    lat.sort()
    k = max(0, int(np.ceil(0.99 * len(lat))) - 1)
    return {"requests": len(requests), "frames_per_s": len(requests) / makespan, "p50_ms": statistics.median(lat),
            "p99_ms": lat[k], "mean_ms": float(np.mean(lat)), "makespan_s": makespan}


def poisson_trace(n_agents, rate_hz, duration_s, frames_per_agent, map_every=5, seed=0):
    """Poisson tracking requests per agent; every `map_every`-th frame of an
    agent also carries a mapping request."""
    rng = np.random.default_rng(seed)
    reqs = []
    for a in range(n_agents):
        t, k = 0.0, 0
        while True:
            t += rng.exponential(1.0 / rate_hz)
            if t > duration_s:
                break
            f = k % frames_per_agent
            reqs.append(Request(a, "track", f, t))
            if (k + 1) % map_every == 0:
                reqs.append(Request(a, "map", f, t))
            k += 1
    reqs.sort(key=lambda r: r.arrival)
    for i, r in enumerate(reqs):
        r.rid = i
    return reqs


def make_agents_workload(server: Server, agents_spec, frames_per_agent=8, seed=0, device=None):
    """Register agents (dicts with n, seed, cam) on `server`: each gets a room
    map, a start pose near the room centre and `frames_per_agent` observation
    frames rendered from a trajectory of poses 1 cm / 0.5 degree apart (on the
    GPU, then kept in pinned host memory)."""
    from . import scenes

    device = device or server.device
    for spec in agents_spec:
        sc = scenes.scene_room(spec["n"], spec["seed"])
        w2c0 = scenes.perturbed_w2c(spec["seed"] + 7, 0.05, 5.0)
        tmp = Agent(sc, w2c0, spec["cam"], device)
        frames = []
        pose = w2c0
        for f in range(frames_per_agent):
            pose = scenes.perturbed_w2c(spec["seed"] * 100 + f, 0.01, 0.5, base=pose)
            fb = tmp.render_observation_from(pose)
            frames.append((fb.image["rgb"].cpu().pin_memory(), fb.image["depth"].cpu().pin_memory()))
        del tmp
        server.add_agent(sc, w2c0, spec["cam"], frames)
    torch.cuda.synchronize()
