"""Serving loop for scene updates: continuous batching of local optimisations.

Each request is one CL-Splats update of a resident scene (Sec. 3): a few new
posed views with their change masks and target images, lifted to an active set
and optimised for a fixed number of local iterations. The paper applies the
method "in parallel to each change" (Sec. 5, "Concurrent Updates"); here the
updates of different scenes share the GPU:

* every scene's Gaussians and Adam state stay resident on the device;
* requests wait in a FIFO queue and are admitted at iteration boundaries when a
  slot is free, their scene is not already being updated, and their estimated
  HBM footprint fits the budget (continuous batching: requests that arrive
  while others run join the next iteration);
* one engine step runs one iteration of every in-flight request in the same
  launches (one scene table and one view table spanning all requests, views of
  different resolutions side by side); a composition's first step runs
  eagerly, its second is captured in a CUDA graph, and later steps replay it;
* admission work (optimiser reset, copies, lifting) and a new composition's
  tables and capacity plan run on a side stream, so the host waits only for
  that small work, never for the queued steps; the main stream waits for it
  with an event;
* a request completes after its iterations; its latency is arrival to
  completion, read back with its loss. A completed request's scene is
  deactivated in the batch (its active count set to 0 in the device table,
  which a captured graph reads too); the batch is rebuilt only when a request
  is admitted.

The plain baseline runs the same requests one at a time on the same kernels.
`Scheduler` holds the host-side policy and runs without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    scene: int
    cams: list
    masks: object          # flat uint8 tensor, views concatenated (pinned host memory)
    targets: object        # flat float32 tensor, [3][H][W] per view (pinned host memory)
    iters: int = 10
    arrival: float = 0.0
    footprint: int = 0     # estimated device bytes while in flight
    # filled while serving
    admitted: float = -1.0
    done: float = -1.0
    it: int = 0
    loss: float = float("nan")
    n_active: int = 0
    status: str = "queued"  # then "ok", "rejected: ...", "empty: ..." or "error: ..."


def _numel(x) -> int:
    return int(x.numel()) if hasattr(x, "numel") and callable(x.numel) else int(np.size(x))


def validate_request(req: Request) -> Optional[str]:
    """Host-side checks of a request before it is queued; the reason it is
    rejected, or None. A view needs a positive size, a finite pose and finite,
    positive focal lengths; the masks and targets must match the views' pixel
    counts (uint8 masks, float32 [3][H][W] targets, views concatenated); a
    change mask with no set pixel lifts no Gaussian, so there is nothing to
    optimise. Non-finite target values are not scanned here (that would read
    every pixel on the host); they show up as a non-finite loss, which marks
    the finished request as an error."""
    if not req.cams:
        return "no views"
    if req.iters <= 0:
        return "the number of iterations must be positive"
    pix = 0
    for c in req.cams:
        W, H = int(c["width"]), int(c["height"])
        if W <= 0 or H <= 0:
            return "view size must be positive"
        pose = np.concatenate([np.ravel(np.asarray(c[k], np.float64)) for k in ("R", "t", "pos")]
                              + [np.array([c["fx"], c["fy"], c["cx"], c["cy"], c["znear"]],
                                          np.float64)])
        if not np.all(np.isfinite(pose)):
            return "camera pose or intrinsics not finite"
        if not (c["fx"] > 0 and c["fy"] > 0):
            return "focal lengths must be positive"
        pix += W * H
    if req.masks is None or _numel(req.masks) != pix:
        return "change masks do not match the views"
    if not bool(req.masks.any()):
        return "empty change mask: no Gaussian can be lifted"
    if req.targets is None or _numel(req.targets) != 3 * pix:
        return "target images do not match the views"
    return None


def estimate_footprint(n_gauss: int, cams: Sequence, pairs_per_tile: int = 1024) -> int:
    """Device bytes one in-flight request needs beyond its resident scene:
    per Gaussian and view the projected record (48 B) and its binning
    workspace (packed rectangle, work-list entry, large-rectangle slot: 36 B),
    per-pixel buffers (image, target, dL/dimage, final T, last contributor,
    state after the static prefix: 64 B), per-tile tables and a key allowance
    of `pairs_per_tile` pairs of 16 B (key + scratch) per tile."""
    total = 0
    for c in cams:
        W, H = int(c["width"]), int(c["height"])
        tiles = ((W + 15) // 16) * ((H + 15) // 16)
        total += n_gauss * (48 + 36) + W * H * 64 + tiles * (256 * 8 + 80) + \
            tiles * pairs_per_tile * 16
    return total


class Scheduler:
    """Admission policy: FIFO queue, `max_slots` concurrent requests, at most
    one in-flight request per scene, and the sum of in-flight footprints within
    `budget` bytes. A request that alone exceeds the budget is rejected."""

    def __init__(self, max_slots: int, budget: int):
        self.max_slots = max_slots
        self.budget = budget
        self.queue: collections.deque = collections.deque()
        self.inflight: List[Request] = []
        self.rejected: List[Request] = []
        self.finished: List[Request] = []
        self.empty: List[Request] = []
        self.used = 0

    def submit(self, req: Request) -> None:
        reason = validate_request(req)
        if reason is None and req.footprint > self.budget:
            reason = "footprint exceeds the device budget"
        if reason is not None:
            req.status = "rejected: " + reason
            self.rejected.append(req)
            return
        self.queue.append(req)

    def retire_empty(self, req: Request, now: float, reason: str) -> None:
        """An admitted request whose lifting found no active Gaussian: it
        leaves the in-flight set without running an iteration."""
        self.inflight = [r for r in self.inflight if r is not req]
        self.used -= req.footprint
        req.done = now
        req.status = "empty: " + reason
        self.empty.append(req)

    def holds(self, age: int, interval: int) -> bool:
        """Whether admissions wait this step: requests are in flight, their
        composition has run fewer than `interval` steps, and fewer requests are
        queued than there are free slots (a full set of waiting requests is
        admitted at once)."""
        free = self.max_slots - len(self.inflight)
        return bool(self.inflight) and age < interval and len(self.queue) < free

    def admit(self, now: float) -> List[Request]:
        """Move every queued request that fits into the in-flight set, in
        arrival order, skipping (not reordering) requests whose scene is busy
        or that do not fit yet."""
        admitted = []
        busy = {r.scene for r in self.inflight}
        keep = collections.deque()
        while self.queue:
            r = self.queue.popleft()
            if (len(self.inflight) < self.max_slots and r.scene not in busy
                    and self.used + r.footprint <= self.budget):
                r.admitted = now
                self.inflight.append(r)
                busy.add(r.scene)
                self.used += r.footprint
                admitted.append(r)
            else:
                keep.append(r)
        self.queue = keep
        return admitted

    def advance(self, now: float) -> List[Request]:
        """One iteration of every in-flight request has run; retire finished
        ones and free their memory."""
        done = []
        for r in self.inflight:
            r.it += 1
            if r.it >= r.iters:
                r.done = now
                done.append(r)
        if done:
            for r in done:
                r.status = "ok"
            self.inflight = [r for r in self.inflight if r.done < 0]
            for r in done:
                self.used -= r.footprint
            self.finished.extend(done)
        return done

    def idle(self) -> bool:
        return not self.queue and not self.inflight


def latency_stats(reqs: Sequence[Request], wall: float) -> Dict[str, float]:
    lat = np.array([r.done - r.arrival for r in reqs if r.done >= 0])
    if lat.size == 0:
        return {"completed": 0}
    return {"completed": int(lat.size), "updates_per_s": lat.size / wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}


class Server:
    """GPU engine. `states` are resident SceneStates (index = scene id)."""

    def __init__(self, states, max_slots: int = 8, budget: Optional[int] = None,
                 graphs: bool = True, loss: str = "l1", lr: float = 1e-3, vote_mode: int = 0,
                 clock: Callable[[], float] = time.perf_counter, admit_interval: int = 1):
        import torch
        self.torch = torch
        self.states = states
        self.graphs = graphs
        self.loss_mode = {"l1": 1, "l2": 2}[loss]
        self.lr = lr
        self.vote_mode = vote_mode
        self.clock = clock
        if budget is None:
            free, _ = torch.cuda.mem_get_info()
            budget = int(free * 0.6)
        self.sched = Scheduler(max_slots, budget)
        self.batch = None
        self.graph = None
        self.fresh = False
        self.composition = None
        self.device_targets: Dict[int, object] = {}
        # admission and planning run beside the queued steps; high priority so
        # their short kernels take SMs as soon as the steps' blocks retire
        self.side = torch.cuda.Stream(priority=-1)
        self.capture_stream = torch.cuda.Stream()
        self.scene_free: Dict[int, object] = {}  # event after a scene's last queued step
        # while requests are in flight, admissions (each one rebuilds the
        # composition) wait until the composition has run `admit_interval`
        # steps, unless enough requests wait to fill every free slot; the check
        # comes after a step, so 1 admits at every step
        self.admit_interval = max(1, int(admit_interval))
        self._age = 0  # steps run by the current composition
        self.stats = {"steps": 0, "graph_captures": 0, "graph_replays": 0, "rebuilds": 0}

    # -- request life cycle ----------------------------------------------------
    def submit(self, req: Request) -> None:
        if not 0 <= req.scene < len(self.states):
            req.status = "rejected: unknown scene"
            self.sched.rejected.append(req)
            return
        if req.footprint == 0 and req.cams:
            req.footprint = estimate_footprint(self.states[req.scene].n, req.cams)
        self.sched.submit(req)

    def _start(self, req: Request) -> None:
        """Admission on the device (side stream, after the scene's previous
        request's queued steps): reset the scene's optimiser, copy the
        request's masks and targets from pinned host memory, lift."""
        from .update import lift
        torch = self.torch
        st = self.states[req.scene]
        main = torch.cuda.current_stream()
        with torch.cuda.stream(self.side):
            if req.scene in self.scene_free:
                self.side.wait_event(self.scene_free.pop(req.scene))
            st.adam_m.zero_()
            st.adam_v.zero_()
            st.adam_step.zero_()
            masks = req.masks.to(st.params.device, non_blocking=True)
            tgt = req.targets.to(st.params.device, non_blocking=True)
            lift(st, req.cams, masks, self.vote_mode, st.params.device)
        tgt.record_stream(main)
        for t in (st.active, st.active_idx, st.adam_m, st.adam_v, st.adam_step):
            t.record_stream(main)
        self.device_targets[req.rid] = tgt
        req.n_active = st.n_active

    def _rebuild(self) -> None:
        """Tables, buffers and capacity plan of the new composition on the side
        stream; the main stream waits for them."""
        from .update import Batch
        torch = self.torch
        reqs = self.sched.inflight
        main = torch.cuda.current_stream()
        with torch.cuda.stream(self.side):
            b = Batch([self.states[r.scene] for r in reqs], [r.cams for r in reqs],
                      self.states[reqs[0].scene].params.device)
            b.target = torch.cat([self.device_targets[r.rid] for r in reqs])
            b.plan_capacity()
            ready = torch.cuda.Event()
            ready.record(self.side)
        b.record_stream(main)
        main.wait_event(ready)
        self.batch = b
        self.batch_requests = list(reqs)
        self.composition = tuple(r.rid for r in reqs)
        self.graph = None
        self.fresh = True
        self._age = 0
        self.stats["rebuilds"] += 1

    def _iteration(self) -> None:
        b = self.batch
        b.project_and_bin(1)
        b.sort()
        b.forward(self.loss_mode)
        b.backward()
        b.adam(self.lr)

    def _step(self) -> None:
        torch = self.torch
        if not self.graphs or (self.graph is None and self.fresh):
            self._iteration()  # a composition's first step runs eagerly
            self.fresh = False
        elif self.graph is None:
            # second step of a composition: capture it (nothing runs while
            # capturing), then replay it for this step
            g = torch.cuda.CUDAGraph()
            main = torch.cuda.current_stream()
            self.capture_stream.wait_stream(main)
            with torch.cuda.stream(self.capture_stream):
                g.capture_begin()
                self._iteration()
                g.capture_end()
            main.wait_stream(self.capture_stream)
            g.replay()
            self.graph = g
            self.stats["graph_captures"] += 1
            self.stats["graph_replays"] += 1
        else:
            self.graph.replay()
            self.stats["graph_replays"] += 1
        self.stats["steps"] += 1
        self._age += 1

    def _finish(self, done: Sequence[Request]) -> None:
        """Read the finished requests' losses, take their scenes out of the
        batch's later iterations, and mark the scenes free after that."""
        torch = self.torch
        order = {r.rid: i for i, r in enumerate(self.batch_requests)}
        self.pending_losses.append((self.batch.loss.clone(), [(r, order[r.rid]) for r in done]))
        self.batch.deactivate([order[r.rid] for r in done])
        free = torch.cuda.Event()
        free.record()
        for r in done:
            self.device_targets.pop(r.rid, None)
            self.scene_free[r.scene] = free

    # -- driving loops -----------------------------------------------------------
    def serve(self, schedule: Sequence[Request], realtime: bool = True,
              run_ahead: int = 2, deadline: Optional[float] = None) -> Dict[str, float]:
        """Serve `schedule` (requests with arrival offsets in seconds). With
        `realtime` a request becomes visible at its arrival time; otherwise all
        are queued at once (closed loop, saturation). The host does not wait
        for each step: a CUDA event marks the end of every step, completion
        times are read from those events, and the host runs at most
        `run_ahead` steps ahead of the device. With a `deadline` (seconds
        after the start) no request is admitted after it; requests not
        finished are counted as `unfinished`."""
        torch = self.torch
        gc_was = gc.isenabled()
        gc.disable()  # no collector pauses inside the loop; collected once after it
        try:
            return self._serve(schedule, realtime, run_ahead, deadline)
        finally:
            if gc_was:
                gc.enable()
            gc.collect()

    def _serve(self, schedule, realtime, run_ahead, deadline) -> Dict[str, float]:
        torch = self.torch
        pending = collections.deque(sorted(schedule, key=lambda r: r.arrival))
        self.pending_losses = []
        marks = []  # (event, requests finished by that step)
        torch.cuda.synchronize()
        ref = torch.cuda.Event(enable_timing=True)
        ref.record()
        t0 = self.clock()
        for r in pending:
            r.arrival = t0 + (r.arrival if realtime else 0.0)
        recent = collections.deque()
        unfinished = 0
        while pending or not self.sched.idle():
            now = self.clock()
            if deadline is not None and now - t0 > deadline:
                unfinished = len(pending) + len(self.sched.queue)
                pending.clear()
                self.sched.queue.clear()
                if not self.sched.inflight:
                    break
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            hold = self.sched.holds(self._age, self.admit_interval)
            started = [] if hold else self.sched.admit(now)
            for r in started:
                self._start(r)
                if r.n_active == 0:  # lifting found nothing to optimise
                    self.sched.retire_empty(r, self.clock(), "no Gaussian lifted")
                    self.device_targets.pop(r.rid, None)
            if not self.sched.inflight:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - self.clock(), 0.002)))
                continue
            in_batch = set(self.composition or ())
            if any(r.rid not in in_batch for r in self.sched.inflight):
                self._rebuild()  # admissions; completions only deactivate
            self._step()
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            recent.append(ev)
            if len(recent) > run_ahead:
                recent.popleft().synchronize()
            done = self.sched.advance(self.clock())
            if done:
                self._finish(done)
                marks.append((ev, done))
        torch.cuda.synchronize()
        for ev, done in marks:
            t = t0 + ref.elapsed_time(ev) / 1e3
            for r in done:
                r.done = t
        for loss, items in self.pending_losses:
            vals = loss.cpu().numpy()
            for r, i in items:
                r.loss = float(vals[i])
                if not np.isfinite(r.loss):
                    r.status = "error: non-finite loss"
        if self.batch is not None:
            self.batch.check_status()
        wall = max(r.done for r in self.sched.finished) - t0 if self.sched.finished else 0.0
        out = latency_stats(self.sched.finished, max(wall, 1e-9))
        out.update(self.stats)
        out["rejected"] = len(self.sched.rejected)
        out["empty"] = len(self.sched.empty)
        out["errors"] = sum(1 for r in self.sched.finished if r.status.startswith("error"))
        out["unfinished"] = unfinished
        return out


def run_plain(states, schedule: Sequence[Request], loss: str = "l1", lr: float = 1e-3,
              realtime: bool = True, graphs: bool = True, deadline: Optional[float] = None,
              clock: Callable[[], float] = time.perf_counter) -> Dict[str, float]:
    """The plain loop: one request at a time, FIFO, same kernels."""
    srv = Server(states, max_slots=1, graphs=graphs, loss=loss, lr=lr, clock=clock)
    return srv.serve(schedule, realtime, deadline=deadline)
