"""Continuous-batching evaluation server for many concurrent pulse optimisations.

Each session (one optimiser) owns a resident problem: its model tables, its controls and window
states and its scratch stay on the device between optimiser iterations; a request carries the
optimiser's new iterate (alpha, W) and asks for the objective or the objective and gradient.
Sessions are admitted while their device memory (including the midpoint history a gradient
needs) fits the server's budget; a session that does not fit raises ``NotAdmitted``.

Scheduling (host side, this module): requests join their session's queue on arrival; a session
has at most one request on the GPU (an optimiser needs the previous result before its next
step), so the head of every idle session's queue is *ready*.  Whenever one of the
``MSQOC_BATCH_SLOTS`` dispatch slots is free, the scheduler picks a (shape, kind) class and
dispatches ready requests of that class as one subset of the server's batch
(``msqoc_batch_eval_subset``): their sweeps share launches.  Each class has at most one
dispatch in flight and each slot its own CUDA streams, so requests that arrive while others run
are admitted as slots free up and their kernels overlap on the device.  Two policies:

* ``fifo`` (default): requests advance in arrival order.  A ready request is eligible while
  fewer than ``lookahead`` requests that arrived before it are unfinished; the class of the
  oldest eligible ready request is dispatched with every eligible ready request of that class.
  The dispatch holding the oldest unfinished request runs on the highest-priority stream, the
  other eligible dispatches on a middle one.  Requests of cheap classes (each below
  ``cheap_flops``) may also run ahead of the window, on at most ``background_slots`` slots and
  the lowest-priority stream, so they fill what the large shapes leave idle without holding
  them back.
* ``throughput``: any ready request is eligible; cheap classes and classes that waited longer
  than ``age_limit`` run on high-priority streams.  It completes the most evaluations but
  serves the expensive shapes later than arrival order.

All arithmetic runs in the library's kernels; this module only moves pointers, streams and
events.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import msqoc

SLOTS = 4   # MSQOC_BATCH_SLOTS


class NotAdmitted(RuntimeError):
    """The session's device memory does not fit the server's budget."""


@dataclasses.dataclass
class Request:
    session: int
    gradient: bool
    alpha: np.ndarray
    W: Optional[np.ndarray]
    arrival: float = 0.0          # seconds from the start of Server.run
    ready: float = math.nan       # reached the head of an idle session's queue
    dispatched: float = math.nan
    done: float = math.nan
    result: Optional[dict] = None
    slot: int = -1                # dispatch slot (served) or -1 (one at a time)
    events: Optional[tuple] = None   # (start, end) CUDA events of its dispatch, when recorded


def eval_flops(spec, gradient: bool) -> float:
    """Algorithmic FP64 flops of one evaluation (one H-apply per implicit step, the 2Ubar - U
    update, and for the gradient the adjoint sweep and its inner products): the scheduler's
    cost estimate of a request."""
    nnz = spec.q * 2 * spec.N * (spec.L - 1) // spec.L
    f_step = 8 * nnz + 6 * spec.N
    fwd = spec.E * spec.nsteps * f_step
    return float(fwd + (spec.E * spec.nsteps * (f_step + 8 * nnz) if gradient else 0))


class _Dispatched:
    """Fenwick tree over request indices marking requests (the finished ones): how many marked
    requests precede index i, in O(log n)."""

    def __init__(self, n: int):
        self.t = [0] * (n + 1)

    def mark(self, i: int):
        i += 1
        while i < len(self.t):
            self.t[i] += 1
            i += i & -i

    def before(self, i: int) -> int:
        c = 0
        while i > 0:
            c += self.t[i]
            i -= i & -i
        return c


class _CudaDevice:
    """The streams, events and synchronisation of the serving loop (torch.cuda)."""

    def __init__(self):
        import torch
        self.torch = torch

    def priority_range(self):
        S = self.torch.cuda.Stream
        return S.priority_range() if hasattr(S, "priority_range") else (0, -5)

    def stream(self, priority: int):
        return self.torch.cuda.Stream(priority=priority)

    def event(self, timing: bool):
        return self.torch.cuda.Event(enable_timing=timing)

    def current_stream(self):
        return self.torch.cuda.current_stream()

    def synchronize(self):
        self.torch.cuda.synchronize()


class Server:
    """Sessions and the continuous-batching loop.

    policy "fifo": a ready request is eligible while fewer than `lookahead` requests that
    arrived before it are unfinished; a dispatch takes every eligible ready request of the class
    of the oldest one (up to `dispatch_flops` of estimated work, at least one request); the
    dispatch holding the oldest unfinished request runs on the highest-priority stream.  Ready
    requests of classes costing less than `cheap_flops` each may run ahead of the window on at
    most `background_slots` slots, at the lowest priority.
    policy "throughput": every ready request is eligible; a dispatch takes the ready requests of
    the oldest one's class up to `dispatch_flops`; classes whose requests cost less than
    `cheap_flops` each, or whose oldest ready request has waited longer than `age_limit`
    seconds, run on high-priority streams."""

    def __init__(self, device_budget_bytes: int, policy: str = "fifo", lookahead: int = 16,
                 dispatch_flops: float = 2.1e11, cheap_flops: float = 1e9, background_slots: int = 2,
                 age_limit: float = 1.0):
        if policy not in ("fifo", "throughput"):
            raise ValueError(f"unknown policy {policy!r}")
        self.budget = int(device_budget_bytes)
        self.used = 0
        self.sessions: List[msqoc.Problem] = []
        self.batch: Optional[msqoc.Batch] = None
        self.policy = policy
        self.lookahead = int(lookahead)
        self.dispatch_flops = dispatch_flops
        self.cheap_flops = cheap_flops
        self.background_slots = int(background_slots)
        self.age_limit = age_limit

    # ------------------------------------------------------------------ sessions
    def admit(self, spec, ckpt_interval: int = 0, solver: int = msqoc.SOLVER_DEFAULT) -> int:
        """Create a session for `spec` if its device memory fits; returns the session id."""
        p = msqoc.Problem(spec, ckpt_interval=ckpt_interval, solver=solver)
        if self.used + p.device_bytes > self.budget:
            need = p.device_bytes
            p.close()
            raise NotAdmitted(f"session needs {need} bytes; {self.budget - self.used} of {self.budget} free")
        self.used += p.device_bytes
        self.sessions.append(p)
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        return len(self.sessions) - 1

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for p in self.sessions:
            p.close()
        self.sessions = []
        self.used = 0

    def _shape(self, sid: int):
        sp = self.sessions[sid].spec
        return (sp.L, sp.q)

    # ------------------------------------------------------------------ serving
    def run(self, requests: Sequence[Request], duration: Optional[float] = None,
            record_events: bool = False, device=None, trace: Optional[list] = None) -> List[Request]:
        """Serve `requests` (sorted by arrival time, seconds from now).  Stops when all are done,
        or at `duration` seconds (requests then still queued or in flight are not completed).
        Returns the completed requests with their results and timestamps.  With
        `record_events`, each request's `events` holds CUDA timing events recorded on its
        dispatch's stream before its inputs are staged and after its launches, and
        `self.base_event` one recorded before the loop (device-side start and end offsets of
        every dispatch: `base_event.elapsed_time(ev)`).  `device` replaces torch.cuda's streams
        and events (tests of the scheduling on CPU); `trace`, if a list, receives one tuple
        (time, slot, priority level 0-2, background, [request indices], class) per dispatch."""
        dv = device if device is not None else _CudaDevice()
        if self.batch is None:
            self.batch = msqoc.Batch(self.sessions, gradient=True)
        b = self.batch
        fifo = self.policy == "fifo"
        # per slot a lowest-, a middle- and a highest-priority stream (a lower number is a higher
        # priority; CUDA clamps values beyond the device's range)
        lo_pri, hi_pri = dv.priority_range()
        mid_pri = (lo_pri + hi_pri) // 2 if hi_pri < lo_pri else lo_pri
        streams = [(dv.stream(lo_pri), dv.stream(mid_pri), dv.stream(hi_pri)) for _ in range(SLOTS)]
        cost = [(eval_flops(p.spec, False), eval_flops(p.spec, True)) for p in self.sessions]
        queues: Dict[int, collections.deque] = {s: collections.deque() for s in range(len(self.sessions))}
        n = len(requests)
        index = {id(r): i for i, r in enumerate(requests)}
        finished = _Dispatched(n)          # marks finished requests
        is_done = [False] * n
        oldest = 0                         # index of the oldest unfinished request
        busy = [False] * len(self.sessions)
        inflight = {}            # slot -> (event, class, [requests], background)
        busy_class = set()
        free_slots = list(range(SLOTS))
        n_background = 0
        done: List[Request] = []
        self.base_event = None
        if record_events:
            self.base_event = dv.event(True)
            self.base_event.record(dv.current_stream())
        t0 = time.perf_counter()
        nxt = 0
        while len(done) < n:
            now = time.perf_counter() - t0
            if duration is not None and now >= duration:
                break
            progressed = False
            while nxt < n and requests[nxt].arrival <= now:
                r = requests[nxt]
                queues[r.session].append(r)
                nxt += 1
                progressed = True
            # completions
            for slot in list(inflight):
                ev, cls, reqs, bg = inflight[slot]
                if ev.query():
                    tdone = time.perf_counter() - t0
                    for r in reqs:
                        r.result = b.get_gradient(r.session) if r.gradient else b.get_objective(r.session)
                        r.done = tdone
                        busy[r.session] = False
                        i = index[id(r)]
                        is_done[i] = True
                        finished.mark(i)
                    done.extend(reqs)
                    del inflight[slot]
                    busy_class.discard(cls)
                    free_slots.append(slot)
                    n_background -= 1 if bg else 0
                    progressed = True
            while oldest < n and is_done[oldest]:
                oldest += 1
            if progressed:
                now = time.perf_counter() - t0   # dispatches below come after these completions
            # dispatch
            while free_slots:
                ready = []
                for s, q in queues.items():
                    if q and not busy[s]:
                        r = q[0]
                        if math.isnan(r.ready):
                            r.ready = max(r.arrival, now)
                        if (self._shape(r.session), r.gradient) not in busy_class:
                            ready.append(r)
                if not ready:
                    break
                background = False
                if fifo:
                    # eligible: fewer than `lookahead` unfinished requests arrived before it
                    elig = [r for r in ready if index[id(r)] - finished.before(index[id(r)]) < self.lookahead]
                    if not elig and n_background < self.background_slots:
                        elig = [r for r in ready if cost[r.session][1 if r.gradient else 0] < self.cheap_flops]
                        background = True
                    if not elig:
                        break
                    pool = elig
                else:
                    pool = ready
                first = min(pool, key=lambda r: r.arrival)
                cls = (self._shape(first.session), first.gradient)
                sel, work = [], 0.0
                for r in sorted((r for r in pool if (self._shape(r.session), r.gradient) == cls),
                                key=lambda r: r.arrival):
                    c = cost[r.session][1 if r.gradient else 0]
                    if sel and work + c > self.dispatch_flops:
                        break
                    sel.append(r)
                    work += c
                slot = free_slots.pop()
                if fifo:
                    pri = 0 if background else (2 if any(index[id(r)] == oldest for r in sel) else 1)
                else:
                    cheap = cost[first.session][1 if first.gradient else 0] < self.cheap_flops
                    pri = 2 if (cheap or now - first.ready > self.age_limit) else 0
                stream = streams[slot][pri]
                ev0 = None
                if record_events:
                    ev0 = dv.event(True)
                    ev0.record(stream)
                for r in sel:
                    queues[r.session].popleft()
                    busy[r.session] = True
                    r.dispatched = now
                    r.slot = slot
                    b.set_inputs(r.session, r.alpha, r.W, stream=stream)
                b.eval_subset([r.session for r in sel], gradient=cls[1], slot=slot, stream=stream)
                ev = dv.event(record_events)
                ev.record(stream)
                if trace is not None:
                    trace.append((now, slot, pri, background, [index[id(r)] for r in sel], cls))
                if record_events:
                    for r in sel:
                        r.events = (ev0, ev)
                inflight[slot] = (ev, cls, sel, background)
                n_background += 1 if background else 0
                busy_class.add(cls)
                progressed = True
            if not progressed:
                time.sleep(0.0002)
        dv.synchronize()
        return done

    def run_plain(self, requests: Sequence[Request], duration: Optional[float] = None) -> List[Request]:
        """The same requests one at a time in arrival order, each its own synchronous
        evaluation (one problem per launch sequence, nothing overlapped).  A request is ready,
        as in `run`, once it has arrived and its session's previous request is done; as in
        `run`, a request that finishes after `duration` is not counted."""
        t0 = time.perf_counter()
        done: List[Request] = []
        last_done: Dict[int, float] = {}
        for r in requests:
            now = time.perf_counter() - t0
            if duration is not None and now >= duration:
                break
            if r.arrival > now:
                time.sleep(r.arrival - now)
                now = time.perf_counter() - t0
            r.ready = max(r.arrival, last_done.get(r.session, 0.0))
            r.dispatched = now
            p = self.sessions[r.session]
            r.result = p.eval_gradient(r.alpha, r.W) if r.gradient else p.eval_objective(r.alpha, r.W)
            r.done = time.perf_counter() - t0
            last_done[r.session] = r.done
            if duration is not None and r.done > duration:
                break            # finished after the end of the run: not counted, as in `run`
            done.append(r)
        return done


def poisson_requests(sessions: Sequence, rate: float, duration: float, seed: int,
                     gradient_fraction: float = 0.5, inputs=None, variants: int = 2) -> List[Request]:
    """A Poisson stream of `rate` requests/s for `duration` s over the given sessions (uniformly
    drawn), objective or gradient with the given split.  inputs(session, k) gives the k-th
    iterate (alpha, W) of a session; by default each session cycles through `variants` seeded
    synthetic iterates, generated once (an iterate of the 5-transmon workload is 32 MB, so a
    long stream must not hold one per request)."""
    from . import synthetic as S
    rng = np.random.default_rng(seed)
    cache = {}

    def default_inputs(s, k):
        key = (s, k % variants)
        if key not in cache:
            sp = sessions[s]
            v = seed + 1000 * key[1]
            cache[key] = (S.random_alpha(sp, v, problem=s), S.random_W(sp, v, problem=s) if sp.M > 1 else None)
        return cache[key]

    get = inputs if inputs is not None else default_inputs
    t, out, count = 0.0, [], collections.Counter()
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        s = int(rng.integers(len(sessions)))
        k = count[s]
        count[s] += 1
        a, W = get(s, k)
        out.append(Request(session=s, gradient=bool(rng.random() < gradient_fraction), alpha=a,
                           W=W if sessions[s].M > 1 else None, arrival=t))
    return out


def latency_summary(done: Sequence[Request]) -> dict:
    """p50/p99 (ms) from arrival, from readiness (head of an idle session's queue) and of the
    service alone (dispatch to completion)."""
    if not done:
        return {}
    out = {}
    for key, t in (("from_arrival", lambda r: r.arrival), ("from_ready", lambda r: r.ready),
                   ("service", lambda r: r.dispatched)):
        x = np.array([r.done - t(r) for r in done]) * 1e3
        out[key] = {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99))}
    return out
