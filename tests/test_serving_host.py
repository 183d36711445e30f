"""Host-side parts of the serving loop (no GPU): the request stream and the latency summary."""
import math

import numpy as np
import pytest

from paper_2407_13950_gb300 import serving
from paper_2407_13950_gb300 import synthetic as S


def test_poisson_stream_is_seeded_sorted_and_has_the_rate():
    sessions = [S.config_2q(), S.config_3q()]
    a = serving.poisson_requests(sessions, rate=500.0, duration=4.0, seed=3)
    b = serving.poisson_requests(sessions, rate=500.0, duration=4.0, seed=3)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))
    assert abs(len(a) - 2000) < 5 * math.sqrt(2000)          # Poisson count, 5 sigma
    frac = np.mean([r.gradient for r in a])
    assert abs(frac - 0.5) < 0.05
    for r in a[:20]:
        sp = sessions[r.session]
        assert r.alpha.shape == (sp.d,) and r.W.shape == (sp.nW,)


def test_latency_summary():
    reqs = [serving.Request(session=0, gradient=True, alpha=None, W=None, arrival=0.0, ready=0.5, done=1.0 + i)
            for i in range(100)]
    lat = serving.latency_summary(reqs)
    assert abs(lat["from_arrival"]["p50"] - 1000 * np.percentile(1.0 + np.arange(100), 50)) < 1e-6
    assert lat["from_ready"]["p99"] < lat["from_arrival"]["p99"]


# ---------------------------------------------------------------- the scheduler on CPU
# A fake device and batch stand in for the GPU: a dispatch takes its requests' algorithmic flops
# / 2e13 seconds of wall time on its stream, and each request's result is a function of its own
# inputs, so the scheduling rules can be checked without a GPU.
import time as _time


class _FakeStream:
    def __init__(self, priority):
        self.priority = priority


class _FakeEvent:
    def __init__(self, dev):
        self.dev, self.t = dev, None

    def record(self, stream):
        self.t = self.dev.end.get(id(stream), _time.perf_counter())

    def query(self):
        return _time.perf_counter() >= self.t


class _FakeDevice:
    def __init__(self):
        self.end = {}

    def priority_range(self):
        return (0, -5)

    def stream(self, priority):
        return _FakeStream(priority)

    def event(self, timing):
        return _FakeEvent(self)

    def current_stream(self):
        return _FakeStream(0)

    def synchronize(self):
        while self.end and _time.perf_counter() < max(self.end.values()):
            _time.sleep(0.0005)


class _FakeBatch:
    def __init__(self, dev, specs):
        self.dev, self.specs, self.inputs, self.results = dev, specs, {}, {}

    def set_inputs(self, i, alpha, W, stream=None):
        self.inputs[i] = float(alpha[0])

    def eval_subset(self, members, gradient=True, slot=0, stream=None):
        now = _time.perf_counter()
        work = sum(serving.eval_flops(self.specs[m], gradient) for m in members)
        self.dev.end[id(stream)] = max(now, self.dev.end.get(id(stream), now)) + work / 2e13
        for m in members:
            self.results[m] = {"P": self.inputs[m] * (2.0 if gradient else 3.0)}

    def get_gradient(self, i):
        return self.results[i]

    def get_objective(self, i):
        return self.results[i]


class _FakeSession:
    def __init__(self, spec):
        self.spec, self.device_bytes = spec, 1


def _fake_server(policy, lookahead=6):
    specs = [S.config_2q(), S.config_3q(), S.config_4q(), S.config_5q()] * 4
    srv = serving.Server(device_budget_bytes=1 << 40, policy=policy, lookahead=lookahead)
    srv.sessions = [_FakeSession(sp) for sp in specs]
    dev = _FakeDevice()
    srv.batch = _FakeBatch(dev, specs)
    reqs = []
    rng = np.random.default_rng(4)
    t = 0.0
    for k in range(160):
        t += rng.exponential(0.0003)
        s = int(rng.integers(len(specs)))
        reqs.append(serving.Request(session=s, gradient=bool(k % 2), alpha=np.array([k + 1.0]), W=None,
                                    arrival=t))
    return srv, dev, reqs, specs


@pytest.mark.parametrize("policy", ["fifo", "throughput"])
def test_scheduler_rules_on_a_fake_device(policy):
    srv, dev, reqs, specs = _fake_server(policy)
    trace = []
    done = srv.run(reqs, device=dev, trace=trace)
    assert len(done) == len(reqs)
    for k, r in enumerate(reqs):   # every request got its own result
        assert r.result["P"] == (k + 1.0) * (2.0 if r.gradient else 3.0)
        assert r.arrival <= r.dispatched <= r.done
    # a session has one request on the device at a time, in arrival order
    for s in range(len(specs)):
        mine = [r for r in reqs if r.session == s]
        for a, b in zip(mine, mine[1:]):
            assert b.dispatched >= a.done and b.dispatched >= a.dispatched
    # a class has one dispatch in flight at a time
    disp = [(t, slot, pri, bg, idx, cls, max(reqs[i].done for i in idx)) for t, slot, pri, bg, idx, cls in trace]
    for i, a in enumerate(disp):
        for b in disp[i + 1:]:
            if a[5] == b[5]:
                assert b[0] >= a[6] or a[0] >= b[6]
    if policy == "fifo":
        done_at = [r.done for r in reqs]
        for t, slot, pri, bg, idx, cls, end in disp:
            if bg:      # background: cheap classes only, at the lowest priority
                assert pri == 0
                assert all(serving.eval_flops(specs[reqs[i].session], reqs[i].gradient) < srv.cheap_flops
                           for i in idx)
            else:       # inside the window of unfinished requests
                for i in idx:
                    assert sum(1 for j in range(i) if done_at[j] > t) < srv.lookahead
            oldest = next(j for j in range(len(reqs)) if done_at[j] > t)
            if oldest in idx:
                assert pri == 2
        # at most `background_slots` background dispatches in flight at once
        bgs = [(a[0], a[6]) for a in disp if a[3]]
        for t0, _ in bgs:
            assert sum(1 for a, b in bgs if a <= t0 < b) <= srv.background_slots
