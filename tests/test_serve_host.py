"""Scheduling logic of the serving loop on the host, with stand-in slots (no GPU).

The stand-in slot of a request completes one cycle every `dt` seconds of a simulated clock,
so the tests control time exactly: admission waits for arrival and for memory, never exceeds
the budget, keeps first-come-first-served order, overlaps requests that fit together, and
accounts every cycle and every grid-point analysis.
"""
import pytest

import synth
from paper_2308_03310_gb300.serve import Request, Server


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeSlot:
    def __init__(self, req, clock, dt=0.01):
        self.req, self.clock, self.dt = req, clock, dt
        self.enqueued = self.finished = 0
        self.latencies_ms = []
        self.queue = []

    def enqueue_cycle(self):
        start = max([self.clock()] + [t for t in self.queue])
        self.queue.append(start + self.dt)
        self.enqueued += 1

    def poll(self):
        n = 0
        while self.queue and self.queue[0] <= self.clock():
            self.queue.pop(0)
            self.finished += 1
            self.latencies_ms.append(self.dt * 1e3)
            n += 1
        return n

    def done(self):
        return self.finished >= self.req.cycles

    def close(self):
        self.closed_at = self.clock()


def _serve(reqs, budget, fp):
    clk = Clock()
    srv = Server(budget, lambda r: FakeSlot(r, clk), fp, clock=clk, sleep=clk.sleep)
    return srv.run(reqs)


def _reqs(specs):
    return [Request(rid=i, arrival_s=a, nx=n, ny=n, k=8, obs_stride=4, cycles=c)
            for i, (a, n, c) in enumerate(specs)]


def test_every_request_completes_and_is_accounted():
    reqs = _reqs([(0.0, 16, 3), (0.001, 32, 5), (0.002, 24, 2)])
    rep = _serve(reqs, budget=10 ** 9, fp=lambda r: 1000)
    assert rep["completed"] == 3 and rep["cycles"] == 10
    assert rep["analyses"] == 16 * 16 * 3 + 32 * 32 * 5 + 24 * 24 * 2
    assert rep["max_concurrent"] == 3        # all fit: they overlap


def test_admission_waits_for_memory_and_never_exceeds_the_budget():
    reqs = _reqs([(0.0, 16, 5), (0.0, 16, 5), (0.0, 16, 5), (0.0, 16, 5)])
    fp = lambda r: 400
    rep = _serve(reqs, budget=1000, fp=fp)            # two at a time
    assert rep["completed"] == 4
    assert rep["peak_footprint_bytes"] <= 1000 and rep["max_concurrent"] == 2
    used = [u for (_, _, _, u) in rep["timeline"]]
    assert max(used) <= 1000
    admits = [(t, rid) for (t, ev, rid, _) in rep["timeline"] if ev == "admit"]
    assert [rid for _, rid in admits] == [0, 1, 2, 3]    # first come, first served
    assert admits[2][0] > 0.0 and admits[3][0] > 0.0     # the last two waited
    assert rep["admission_wait_s"]["max"] > 0.0


def test_admission_waits_for_arrival():
    reqs = _reqs([(0.0, 16, 2), (0.5, 16, 2)])
    rep = _serve(reqs, budget=10 ** 6, fp=lambda r: 10)
    admits = {rid: t for (t, ev, rid, _) in rep["timeline"] if ev == "admit"}
    assert admits[1] >= 0.5


def test_oversized_request_is_rejected():
    with pytest.raises(ValueError):
        _serve(_reqs([(0.0, 16, 1)]), budget=10, fp=lambda r: 11)


def test_poisson_stream_is_seeded_and_ordered():
    a = synth.poisson_requests(50, 20.0, 5)
    b = synth.poisson_requests(50, 20.0, 5)
    assert a == b
    t = [r["arrival_s"] for r in a]
    assert t == sorted(t) and 1.0 < t[-1] < 5.0          # ~2.5 s for 50 arrivals at 20/s
    assert {r["nx"] for r in a} <= {128, 256, 512, 1024}
    assert all(10 <= r["cycles"] <= 100 for r in a)


def test_small_cycles_get_the_urgent_stream_priority():
    from paper_2308_03310_gb300.serve import SMALL_WORK, size_class, stream_priority
    small = Request(rid=0, arrival_s=0.0, nx=256, ny=256, k=64, obs_stride=4, cycles=1)
    large = Request(rid=1, arrival_s=0.0, nx=1024, ny=1024, k=16, obs_stride=4, cycles=1)
    tiny = Request(rid=2, arrival_s=0.0, nx=128, ny=128, k=128, obs_stride=8, cycles=1)
    assert 256 * 256 * 64 == SMALL_WORK
    assert [size_class(r) for r in (small, large, tiny)] == ["small", "large", "small"]
    assert stream_priority(small) < stream_priority(large) == 0


def test_latency_is_reported_per_size_class():
    reqs = [Request(rid=i, arrival_s=0.0, nx=n, ny=n, k=16, obs_stride=4, cycles=2)
            for i, n in enumerate([64, 1024, 128])]
    clock = Clock()
    srv = Server(10 ** 12, lambda r: FakeSlot(r, clock), lambda r: 1, clock=clock,
                       sleep=clock.sleep)
    rep = srv.run(reqs)
    by = rep["latency_ms"]["by_class"]
    assert by["small"]["cycles"] == 4 and by["large"]["cycles"] == 2
    assert by["small"]["p99"] == by["small"]["p99"] and by["large"]["p50"] > 0
