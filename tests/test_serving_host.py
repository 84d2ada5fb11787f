"""Host logic of the continuous-batching server, on CPU, with a fake executor
that has the same slot/step interface as the GPU one.  Faults are injected on
the host: failing opens, a diverging request, a failing device step, an
injected check failure."""
import math

import numpy as np
import pytest

from paper_2408_06880_gb300 import _capi as A
from paper_2408_06880_gb300.serving import Request, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeDomain:
    def __init__(self, req):
        self.req = req
        self.nf = int(np.count_nonzero(req.flags == 0))
        self.t = 0
        self.closed = False


class FakeExecutor:
    """Mean velocity relaxes as U (1 - exp(-t / T)) with T from the request;
    'diverge' requests return NaN sums; 'bad' requests fail to open."""

    def __init__(self, capacity=4, clock=None, dt_per_step=1e-5):
        self.capacity = capacity
        self.slots = {}
        self.max_active = 0
        self.clock = clock
        self.dt = dt_per_step
        self.fail_step = False
        self.opened = []
        self.max_used = 0

    def footprint(self, req):
        return int(np.count_nonzero(req.flags == 0)) * 100

    def open(self, req):
        if req.meta.get("bad"):
            raise ValueError("invalid geometry")
        self.opened.append(req.rid)
        return FakeDomain(req)

    def add(self, dom):
        for s in range(self.capacity):
            if s not in self.slots:
                self.slots[s] = dom
                self.max_active = max(self.max_active, len(self.slots))
                self.max_used = max(self.max_used, sum(self.footprint(d.req) for d in self.slots.values()))
                return s
        raise RuntimeError("full")

    def remove(self, slot, dom):
        del self.slots[slot]
        dom.closed = True

    def step(self, k):
        if self.fail_step:
            self.fail_step = False
            raise A.SlbmError(A.ECUDA, "injected launch failure")
        for d in self.slots.values():
            d.t += k
        if self.clock is not None:
            self.clock.t += self.dt * k

    def sums(self):
        out = np.zeros((self.capacity, 5))
        for s, d in self.slots.items():
            T = d.req.meta.get("T", 500.0)
            m = 1e-3 * (1 - math.exp(-d.t / T))
            if d.req.meta.get("diverge") and d.t >= 200:
                m = float("nan")
            out[s, 4] = m * d.nf
        return out


def req(rid, n=8, arrival=0.0, **meta):
    flags = np.zeros((n, n, n), np.uint8)
    return Request(rid, flags, arrival=arrival, max_steps=20000, tol=1e-6, meta=meta)


def test_all_requests_solved_and_converge_when_expected():
    ex = FakeExecutor(capacity=3)
    reqs = [req(i, T=200.0 * (1 + i)) for i in range(7)]
    res, st = Server(ex, budget_bytes=10 ** 9, chunk=100).run(reqs, realtime=False)
    assert st["solved"] == 7 and st["failed"] == 0 and st["converged"] == 7
    assert ex.max_active == 3
    by = {r.rid: r for r in res}
    # the exponential model converges (rel. change over 100 steps < 1e-6) at
    # t ~ T ln(100/T * 1e6): later for slower requests
    assert by[0].steps < by[6].steps
    for r in res:
        T = 200.0 * (1 + r.rid)
        assert abs(r.mean_ux - 1e-3) < 1e-3 * 2e-5      # residual ~ (T/chunk) * tol
        assert r.steps == pytest.approx(T * math.log(1e6 * (math.exp(100 / T) - 1)), abs=200)


def test_results_do_not_depend_on_the_mix():
    alone = {}
    for i in range(5):
        res, _ = Server(FakeExecutor(1), 10 ** 9).run([req(i, T=150.0 + 70 * i)], realtime=False)
        alone[i] = res[0]
    res, _ = Server(FakeExecutor(3), 10 ** 9).run([req(i, T=150.0 + 70 * i) for i in range(5)], realtime=False)
    for r in res:
        assert r.steps == alone[r.rid].steps and r.permeability == alone[r.rid].permeability


def test_budget_limits_concurrency_and_lookahead_skips_a_big_head():
    ex = FakeExecutor(capacity=8)
    small0 = req(0, n=8)                          # 512 cells -> 51,200 bytes
    big = req(1, n=20)                            # 8000 cells -> 800,000 bytes
    small = [req(i, n=8) for i in range(2, 6)]
    budget = 840_000                              # big does not fit beside a small one
    res, st = Server(ex, budget_bytes=budget, lookahead=8).run([small0, big] + small, realtime=False)
    assert st["solved"] == 6
    assert ex.max_used <= budget
    # the big request waited; the small ones behind it were not blocked
    assert ex.opened == [0, 2, 3, 4, 5, 1]


def test_request_larger_than_budget_fails_alone():
    ex = FakeExecutor(capacity=2)
    res, st = Server(ex, budget_bytes=10_000).run([req(0, n=20), req(1, n=2)], realtime=False)
    by = {r.rid: r for r in res}
    assert by[0].error and "budget" in by[0].error
    assert by[1].error is None


def test_faults_are_isolated():
    ex = FakeExecutor(capacity=4)
    reqs = [req(0, bad=True), req(1, diverge=True), req(2), req(3), req(4)]
    res, st = Server(ex, budget_bytes=10 ** 9).run(reqs, realtime=False)
    by = {r.rid: r for r in res}
    assert "open failed" in by[0].error
    assert "diverged" in by[1].error
    assert all(by[i].error is None and by[i].converged for i in (2, 3, 4))
    assert not ex.slots                        # nothing left open


def test_failed_device_step_fails_active_requests_only():
    ex = FakeExecutor(capacity=2)
    clock = FakeClock()
    ex.clock = clock
    calls = {"n": 0}

    def hook(event, rid):
        if event == "step":
            calls["n"] += 1
            if calls["n"] == 3:
                ex.fail_step = True

    reqs = [req(0), req(1), req(2, arrival=0.5), req(3, arrival=0.6)]
    res, st = Server(ex, budget_bytes=10 ** 9, clock=clock, sleep=clock.sleep, fault_hook=hook).run(reqs, realtime=True)
    by = {r.rid: r for r in res}
    assert "step failed" in by[0].error and "step failed" in by[1].error
    assert by[2].error is None and by[3].error is None


def test_injected_check_fault_retires_one_request():
    ex = FakeExecutor(capacity=3)

    def hook(event, rid):
        if event == "check" and rid == 1:
            raise RuntimeError("host lost the request")

    res, st = Server(ex, budget_bytes=10 ** 9, fault_hook=hook).run([req(0), req(1), req(2)], realtime=False)
    by = {r.rid: r for r in res}
    assert "injected" in by[1].error
    assert by[0].error is None and by[2].error is None


def test_realtime_arrivals_and_latency_stats():
    clock = FakeClock()
    ex = FakeExecutor(capacity=2, clock=clock, dt_per_step=1e-4)
    reqs = [req(i, arrival=0.2 * i, T=100.0) for i in range(6)]
    res, st = Server(ex, budget_bytes=10 ** 9, clock=clock, sleep=clock.sleep).run(reqs, realtime=True)
    assert st["solved"] == 6
    for r in res:
        assert r.t_admit >= r.t_arrival - 1e-12
        assert r.latency > 0
    assert st["latency_p99_s"] >= st["latency_p50_s"] > 0


def test_chunk_must_be_even():
    with pytest.raises(ValueError):
        Server(FakeExecutor(), 1, chunk=7)


class FakeLaneExecutor(FakeExecutor):
    """Two lanes: requests below `small` cells advance `chunks` chunks per
    tick and report the sums after each; the others one chunk."""

    def __init__(self, capacity=4, small=600, chunks=4):
        super().__init__(capacity)
        self.small, self.chunks = small, chunks
        self.series = {}

    def _sums_of(self, d):
        T = d.req.meta.get("T", 500.0)
        return np.array([0, 0, 0, 0, 1e-3 * (1 - math.exp(-d.t / T)) * d.nf])

    def launch(self, k):
        self.series = {}
        for s, d in self.slots.items():
            n = self.chunks if d.nf < self.small else 1
            rows = []
            for _ in range(n):
                d.t += k
                rows.append(self._sums_of(d))
            self.series[s] = np.array(rows)

    def collect(self):
        return self.series


def test_lanes_keep_results_and_let_small_requests_finish_sooner():
    def reqs():
        return [req(0, n=12, T=900.0), req(1, n=8, T=300.0), req(2, n=12, T=700.0), req(3, n=8, T=500.0)]
    alone = {}
    for r in reqs():
        res, _ = Server(FakeExecutor(1), 10 ** 9).run([r], realtime=False)
        alone[r.rid] = res[0]
    clock = FakeClock()
    ex = FakeLaneExecutor(capacity=4, small=600, chunks=4)
    srv = Server(ex, 10 ** 9, clock=clock, sleep=clock.sleep)
    orig = ex.launch

    def timed_launch(k):
        orig(k)
        clock.t += 1.0                          # one tick = one unit of time
    ex.launch = timed_launch
    res, st = srv.run(reqs(), realtime=False)
    assert st["solved"] == 4
    by = {r.rid: r for r in res}
    for rid, r in by.items():                   # identical to a solve alone
        assert r.steps == alone[rid].steps and r.permeability == alone[rid].permeability
    # the 8^3 requests (512 cells) advance 4 chunks per tick: they retire after
    # a quarter of the ticks a lockstep server would need
    for rid in (1, 3):
        assert by[rid].t_finish <= math.ceil(by[rid].steps / 400) + 1


def test_lane_cap_bounds_concurrent_large_requests():
    class Capped(FakeLaneExecutor):
        def __init__(self):
            super().__init__(capacity=6, small=600, chunks=2)
            self.peak_large = 0

        def can_admit(self, r):
            large = sum(1 for d in self.slots.values() if d.nf >= self.small)
            return r.n_fluid < self.small or large < 2

        def launch(self, k):
            self.peak_large = max(self.peak_large, sum(1 for d in self.slots.values() if d.nf >= self.small))
            super().launch(k)

    ex = Capped()
    reqs = [req(i, n=12 if i % 2 else 8, T=300.0 + 40 * i) for i in range(8)]
    res, st = Server(ex, 10 ** 9).run(reqs, realtime=False)
    assert st["solved"] == 8
    assert ex.peak_large == 2
