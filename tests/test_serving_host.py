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


# ------------------------------------------------------ reduced precision
from paper_2408_06880_gb300.serving import Precision, Track  # noqa: E402


class FakeMixedExecutor(FakeExecutor):
    """16-bit requests relax like FP32 ones until the relative error of the
    mean velocity reaches `floor`, where they stall (the rounding of small
    changes); after a conversion to FP32 they relax to the steady state from
    where they stood.  Sums carry the two maxima of reduce_ext (max|g| grows
    with the velocity; max|u| is 10 x the mean)."""

    def __init__(self, capacity=4, floor=2e-3, gscale=0.05, chunks=None):
        super().__init__(capacity)
        self.storage, self.scale_exp, self.precision = A.FP16, 24, Precision()
        self.floor, self.gscale = floor, gscale
        self.converted = []          # (rid, step, storage, scale)
        self.chunks = chunks
        if chunks is not None:
            self.launch, self.collect = self._launch, self._collect

    def open(self, req):
        d = super().open(req)
        d.storage, d.scale, d.t16, d.m0 = A.FP16, 24, None, 0.0
        return d

    def _mean(self, d):
        U = 1e-3
        T = d.req.meta.get("T", 500.0)
        if d.storage != A.FP32:
            return U * (1 - max(math.exp(-d.t / T), self.floor))
        return U - (U - d.m0) * math.exp(-(d.t - d.t16) / T)

    def _row(self, d):
        m = self._mean(d)
        return np.array([0, 0, 0, 0, m * d.nf, self.gscale * m, 10 * m])

    def sums(self):
        out = np.zeros((self.capacity, 7))
        for s, d in self.slots.items():
            out[s] = self._row(d)
        return out

    def _launch(self, k):
        self.series = {}
        for s, d in self.slots.items():
            rows = []
            for _ in range(self.chunks):
                d.t += k
                rows.append(self._row(d))
            self.series[s] = np.array(rows)

    def _collect(self):
        return self.series

    def convert(self, slot, dom, storage, scale):
        if storage == A.FP32 and dom.storage != A.FP32:
            dom.m0, dom.t16 = self._mean(dom), dom.t
        dom.storage, dom.scale = storage, scale
        self.converted.append((dom.req.rid, dom.t, storage, scale))
        return slot


def test_precision_plan_hands_off_to_fp32_and_converges():
    ex = FakeMixedExecutor(capacity=3)
    reqs = [req(i, T=300.0 + 100 * i) for i in range(5)]
    res, st = Server(ex, budget_bytes=10 ** 9, chunk=100).run(reqs, realtime=False)
    assert st["solved"] == 5 and st["converged"] == 5
    handoffs = {rid: t for rid, t, s, _ in ex.converted if s == A.FP32}
    for r in res:
        assert r.rid in handoffs
        assert 0 < r.low_steps == handoffs[r.rid] < r.steps       # 16-bit phase first, then FP32
        assert abs(r.mean_ux / 1e-3 - 1) < 1e-4                   # converged in FP32, past the 16-bit floor
    assert 0 < st["low_precision_step_share"] < 1


def test_precision_changes_take_effect_at_tick_ends():
    ex = FakeMixedExecutor(capacity=4, chunks=3)
    reqs = [req(i, T=400.0 + 50 * i) for i in range(4)]
    res, st = Server(ex, budget_bytes=10 ** 9, chunk=100).run(reqs, realtime=False)
    assert st["solved"] == 4
    for rid, t, storage, _ in ex.converted:
        assert t % 300 == 0                        # after whole ticks of 3 chunks of 100 steps


def test_rescale_keeps_the_stored_maximum_in_band():
    p = Precision()
    assert p.rescale_to(24, 1e-4) is None                       # 1e-4 * 2^24 = 1678: inside [2^10, 2^14.5]
    s = p.rescale_to(24, 2e-3)                                  # 33554 > 2^14.5
    assert s is not None and 2 ** 12 < 2e-3 * 2.0 ** s <= 2 ** 13
    s = p.rescale_to(24, 1e-6)                                  # 16.8 < 2^10
    assert s is not None and 2 ** 12 < 1e-6 * 2.0 ** s <= 2 ** 13
    assert p.rescale_to(24, float("nan")) is None and p.rescale_to(24, 0.0) is None
    assert p.rescale_to(0, 1e30) == -40                         # clamped to the format's exponent range


def test_track_rescale_pending_and_handoff_override():
    r = req(0)
    tr = Track(r, r.n_fluid, A.FP16, 24, Precision())
    nf = r.n_fluid
    tr.check(np.array([0, 0, 0, 0, 1e-4 * nf, 5e-3, 1e-3]), 100)        # max|h| = 5e-3 * 2^24 > 2^14.5
    assert tr.pending is not None and tr.pending[0] == A.FP16 and tr.pending[1] < 24
    tr.check(np.array([0, 0, 0, 0, 1.00001e-4 * nf, 5e-3, 1e-3]), 100)  # rel change 1e-5 < 3e-3
    assert tr.pending == (A.FP32, 0)
    tr.switched()
    assert tr.storage == A.FP32 and tr.precision is None and tr.low_steps == 200


def test_track_divergence_from_the_largest_speed():
    r = req(0)
    tr = Track(r, r.n_fluid)
    done, err, conv = tr.check(np.array([0, 0, 0, 0, 1e-4 * r.n_fluid, 1e-3, 0.31]), 100)
    assert done and "speed" in err and not conv
