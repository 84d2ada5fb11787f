"""Continuous-batching server for permeability solves.

Requests (voxel geometries with a body force) arrive over time.  The server
admits a request as soon as a pool slot and enough HBM budget are free, keeps
its PDF-list and index-list resident, steps every admitted request together
(one persistent kernel launch per time step through `Pool`, CUDA-graph replay
of `chunk` steps), checks each request's convergence after every chunk from
its FP64 domain sums, and retires it -- freeing its slot and memory for the
next arrival -- when the relative change of its mean fluid velocity over the
last chunk drops below `tol`, or at `max_steps`.  A request whose sums stop
being finite, or whose mean speed exceeds the stability bound, is retired
with an error while the others keep running.

The loop talks to an executor (`GpuExecutor` here; tests use a CPU fake with
the same interface), so admission, batching and retirement are host logic
independent of the device.  Permeability (lattice units^2) of a body-force
driven periodic sample: k = nu * U_D / F_x with U_D = sum_fluid u_x / N.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import _capi as A

U_MAX_STABLE = 0.3


@dataclass
class Request:
    rid: int
    flags: np.ndarray
    periodic: int = 7
    force: tuple = (1e-6, 0.0, 0.0)
    omega: float = 1.0 / 0.8
    trt_magic: float = 3.0 / 16.0
    arrival: float = 0.0                 # seconds after the start of the run
    max_steps: int = 20000
    tol: float = 1e-6
    meta: dict = field(default_factory=dict)
    _nf: int | None = field(default=None, repr=False, compare=False)

    @property
    def n_fluid(self) -> int:
        """Fluid voxels of the geometry (counted once)."""
        if self._nf is None:
            self._nf = int(np.count_nonzero(self.flags == 0))
        return self._nf


@dataclass
class Result:
    rid: int
    permeability: float | None
    steps: int
    converged: bool
    t_arrival: float
    t_admit: float | None
    t_finish: float
    error: str | None = None
    mean_ux: float | None = None

    @property
    def latency(self) -> float:
        return self.t_finish - self.t_arrival


def nu_of(omega: float) -> float:
    return (1.0 / omega - 0.5) / 3.0


class GpuExecutor:
    """Pool-backed executor: one `Domain` per admitted request, stepped by
    pools.  With `lanes` = ((max_cells, chunks[, cap]), ..., (None, chunks[,
    cap])), a
    request goes to the first lane whose max_cells exceeds its fluid cells;
    each lane is a pool on its own stream, and per server tick lane l
    advances its members `chunks` chunks, reducing their FP64 sums on the
    device after each one (no host wait in between), while the lanes run
    concurrently.  Small requests then progress several chunks for one of the
    large ones -- a fairer share of GPU time than lockstep -- and the server
    still tests convergence after every chunk, so results and step counts are
    those of a solve alone.  `cap` bounds a lane's concurrent members (the
    server leaves a request queued while its lane is full)."""

    def __init__(self, q: int = 19, storage: int = A.FP32, capacity: int = 64, scale_exp: int | None = None,
                 graph: bool = True, stream=None, pool_launch: tuple | None = None,
                 group_bytes: int | None = None, streams: int = 2, lanes: tuple | None = None):
        import torch
        from .domain import Domain, auto_scale_exp
        from .pool import Pool
        self._torch = torch
        self._Domain = Domain
        self.q, self.storage, self.graph = q, storage, graph
        self.scale_exp = auto_scale_exp(1e-3) if scale_exp is None else scale_exp
        self.stream = stream
        self.capacity = capacity
        spec = tuple(lanes) if lanes else ((None, 1),)
        self.lanes = []
        for entry in spec:
            max_cells, chunks = entry[0], entry[1]
            cap = entry[2] if len(entry) > 2 and entry[2] else capacity
            st = stream if len(spec) == 1 else torch.cuda.Stream()
            pool = Pool(q, storage, capacity, stream=st)
            if pool_launch:
                pool.set_launch(*pool_launch)
            if group_bytes is not None:
                pool.set_group_bytes(group_bytes)
            if streams > 1:
                pool.set_streams(streams)
            self.lanes.append(dict(max=max_cells, chunks=int(chunks), cap=int(cap), pool=pool, stream=st,
                                   slots=set(), buf=None))
        self.pool = self.lanes[0]["pool"]
        if len(self.lanes) > 1:            # the server drives lanes through launch/collect
            self.launch = self._launch
            self.collect = self._collect

    def footprint(self, req: Request) -> int:
        """Device bytes a request will hold (PDF-list, index-list, cell list,
        reduction partials), from its fluid-cell count."""
        nf = req.n_fluid
        S = (nf + 127) // 128 * 128
        b = 4 if self.storage == A.FP32 else 2
        return self.q * S * b + (self.q - 1) * S * 4 + nf * 4 + ((nf + 2047) // 2048) * 40 + 1024

    def open(self, req: Request):
        return self._Domain(req.flags, periodic=req.periodic, q=self.q, op=A.TRT, omega=req.omega,
                            trt_magic=req.trt_magic, force=req.force, storage=self.storage,
                            scale_exp=self.scale_exp, stream=self.stream)

    def _lane_of(self, nf: int) -> int:
        for li, lane in enumerate(self.lanes):
            if lane["max"] is None or nf < lane["max"]:
                return li
        raise ValueError("no lane takes this request")

    def can_admit(self, req: Request) -> bool:
        """The request's lane has room (at most `cap` active members)."""
        lane = self.lanes[self._lane_of(req.n_fluid)]
        return len(lane["slots"]) < lane["cap"]

    def add(self, dom) -> int:
        li = self._lane_of(dom.n_fluid)
        lane = self.lanes[li]
        s = lane["pool"].add(dom)
        lane["slots"].add(s)
        return li * self.capacity + s

    def remove(self, slot: int, dom) -> None:
        li, s = divmod(slot, self.capacity)
        self.lanes[li]["pool"].remove(s)
        self.lanes[li]["slots"].discard(s)
        dom.close()

    def step(self, k: int) -> None:
        for lane in self.lanes:
            if lane["slots"]:
                lane["pool"].step(k, graph=self.graph)

    def sums(self) -> np.ndarray:
        out = np.zeros((self.capacity * len(self.lanes), 5))
        for li, lane in enumerate(self.lanes):
            out[li * self.capacity:(li + 1) * self.capacity] = lane["pool"].reduce()
        return out

    def _launch(self, k: int) -> None:
        torch = self._torch
        for lane in self.lanes:
            if not lane["slots"]:
                continue
            if lane["buf"] is None:
                # filled by the pool's reductions (which clear their output) on the lane's stream
                lane["buf"] = torch.empty((lane["chunks"], self.capacity, 5), dtype=torch.float64, device="cuda")
            for j in range(lane["chunks"]):
                lane["pool"].step(k, graph=self.graph)
                lane["pool"].reduce_device(lane["buf"][j])

    def _collect(self) -> dict:
        out = {}
        for li, lane in enumerate(self.lanes):
            if not lane["slots"]:
                continue
            lane["stream"].synchronize()
            arr = lane["buf"].cpu().numpy()
            for s in lane["slots"]:
                out[li * self.capacity + s] = arr[:, s, :]
        return out

    def close(self) -> None:
        for lane in self.lanes:
            lane["pool"].close()


class Server:
    """Continuous batching over an executor.  `run()` serves a list of
    requests with given arrival times and returns their results plus run
    statistics (solves/s, p50/p99 latency)."""

    def __init__(self, executor, budget_bytes: int, chunk: int = 100, lookahead: int = 8,
                 clock=time.perf_counter, sleep=time.sleep, fault_hook=None):
        if chunk <= 0 or chunk % 2:
            raise ValueError("chunk must be a positive even number of steps")
        self.ex = executor
        self.budget = int(budget_bytes)
        self.chunk = chunk
        self.lookahead = lookahead
        self.clock = clock
        self.sleep = sleep
        self.fault_hook = fault_hook      # tests: called as hook(event, rid) -> raise to inject

    def run(self, requests: list[Request], realtime: bool = True) -> tuple[list[Result], dict]:
        queue = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = self.clock()
        active: dict[int, dict] = {}      # slot -> state
        results: list[Result] = []
        used = 0
        busy_s = 0.0
        updates = 0

        def admit(fresh: bool) -> None:
            """FIFO admission with bounded lookahead, by slot and budget.
            fresh: a chunk is in flight that the new requests are not part of."""
            nonlocal used
            now = self.clock() - t0
            i = 0
            while i < min(len(queue), self.lookahead) and len(active) < self.ex.capacity:
                req = queue[i]
                if realtime and req.arrival > now:
                    break
                need = self.ex.footprint(req)
                if need > self.budget:
                    queue.pop(i)
                    results.append(Result(req.rid, None, 0, False, req.arrival, None, self.clock() - t0,
                                          error="footprint exceeds the whole HBM budget"))
                    continue
                if used + need > self.budget or (hasattr(self.ex, "can_admit") and not self.ex.can_admit(req)):
                    i += 1
                    continue
                queue.pop(i)
                try:
                    if self.fault_hook:
                        self.fault_hook("open", req.rid)
                    dom = self.ex.open(req)
                    slot = self.ex.add(dom)
                except Exception as e:  # creation failure: report, keep serving
                    results.append(Result(req.rid, None, 0, False, req.arrival, None, self.clock() - t0,
                                          error=f"open failed: {e}"))
                    continue
                active[slot] = dict(req=req, dom=dom, need=need, steps=0, prev=None, fresh=fresh,
                                    t_admit=self.clock() - t0, n=int(req.flags.size), nf=req.n_fluid)
                used += need

        while queue or active:
            # Requests are opened while a chunk runs on the device (below);
            # here only when nothing runs, or when arrivals are timed and a
            # newcomer should not wait for the next chunk.
            if not active or realtime:
                admit(False)
            if not active:
                if queue and realtime:
                    wait = queue[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, 0.05))
                continue
            # ---- one chunk of steps for every active request (an executor
            # with lanes may advance some requests several chunks, reporting
            # the sums after each one)
            tb = self.clock()
            try:
                if self.fault_hook:
                    self.fault_hook("step", None)
                lanes = hasattr(self.ex, "launch")
                if lanes:
                    self.ex.launch(self.chunk)
                else:
                    self.ex.step(self.chunk)
                admit(True)                   # overlaps the chunk in flight
                if lanes:
                    series = self.ex.collect()
                else:
                    sums = self.ex.sums()
                    series = {slot: sums[slot][None, :] for slot in active}
            except A.SlbmError as e:
                # a device-level failure ends every active request
                for slot, st in list(active.items()):
                    results.append(self._retire(slot, st, t0, error=f"step failed: {e}"))
                    used -= st["need"]
                active.clear()
                continue
            busy_s += self.clock() - tb
            for slot, st in list(active.items()):
                if st["fresh"]:               # joined after this chunk was launched
                    st["fresh"] = False
                    continue
                for s in series[slot]:        # the sums after each chunk, in order
                    st["steps"] += self.chunk
                    updates += st["nf"] * self.chunk
                    done, err, conv = self._check(st, s)
                    if done:
                        results.append(self._retire(slot, st, t0, error=err, converged=conv, sums=s))
                        used -= st["need"]
                        del active[slot]
                        break
        wall = self.clock() - t0
        return results, self.stats(results, wall, busy_s, updates)

    def _check(self, st, s) -> tuple[bool, str | None, bool]:
        """Convergence / divergence test of one request after one chunk:
        (done, error, converged)."""
        req = st["req"]
        err = None
        mean_ux = s[4] / max(st["nf"], 1)
        if not np.all(np.isfinite(s)):
            err = "diverged: domain sums are not finite"
        elif abs(mean_ux) > U_MAX_STABLE:
            err = "diverged: mean speed above the stability bound"
        if self.fault_hook:
            try:
                self.fault_hook("check", req.rid)
            except Exception as e:
                err = f"injected: {e}"
        if err is not None:
            return True, err, False
        prev = st["prev"]
        st["prev"] = mean_ux
        if prev is not None and mean_ux != 0.0 and abs(mean_ux - prev) / abs(mean_ux) < req.tol:
            return True, None, True
        return st["steps"] >= req.max_steps, None, False

    def _retire(self, slot, st, t0, error=None, converged=False, sums=None):
        req = st["req"]
        k = mean_ux = None
        if error is None and sums is not None:
            mean_ux = sums[4] / max(st["nf"], 1)
            k = nu_of(req.omega) * (sums[4] / st["n"]) / req.force[0] if req.force[0] else None
        try:
            self.ex.remove(slot, st["dom"])
        except Exception:
            pass
        return Result(req.rid, k, st["steps"], converged, req.arrival, st["t_admit"], self.clock() - t0,
                      error=error, mean_ux=mean_ux)

    @staticmethod
    def stats(results: list[Result], wall: float, busy_s: float = 0.0, updates: int = 0) -> dict:
        ok = [r for r in results if r.error is None]
        lat = np.array([r.latency for r in ok]) if ok else np.array([math.nan])
        return {"requests": len(results), "solved": len(ok), "failed": len(results) - len(ok),
                "wall_s": wall, "solves_per_s": len(ok) / wall if wall > 0 else math.nan,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "latency_mean_s": float(np.mean(lat)),
                "mflups": updates / wall / 1e6 if wall > 0 else math.nan, "device_busy_s": busy_s,
                "converged": sum(r.converged for r in ok)}


def serve_replicas(executor, requests: list[Request], budget_bytes: int, realtime: bool = False,
                   chunk: int = 100, **server_kw) -> tuple[list[Result], dict]:
    """Serve a request stream over all ranks of the process group (one GPU
    each, no exchange on the data path): request i goes to rank i mod world,
    each rank serves its share with its own executor, and rank 0 gets every
    result plus the whole-job statistics -- solves over the slowest rank's
    wall time, latency percentiles over all requests.  Other ranks get their
    own results and local statistics.  Collective: every rank must call it."""
    from . import replicas
    mine = replicas.shard(requests)
    res, st = Server(executor, budget_bytes, chunk=chunk, **server_kw).run(mine, realtime=realtime)
    upd_local = st["mflups"] * 1e6 * st["wall_s"] if st["wall_s"] > 0 else 0.0
    _, updates, wall = replicas.job_rate(upd_local, st["wall_s"])
    _, busy_sum, _ = replicas.job_rate(st["device_busy_s"], st["wall_s"])
    parts = replicas.gather(res)
    if parts is None:
        return res, st
    allres = [r for part in parts for r in part]
    merged = Server.stats(allres, wall, busy_sum, int(round(updates)))
    merged["ranks"] = len(parts)
    return allres, merged


def solve_alone(req: Request, q: int = 19, storage: int = A.FP32, chunk: int = 100, graph: bool = True,
                scale_exp: int | None = None, stream=None) -> Result:
    """One request on its own (no pool): the one-at-a-time baseline, with the
    same convergence test and the same kernels as the server."""
    from .domain import Domain, auto_scale_exp
    se = auto_scale_exp(1e-3) if scale_exp is None else scale_exp
    t0 = time.perf_counter()
    d = Domain(req.flags, periodic=req.periodic, q=q, op=A.TRT, omega=req.omega, trt_magic=req.trt_magic,
               force=req.force, storage=storage, scale_exp=se, stream=stream)
    n, nf = int(req.flags.size), d.n_fluid
    prev, steps, conv, s = None, 0, False, None
    try:
        while steps < req.max_steps:
            d.step(chunk, graph=graph)
            steps += chunk
            s = d.reduce()
            m = s[4] / max(nf, 1)
            if prev is not None and m != 0.0 and abs(m - prev) / abs(m) < req.tol:
                conv = True
                break
            prev = m
    finally:
        d.close()
    k = nu_of(req.omega) * (s[4] / n) / req.force[0]
    return Result(req.rid, k, steps, conv, 0.0, 0.0, time.perf_counter() - t0, mean_ux=s[4] / max(nf, 1))
