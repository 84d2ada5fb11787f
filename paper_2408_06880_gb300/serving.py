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

Reduced-precision solves (FP16/BF16 storage, `Precision`): the stored
populations of a body-forced solve track the FP32 ones through the early
transient, then stall about 1e-4..1e-2 short of the steady state, because near
it the per-step changes of a population fall below half a unit in the last
place of the 16-bit format and round away; the relative change of the mean
velocity per 100 steps then settles at 3e-7..8e-6 instead of reaching the
1e-6 criterion.  So a reduced-precision request runs in 16 bits while the
relative change per chunk is above `handoff_rel`, then its populations are
converted exactly to FP32 (`Domain.set_storage`) and the solve continues in
FP32 until the criterion holds: every result is an FP32-converged solve.
While in 16 bits, the largest stored magnitude (from the device maximum
reduction) keeps the power-of-two storage scale in a band, rescaling exactly
when it drifts out.  Conversions and rescales take effect at the end of the
request's tick (its lane's chunks per tick), so a request served in a mix and
the same request solved alone take them at the same step.

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
    low_steps: int = 0              # steps taken in 16-bit storage before the FP32 phase

    @property
    def latency(self) -> float:
        return self.t_finish - self.t_arrival


def nu_of(omega: float) -> float:
    return (1.0 / omega - 0.5) / 3.0


@dataclass
class Precision:
    """Storage plan of a reduced-precision (FP16/BF16) solve.

    handoff_rel: convert to FP32 once the relative change of the mean fluid
      u_x over one chunk falls below this (the 16-bit state still follows the
      FP32 trajectory there); the FP32 phase then runs to the request's own
      tolerance.
    h_lo, h_hi, h_target: while in 16 bits, when the largest stored magnitude
      max|f_i - w_i| * 2^s leaves [h_lo, h_hi], the scale exponent s is
      re-chosen so that it maps to about h_target (an exact power-of-two
      rescale of every stored value)."""

    handoff_rel: float = 3e-3
    h_lo: float = 2.0 ** 10
    h_hi: float = 2.0 ** 14.5
    h_target: float = 2.0 ** 13

    def rescale_to(self, scale_exp: int, gmax: float) -> int | None:
        """New scale exponent for the largest unscaled magnitude gmax, or None
        if the current one keeps it inside the band."""
        if not (gmax > 0.0) or not math.isfinite(gmax):
            return None
        if self.h_lo <= gmax * 2.0 ** scale_exp <= self.h_hi:
            return None
        s = max(-40, min(40, int(math.floor(math.log2(self.h_target / gmax)))))
        return None if s == scale_exp else s


class Track:
    """Convergence and storage bookkeeping of one solve, fed the domain sums
    after every chunk: [sum(rho-1), sum rho u (3), sum u_x] and optionally
    max|f_i - w_i| and max|u| (sparse_lbm_reduce_ext).  The server and
    `solve_alone` both use it, so they take the same decisions."""

    def __init__(self, req: Request, nf: int, storage: int = A.FP32, scale_exp: int = 0,
                 precision: Precision | None = None):
        self.req, self.nf = req, nf
        self.storage, self.scale_exp = storage, scale_exp
        self.precision = precision if storage != A.FP32 else None
        self.steps = 0
        self.low_steps = 0          # steps taken in 16-bit storage
        self.prev = None
        self.pending = None         # (storage, scale_exp) to switch to at the end of the tick

    def check(self, s, chunk: int) -> tuple[bool, str | None, bool]:
        """Account one chunk and test it: (done, error, converged)."""
        self.steps += chunk
        if self.storage != A.FP32:
            self.low_steps += chunk
        mean_ux = s[4] / max(self.nf, 1)
        if not np.all(np.isfinite(s)):
            return True, "diverged: domain sums are not finite", False
        if abs(mean_ux) > U_MAX_STABLE or (len(s) > 6 and s[6] > U_MAX_STABLE):
            return True, "diverged: a cell's speed exceeds the stability bound", False
        prev, self.prev = self.prev, mean_ux
        rel = abs(mean_ux - prev) / abs(mean_ux) if prev is not None and mean_ux != 0.0 else None
        if self.precision is not None and self.storage != A.FP32:
            if rel is not None and rel < self.precision.handoff_rel:
                self.pending = (A.FP32, 0)
            elif len(s) > 5 and (self.pending is None or self.pending[0] != A.FP32):
                ns = self.precision.rescale_to(self.scale_exp, float(s[5]))
                if ns is not None:
                    self.pending = (self.storage, ns)
            return self.steps >= self.req.max_steps, None, False
        if rel is not None and rel < self.req.tol:
            return True, None, True
        return self.steps >= self.req.max_steps, None, False

    def switched(self) -> None:
        """The pending storage change was applied."""
        self.storage, self.scale_exp = self.pending
        if self.storage == A.FP32:
            self.precision = None
        self.pending = None


class GpuExecutor:
    """Pool-backed executor: one `Domain` per admitted request, stepped by
    pools.  With `lanes` = ((max_cells, chunks[, cap]), ..., (None, chunks[,
    cap])), a request goes to the first lane whose max_cells exceeds its fluid
    cells; each lane has its own stream, and per server tick lane l advances
    its members `chunks` chunks, reducing their FP64 sums (and the two maxima
    of sparse_lbm_reduce_ext) on the device after each one (no host wait in
    between), while the lanes run concurrently.  Small requests then progress
    several chunks for one of the large ones -- a fairer share of GPU time
    than lockstep -- and the server still tests convergence after every chunk,
    so results and step counts are those of a solve alone.  `cap` bounds a
    lane's concurrent members (the server leaves a request queued while its
    lane is full).

    With a 16-bit `storage` and a `precision` plan, every lane holds two
    pools, one per storage: a request starts in the 16-bit pool and moves to
    the FP32 pool of its lane when the plan hands it off (`convert`).  Its
    HBM footprint is then counted at FP32 from admission on."""

    def __init__(self, q: int = 19, storage: int = A.FP32, capacity: int = 64, scale_exp: int | None = None,
                 graph: bool = True, stream=None, pool_launch: tuple | None = None,
                 group_bytes: int | None = None, streams: int = 2, lanes: tuple | None = None,
                 precision: Precision | None = None):
        import torch
        from .domain import Domain, auto_scale_exp
        from .pool import Pool
        self._torch = torch
        self._Domain = Domain
        self.q, self.storage, self.graph = q, storage, graph
        self.scale_exp = auto_scale_exp(1e-3) if scale_exp is None else scale_exp
        self.precision = precision if storage != A.FP32 else None
        self.kinds = [storage] + ([A.FP32] if self.precision is not None else [])
        self.stream = stream
        self.capacity = capacity
        spec = tuple(lanes) if lanes else ((None, 1),)
        self.lanes = []
        for entry in spec:
            max_cells, chunks = entry[0], entry[1]
            cap = entry[2] if len(entry) > 2 and entry[2] else capacity
            st = stream if len(spec) == 1 else torch.cuda.Stream()
            pools = []
            for kind in self.kinds:
                pool = Pool(q, kind, capacity, stream=st)
                if pool_launch:
                    pool.set_launch(*pool_launch)
                if group_bytes is not None:
                    pool.set_group_bytes(group_bytes)
                if streams > 1:
                    pool.set_streams(streams)
                pools.append(pool)
            self.lanes.append(dict(max=max_cells, chunks=int(chunks), cap=int(cap), pools=pools, stream=st,
                                   slots=set(), buf=[None] * len(pools)))
        self.pool = self.lanes[0]["pools"][0]
        if len(self.lanes) > 1:            # the server drives lanes through launch/collect
            self.launch = self._launch
            self.collect = self._collect

    # slot ids: ((lane * kinds) + pool) * capacity + pool slot
    def _sid(self, li: int, pi: int, s: int) -> int:
        return (li * len(self.kinds) + pi) * self.capacity + s

    def _split(self, sid: int) -> tuple[int, int, int]:
        lp, s = divmod(sid, self.capacity)
        li, pi = divmod(lp, len(self.kinds))
        return li, pi, s

    def footprint(self, req: Request) -> int:
        """Device bytes a request will hold (PDF-list, index-list, cell list,
        reduction partials), from its fluid-cell count; at FP32 when a
        16-bit request may be handed off."""
        nf = req.n_fluid
        S = (nf + 127) // 128 * 128
        b = 2 if self.storage != A.FP32 and self.precision is None else 4
        return self.q * S * b + (self.q - 1) * S * 4 + nf * 4 + ((nf + 2047) // 2048) * 48 + 1024

    def open(self, req: Request):
        return self._Domain(req.flags, periodic=req.periodic, q=self.q, op=A.TRT, omega=req.omega,
                            trt_magic=req.trt_magic, force=req.force, storage=self.storage,
                            scale_exp=self.scale_exp, stream=self.stream)

    def _lane_of(self, nf: int) -> int:
        for li, lane in enumerate(self.lanes):
            if lane["max"] is None or nf < lane["max"]:
                return li
        raise ValueError("no lane takes this request")

    def tick_chunks(self, req: Request) -> int:
        """Chunks a request advances per server tick (its lane's)."""
        return self.lanes[self._lane_of(req.n_fluid)]["chunks"] if len(self.lanes) > 1 else 1

    def can_admit(self, req: Request) -> bool:
        """The request's lane has room (at most `cap` active members)."""
        lane = self.lanes[self._lane_of(req.n_fluid)]
        return len(lane["slots"]) < lane["cap"]

    def add(self, dom) -> int:
        li = self._lane_of(dom.n_fluid)
        lane = self.lanes[li]
        pi = self.kinds.index(dom.params["storage"])
        s = lane["pools"][pi].add(dom)
        lane["slots"].add((pi, s))
        return self._sid(li, pi, s)

    def remove(self, slot: int, dom) -> None:
        li, pi, s = self._split(slot)
        self.lanes[li]["pools"][pi].remove(s)
        self.lanes[li]["slots"].discard((pi, s))
        dom.close()

    def convert(self, slot: int, dom, storage: int, scale_exp: int) -> int:
        """Change a member's storage (hand-off to FP32 or a rescale): it
        leaves its pool, its populations are converted in place, and it joins
        its lane's pool of the new storage.  Returns its new slot id."""
        li, pi, s = self._split(slot)
        lane = self.lanes[li]
        lane["pools"][pi].remove(s)
        lane["slots"].discard((pi, s))
        dom.set_storage(storage, scale_exp)
        pj = self.kinds.index(storage)
        s2 = lane["pools"][pj].add(dom)
        lane["slots"].add((pj, s2))
        return self._sid(li, pj, s2)

    def step(self, k: int) -> None:
        for lane in self.lanes:
            for pool in lane["pools"]:
                if pool.members:
                    pool.step(k, graph=self.graph)

    def sums(self) -> np.ndarray:
        out = np.zeros((self.capacity * len(self.kinds) * len(self.lanes), 7))
        for li, lane in enumerate(self.lanes):
            for pi, pool in enumerate(lane["pools"]):
                if pool.members:
                    b = self._sid(li, pi, 0)
                    out[b:b + self.capacity] = pool.reduce_ext()
        return out

    def _launch(self, k: int) -> None:
        torch = self._torch
        for lane in self.lanes:
            if not lane["slots"]:
                continue
            for pi, pool in enumerate(lane["pools"]):
                if lane["buf"][pi] is None:
                    # filled by the pool's reductions (which clear their output) on the lane's stream
                    lane["buf"][pi] = torch.empty((lane["chunks"], self.capacity, 7), dtype=torch.float64,
                                                  device="cuda")
            for j in range(lane["chunks"]):
                for pi, pool in enumerate(lane["pools"]):
                    if pool.members:
                        pool.step(k, graph=self.graph)
                        pool.reduce_ext_device(lane["buf"][pi][j])

    def _collect(self) -> dict:
        out = {}
        for li, lane in enumerate(self.lanes):
            if not lane["slots"]:
                continue
            lane["stream"].synchronize()
            arrs = {}
            for pi, s in lane["slots"]:
                if pi not in arrs:
                    arrs[pi] = lane["buf"][pi].cpu().numpy()
                out[self._sid(li, pi, s)] = arrs[pi][:, s, :]
        return out

    def close(self) -> None:
        for lane in self.lanes:
            for pool in lane["pools"]:
                pool.close()


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

    def _track(self, req: Request) -> Track:
        return Track(req, req.n_fluid, getattr(self.ex, "storage", A.FP32), getattr(self.ex, "scale_exp", 0),
                     getattr(self.ex, "precision", None))

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
                active[slot] = dict(req=req, dom=dom, need=need, track=self._track(req), fresh=fresh,
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
                retired = False
                for s in series[slot]:        # the sums after each chunk, in order
                    updates += st["nf"] * self.chunk
                    done, err, conv = self._check(st, s)
                    if done:
                        results.append(self._retire(slot, st, t0, error=err, converged=conv, sums=s))
                        used -= st["need"]
                        del active[slot]
                        retired = True
                        break
                tr = st["track"]
                if not retired and tr.pending is not None:
                    # the end of this request's tick: change its storage
                    try:
                        new_slot = self.ex.convert(slot, st["dom"], *tr.pending)
                    except Exception as e:
                        results.append(self._retire(slot, st, t0, error=f"storage change failed: {e}"))
                        used -= st["need"]
                        del active[slot]
                        continue
                    tr.switched()
                    del active[slot]
                    active[new_slot] = st
        wall = self.clock() - t0
        return results, self.stats(results, wall, busy_s, updates)

    def _check(self, st, s) -> tuple[bool, str | None, bool]:
        """Convergence / divergence test of one request after one chunk:
        (done, error, converged)."""
        done, err, conv = st["track"].check(s, self.chunk)
        if self.fault_hook and err is None:
            try:
                self.fault_hook("check", st["req"].rid)
            except Exception as e:
                return True, f"injected: {e}", False
        return done, err, conv

    def _retire(self, slot, st, t0, error=None, converged=False, sums=None):
        req = st["req"]
        tr = st["track"]
        k = mean_ux = None
        if error is None and sums is not None:
            mean_ux = sums[4] / max(st["nf"], 1)
            k = nu_of(req.omega) * (sums[4] / st["n"]) / req.force[0] if req.force[0] else None
        try:
            self.ex.remove(slot, st["dom"])
        except Exception:
            pass
        return Result(req.rid, k, tr.steps, converged, req.arrival, st["t_admit"], self.clock() - t0,
                      error=error, mean_ux=mean_ux, low_steps=tr.low_steps)

    @staticmethod
    def stats(results: list[Result], wall: float, busy_s: float = 0.0, updates: int = 0) -> dict:
        ok = [r for r in results if r.error is None]
        lat = np.array([r.latency for r in ok]) if ok else np.array([math.nan])
        return {"requests": len(results), "solved": len(ok), "failed": len(results) - len(ok),
                "wall_s": wall, "solves_per_s": len(ok) / wall if wall > 0 else math.nan,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "latency_mean_s": float(np.mean(lat)),
                "mflups": updates / wall / 1e6 if wall > 0 else math.nan, "device_busy_s": busy_s,
                "converged": sum(r.converged for r in ok),
                "low_precision_step_share": (sum(r.low_steps for r in ok) / max(sum(r.steps for r in ok), 1))}


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
                scale_exp: int | None = None, stream=None, precision: Precision | None = None,
                tick: int = 1) -> Result:
    """One request on its own (no pool): the one-at-a-time baseline, with the
    same convergence test, the same storage plan and the same kernels as the
    server.  `tick`: chunks per server tick of the lane the request would be
    served in (storage changes take effect at tick ends, as in the server)."""
    from .domain import Domain, auto_scale_exp
    se = auto_scale_exp(1e-3) if scale_exp is None else scale_exp
    t0 = time.perf_counter()
    d = Domain(req.flags, periodic=req.periodic, q=q, op=A.TRT, omega=req.omega, trt_magic=req.trt_magic,
               force=req.force, storage=storage, scale_exp=se, stream=stream)
    n, nf = int(req.flags.size), d.n_fluid
    tr = Track(req, nf, storage, d.params["scale_exp"], precision)
    conv, err, s, chunks = False, None, None, 0
    try:
        while True:
            d.step(chunk, graph=graph)
            chunks += 1
            s = d.reduce_ext(check=False)
            done, err, conv = tr.check(s, chunk)
            if done:
                break
            if tr.pending is not None and chunks % tick == 0:
                d.set_storage(*tr.pending)
                tr.switched()
    finally:
        d.close()
    k = nu_of(req.omega) * (s[4] / n) / req.force[0] if err is None else None
    return Result(req.rid, k, tr.steps, conv, 0.0, 0.0, time.perf_counter() - t0, error=err,
                  mean_ux=s[4] / max(nf, 1), low_steps=tr.low_steps)
