#!/usr/bin/env python
"""Benchmark of the sparse AA lattice Boltzmann hot path on GB300.

Workload (default): the 256^3 porosity sweep -- periodic Boolean sphere
packings, radii U(6, 12), porosity 0.3 / 0.5 / 0.7 / 0.9 (seeds 11-14), D3Q19
TRT (magic 3/16, tau 0.8), body force 1e-6 along x, FP32 shifted PDFs.
One benchmark step = `--lbm-steps` (default 100, even) LBM time steps, i.e.
alternating even/odd AA kernels, on each of the four domains.  The metric is
fluid lattice updates per second (MFLUPS) over all four domains; each domain's
PDF-list (>= 0.38 GB) exceeds the 129 MB L2, so no L2 flush is needed.

Also measured in the same run and added to the JSON line: per-porosity MFLUPS
and achieved HBM GB/s of each kernel against the measured copy peak, the dense
direct-addressing comparator, the FP16-storage form, memory per fluid cell,
an end-to-end solve through the public API from host buffers, and the FP64
oracle on the host cores as a CPU baseline.

`--impl reference` times the FP64 CPU oracle (a plain dense two-grid push
LBM) on the host cores, on a bounded sample of the same workload.

Multi-GPU: domains are independent, so every rank runs its own replica of
the workload (weak scaling, no data-path collective)."""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fluid lattice updates/s (MFLUPS), D3Q19 TRT sparse AA, FP32"
UNIT = "MFLUPS"
POROSITIES = (0.3, 0.5, 0.7, 0.9)
SEEDS = {0.3: 11, 0.5: 12, 0.7: 13, 0.9: 14}
N = 256
FORCE = (1e-6, 0.0, 0.0)
OMEGA = 1.0 / 0.8
MAGIC = 3.0 / 16.0
Q = 19
B_IDX = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lbm-steps", type=int, default=100, help="LBM time steps per benchmark step (even)")
    ap.add_argument("--porosities", default=",".join(str(p) for p in POROSITIES))
    ap.add_argument("--size", type=int, default=N)
    ap.add_argument("--no-extras", action="store_true", help="skip dense / FP16 / e2e / CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU baseline sample")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="PDF storage of the timed domains (the headline metric is FP32)")
    ap.add_argument("--shape-even", default=None, help="threads,cells,variant of the even kernel")
    ap.add_argument("--shape-odd", default=None, help="threads,cells,variant of the odd kernel")
    ap.add_argument("--cell-order", choices=["lex", "brick8"], default="lex",
                    help="compacted cell order of the timed domains")
    ap.add_argument("--mode", default="kernel", choices=["kernel", "serve", "workloads", "case"],
                    help="kernel: the porosity sweep (default); serve: the permeability-request stream; "
                         "workloads: the application-shaped domains; case: one domain stepped --lbm-steps "
                         "times without timing (the small cases the profiles are captured on)")
    ap.add_argument("--case", default="bed", choices=["bed", "bed16", "cm", "cumulant"],
                    help="case mode: the particle bed (FP32 / FP16, D3Q27 TRT, tuned shapes) or a "
                         "--size^3 porosity-0.5 packing with the central-moment / cumulant operator")
    ap.add_argument("--requests", type=int, default=64, help="serve mode: number of requests")
    ap.add_argument("--max-steps", type=int, default=20000, help="serve mode: step cap per request")
    ap.add_argument("--budget-gb", type=float, default=16.0, help="serve mode: HBM admission budget")
    ap.add_argument("--capacity", type=int, default=128, help="serve mode: pool slots")
    ap.add_argument("--arrivals", default="closed", choices=["closed", "poisson"],
                    help="serve mode: all at t=0, or Poisson arrivals at --load x the measured capacity")
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--sequential", action="store_true", help="serve mode: also time one-at-a-time solves")
    ap.add_argument("--pool-graph", type=int, default=1, help="serve mode: replay pool steps as CUDA graphs")
    ap.add_argument("--pool-streams", type=int, default=2, help="serve mode: streams of a pool step")
    ap.add_argument("--large-cap", type=int, default=2,
                    help="serve mode with lanes: at most this many requests in the large lane (0: no bound)")
    ap.add_argument("--lanes", default="1000000:4",
                    help="serve mode: 'CELLS:CHUNKS' puts requests below CELLS fluid cells in a lane that "
                         "advances CHUNKS chunks per tick ('none': one lockstep lane)")
    ap.add_argument("--group-mb", type=float, default=None,
                    help="serve mode: L2 group size of the pool in MiB (0 = one group; default: the library's)")
    ap.add_argument("--precision", default="plan", choices=["plan", "none"],
                    help="serve mode, 16-bit storage: 'plan' hands each solve off to FP32 storage once its "
                         "relative change per chunk falls below 3e-3 (and rescales while in 16 bits); 'none' "
                         "solves in 16 bits throughout")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="default run: requests of the serving summary (0 skips it)")
    ap.add_argument("--serve-repeats", type=int, default=3, help="default run: repeats of the serving summary")
    a = ap.parse_args()
    if a.lbm_steps % 2:
        raise SystemExit("--lbm-steps must be even (whole AA pairs)")
    a.porosities = tuple(float(x) for x in a.porosities.split(","))
    return a


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def geometry_for(phi, n):
    import geometry as G
    return G.boolean_spheres(n, phi, SEEDS.get(phi, 10 + int(phi * 10)))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].strip() == "Active"})
        power = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------- our arm
def workload_name(a):
    return (f"{a.size}^3 periodic Boolean sphere packings, porosity {'/'.join(str(p) for p in a.porosities)}, "
            f"D3Q19 TRT magic 3/16, tau 0.8, F=1e-6 x, {a.storage.upper()} PDFs")


def algorithmic_bytes(nf, b_pdf, q=Q, parity=0):
    """AA access model (Table 2, Sec. 5.1): even 2Q B_pdf, odd 2Q B_pdf + (Q-1) B_idx per cell."""
    return nf * (2 * q * b_pdf + (0 if parity == 0 else (q - 1) * B_IDX))


def run_ours(a, rank, world):
    import torch
    import paper_2408_06880_gb300 as P

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    peak, peak_kind = load_peaks()
    doms = []
    storage = {"fp32": P.FP32, "fp16": P.FP16, "bf16": P.BF16}[a.storage]
    b_pdf = 4 if storage == P.FP32 else 2
    for phi in a.porosities:
        g = geometry_for(phi, a.size)
        d = P.Domain(g.flags, periodic=7, q=Q, op=P.TRT, omega=OMEGA, trt_magic=MAGIC, force=FORCE,
                     storage=storage, scale_exp=P.auto_scale_exp(1e-3), stream=stream,
                     cell_order=P.ORDER_BRICK8 if a.cell_order == "brick8" else P.ORDER_LEX)
        apply_shapes(d, a)
        doms.append((phi, g, d))
    half = a.lbm_steps // 2

    def one_step(events=None):
        for j, (_, _, d) in enumerate(doms):
            for _ in range(half):
                if events is not None:
                    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    e[0].record(stream)
                    d.step(1)
                    e[1].record(stream)
                    d.step(1)
                    e[2].record(stream)
                    events[j].append(e)
                else:
                    d.step(2)

    for _ in range(a.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    events = [[] for _ in doms]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(a.steps):
        one_step(events)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    # whole job: the updates of every rank over the slowest rank's time
    from paper_2408_06880_gb300 import replicas
    updates_rank = sum(d.n_fluid for _, _, d in doms) * a.lbm_steps * a.steps
    rate, _, secs = replicas.job_rate(updates_rank, elapsed_ms / 1e3)
    elapsed_ms = secs * 1e3
    value = rate / 1e6

    # per-kernel durations from the events recorded on the launching stream
    per = []
    tot = {0: [0.0, 0.0], 1: [0.0, 0.0]}     # parity -> [bytes, ms]
    for j, (phi, g, d) in enumerate(doms):
        ev_ms = [e[0].elapsed_time(e[1]) for e in events[j]]
        od_ms = [e[1].elapsed_time(e[2]) for e in events[j]]
        nf = d.n_fluid
        be, bo = algorithmic_bytes(nf, b_pdf, parity=0), algorithmic_bytes(nf, b_pdf, parity=1)
        me, mo = float(np.mean(ev_ms)), float(np.mean(od_ms))
        tot[0][0] += be * len(ev_ms)
        tot[0][1] += sum(ev_ms)
        tot[1][0] += bo * len(od_ms)
        tot[1][1] += sum(od_ms)
        per.append({"porosity": phi, "n_fluid": nf, "achieved_porosity": round(g.porosity, 4),
                    "mflups": round(2 * nf / ((me + mo) / 1e3) / 1e6, 1),
                    "even_ms": round(me, 4), "odd_ms": round(mo, 4),
                    "even_gbs": round(be / me / 1e6, 1), "odd_gbs": round(bo / mo / 1e6, 1),
                    "pair_gbs": round((be + bo) / (me + mo) / 1e6, 1),
                    "pair_frac": round((be + bo) / (me + mo) / 1e6 / peak, 4),
                    "bytes_per_cell": round(d.memory_bytes() / nf, 2)})
    dom_par = 1 if tot[1][1] >= tot[0][1] else 0
    achieved = tot[dom_par][0] / tot[dom_par][1] / 1e6
    kname = "aa_odd_kernel" if dom_par else "aa_even_kernel"
    n_launch = len(doms) * a.lbm_steps * a.steps
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic_for(traffic_key(a.storage, kname), doms),
                "algorithmic_bytes_per_launch": round(tot[dom_par][0] / (n_launch / 2)),
                "both_kernels": {"even_gbs": round(tot[0][0] / tot[0][1] / 1e6, 1),
                                 "odd_gbs": round(tot[1][0] / tot[1][1] / 1e6, 1),
                                 "even_share": round(tot[0][1] / (tot[0][1] + tot[1][1]), 3)}}
    metric = METRIC if a.storage == "fp32" else METRIC.replace("FP32", a.storage.upper() + " storage")
    out = {"metric": metric, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": round(elapsed_ms / a.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16 storage, f32 math",
                                                          "bf16": "bf16 storage, f32 math"}[a.storage],
           "data": "synthetic",
           "config": {"workload": workload_name(a),
                      "lbm_steps_per_step": a.lbm_steps, "domains": len(doms), "cell_order": a.cell_order,
                      "l2": "inputs larger than L2 (PDF-list >= 0.38 GB per domain), no flush",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "roofline": roofline, "per_porosity": per, "clocks": clk, "gpu_launches": n_launch}
    if not a.no_extras and rank == 0:
        out["dense"] = bench_dense(a, P, stream, peak)
        out["pull"] = bench_pull(a, P, stream, peak, per)
        out["operators"] = bench_operators(a, P, stream, peak)
        out["fp16"] = bench_storage(a, P, stream, P.FP16, per)
        out["accuracy"] = bench_accuracy(P, stream)
        out["e2e"] = bench_e2e(a, P)
        if world == 1:
            out["cpu_baseline"] = cpu_baseline(a, [g for _, g, _ in doms])
            if a.serve_requests > 0:
                out["serve"] = bench_serve_summary(a, P)
    for _, _, d in doms:
        d.close()
    return out


def apply_shapes(d, a):
    for parity, spec in ((0, a.shape_even), (1, a.shape_odd)):
        if spec:
            t, c, v = (int(x) for x in spec.split(","))
            d.set_launch(parity, t, c, v)


def traffic_key(storage, kname):
    """Name of a kernel's record in the traffic file for a PDF storage (None: no record)."""
    prefix = {"fp32": "", "fp16": "fp16_"}.get(storage)
    return None if prefix is None else prefix + kname


def traffic_for(kname, doms):
    """DRAM bytes per launch from the committed ncu summary, scaled by cells,
    or None when the kernel source changed since the capture or there is no record."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    if kname is None or t.get("source_digest") != kernel_digest():
        return None
    per_cell = t.get("kernels", {}).get(kname, {}).get("dram_bytes_per_cell")
    if per_cell is None:
        return None
    nf = np.mean([d.n_fluid for _, _, d in doms])
    return round(per_cell * nf)


def kernel_digest():
    h = hashlib.sha256()
    for name in ("common.cuh", "aa_kernels.cuh", "aa_launch.cuh"):
        with open(os.path.join(ROOT, "paper_2408_06880_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def bench_dense(a, P, stream, peak, pairs=10):
    """Dense direct-addressing comparator on the same geometries (fluid MFLUPS)."""
    import torch
    res = []
    for phi in a.porosities:
        g = geometry_for(phi, a.size)
        d = P.Domain(g.flags, periodic=7, q=Q, op=P.TRT, omega=OMEGA, trt_magic=MAGIC, force=FORCE,
                     layout=P.DENSE, stream=stream)
        d.step(4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.step(2 * pairs)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (2 * pairs)
        nf = d.n_fluid
        res.append({"porosity": phi, "mflups": round(nf / (ms / 1e3) / 1e6, 1),
                    "bytes_per_fluid_cell": round(d.memory_bytes() / nf, 2)})
        d.close()
    return res


def bench_pull(a, P, stream, peak, per32, pairs=10):
    """The two-grid pull scheme (Sec. 5.1's comparison) on the same geometries:
    fluid MFLUPS, GB/s at its algorithmic bytes (2 Q B_pdf + (Q-1) 4 per
    update), and the AA pattern's speed-up over it."""
    import torch
    res = []
    for phi, aa in zip(a.porosities, per32):
        g = geometry_for(phi, a.size)
        d = P.Domain(g.flags, periodic=7, q=Q, op=P.TRT, omega=OMEGA, trt_magic=MAGIC, force=FORCE,
                     layout=P.SPARSE_PULL, stream=stream)
        d.step(4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.step(2 * pairs)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (2 * pairs)
        nf = d.n_fluid
        gbs = nf * (2 * Q * 4 + (Q - 1) * B_IDX) / (ms / 1e3) / 1e9
        m = nf / (ms / 1e3) / 1e6
        res.append({"porosity": phi, "mflups": round(m, 1), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                    "aa_speedup": round(aa["mflups"] / m, 4),
                    "bytes_per_fluid_cell": round(d.memory_bytes() / nf, 2)})
        d.close()
    return res


def bench_operators(a, P, stream, peak, pairs=10):
    """Sec. 5.1's comparison of streaming patterns per collision operator:
    AA and pull MFLUPS for SRT, TRT and MRT (D3Q19) and SRT, TRT, central
    moments and cumulants (D3Q27) on the porosity-0.5 domain (GB/s at each
    scheme's algorithmic bytes)."""
    import torch
    phi = 0.5 if 0.5 in a.porosities else a.porosities[0]
    g = geometry_for(phi, a.size)
    res = []
    for q, name, op in ((19, "SRT", P.SRT), (19, "TRT", P.TRT), (19, "MRT", P.MRT), (27, "SRT", P.SRT),
                        (27, "TRT", P.TRT), (27, "CM", P.CM), (27, "CUMULANT", P.CUMULANT)):
        row = {"op": name, "stencil": f"D3Q{q}"}
        for scheme, layout, idx in (("aa", P.SPARSE, (q - 1) * B_IDX / 2), ("pull", P.SPARSE_PULL, (q - 1) * B_IDX)):
            d = P.Domain(g.flags, periodic=7, q=q, op=op, omega=OMEGA, trt_magic=MAGIC, force=FORCE,
                         layout=layout, stream=stream)
            d.step(4)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d.step(2 * pairs)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / (2 * pairs)
            nf = d.n_fluid
            m = nf / (ms / 1e3) / 1e6
            gbs = nf * (2 * q * 4 + idx) / (ms / 1e3) / 1e9
            row[scheme] = {"mflups": round(m, 1), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
            d.close()
        row["aa_over_pull"] = round(row["aa"]["mflups"] / row["pull"]["mflups"], 4)
        res.append(row)
    return {"porosity": phi, "rows": res}


def bench_accuracy(P, stream):
    """Error of each PDF storage against the FP64 oracle, from its stored
    values (tests/golden/packing32_srt_200.npz, written by the oracle-only
    fixture script): the 32^3 relaxed packing, D3Q19 SRT, F = 1e-6 x, 200
    steps from rest -- velocity relative L2 over all fluid cells and the
    relative error of the permeability nu <u_x> / F_x."""
    import geometry as G
    fx = np.load(os.path.join(ROOT, "tests", "golden", "packing32_srt_200.npz"))
    u_o = fx["u"]
    k_o = float(fx["nu"]) * float(np.mean(u_o[:, 0])) / float(fx["force_x"])
    g = G.relaxed_spheres()
    out = {"workload": "32^3 relaxed packing (porosity 0.5), D3Q19 SRT, F = 1e-6 x, 200 steps from rest",
           "reference": "FP64 oracle, stored values"}
    for name, storage in (("fp32", P.FP32), ("fp16", P.FP16), ("bf16", P.BF16)):
        d = P.Domain(g.flags, periodic=7, q=19, op=P.SRT, omega=1.25, force=(1e-6, 0.0, 0.0), storage=storage,
                     scale_exp=P.auto_scale_exp(1e-3) if storage != P.FP32 else 0, stream=stream)
        d.step(int(fx["steps"]))
        _, u = d.macroscopic(P.ORDER_CELLS)
        u = u.T.astype(np.float64)
        d.close()
        k = float(fx["nu"]) * float(np.mean(u[:, 0])) / float(fx["force_x"])
        out[name] = {"u_rel_l2": float(f"{np.linalg.norm(u - u_o) / np.linalg.norm(u_o):.3g}"),
                     "permeability_rel_err": float(f"{abs(k / k_o - 1):.3g}")}
    return out


def bench_storage(a, P, stream, storage, per32, pairs=20):
    import torch
    res = []
    for phi, p32 in zip(a.porosities, per32):
        g = geometry_for(phi, a.size)
        d = P.Domain(g.flags, periodic=7, q=Q, op=P.TRT, omega=OMEGA, trt_magic=MAGIC, force=FORCE,
                     storage=storage, scale_exp=P.auto_scale_exp(1e-3), stream=stream)
        d.step(4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.step(2 * pairs)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (2 * pairs)
        m = d.n_fluid / (ms / 1e3) / 1e6
        res.append({"porosity": phi, "mflups": round(m, 1), "vs_fp32": round(m / p32["mflups"], 3),
                    "bytes_per_cell": round(d.memory_bytes() / d.n_fluid, 2)})
        d.close()
    return res


def bench_e2e(a, P):
    """The benchmark's metric end to end through the public API, from HOST
    buffers: create every porosity domain from its flag array in pinned host
    memory (the H2D copy of the inputs), then `steps` benchmark steps -- each
    `lbm_steps` LBM steps per domain followed by a D2H read of every domain's
    five FP64 sums (the step's result) -- and free.  Wall-clock MFLUPS over
    the whole job, creation included."""
    import torch
    flags = [torch.from_numpy(np.ascontiguousarray(geometry_for(phi, a.size).flags)).pin_memory()
             for phi in a.porosities]
    torch.cuda.synchronize()
    t = time.perf_counter()
    doms = [P.Domain(f.numpy(), periodic=7, q=Q, op=P.TRT, omega=OMEGA, trt_magic=MAGIC, force=FORCE)
            for f in flags]
    sums = None
    for _ in range(a.steps):
        for d in doms:
            d.step(a.lbm_steps, graph=True)
        sums = [d.reduce() for d in doms]
    updates = sum(d.n_fluid for d in doms) * a.lbm_steps * a.steps
    for d in doms:
        d.close()
    wall = time.perf_counter() - t
    h2d = sum(int(f.numel()) for f in flags)
    return {"value": round(updates / wall / 1e6, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d // a.steps), "d2h_bytes_per_step": 40 * len(flags),
            "what": f"create the {len(flags)} domains from pinned host flags, {a.steps} steps of "
                    f"{a.lbm_steps} LBM steps per domain each followed by a host read of every domain's "
                    f"5 FP64 sums, free; wall clock; the flags' H2D bytes amortised over the steps",
            "final_sum_ux": [float(x[4]) for x in sums]}


def _oracle_domains(a, geoms=None):
    """Oracle problems of the sweep's domains, built one at a time (each
    FP64 state is 2.5 GB at 256^3): yields (problem, state, fluid cells)."""
    import oracle as O
    for j, phi in enumerate(a.porosities):
        g = geoms[j] if geoms is not None else geometry_for(phi, a.size)
        p = O.Problem.from_geometry(g, q=Q, op=O.TRT, omega_plus=OMEGA, magic=MAGIC, force=FORCE)
        yield p, O.dense_init(p), int(np.count_nonzero(g.flags == 0))


def cpu_baseline(a, geoms=None):
    """The FP64 oracle as it stands, on this host's cores, on a bounded
    sample of the workload: 2-step runs on each domain of the sweep in turn
    (the geometries of the timed domains when given), a quarter of the budget
    each and at least one run; only the stepping is timed."""
    import oracle as O
    updates, steps, timed = 0, 0, 0.0
    share = a.cpu_seconds / len(a.porosities)
    for p, f, nf in _oracle_domains(a, geoms):
        spent = 0.0
        while True:
            t = time.perf_counter()
            f = O.dense_run(p, f, 2)
            spent += time.perf_counter() - t
            updates += 2 * nf
            steps += 2
            if spent >= share:
                break
        timed += spent
        del p, f
    return {"value": round(updates / timed / 1e6, 3), "unit": UNIT, "cores": O.max_threads(),
            "kind": "oracle", "sample": f"dense FP64 push oracle, 2-step runs on each {a.size}^3 domain of porosity "
                                        f"{'/'.join(str(p) for p in a.porosities)} in turn, {steps} LBM steps "
                                        f"({timed:.1f} s of stepping)"}


# ---------------------------------------------------------- reference arm
def run_reference(a):
    """The FP64 CPU oracle on the host cores, on the same workload: each
    benchmark step is 2 dense two-grid steps (one AA-pair equivalent); the
    steps are split into consecutive blocks over the sweep's domains (one
    domain resident at a time, the warm-up steps on the first), so the
    sample spans every domain.  Only the stepping is timed; the value is the
    fluid updates over that time."""
    import oracle as O
    n = len(a.porosities)
    blocks = [a.steps * (j + 1) // n - a.steps * j // n for j in range(n)]
    updates, timed = 0, 0.0
    for j, (p, f, nf) in enumerate(_oracle_domains(a)):
        if j == 0:
            for _ in range(a.warmup):
                f = O.dense_run(p, f, 2)
        t = time.perf_counter()
        for _ in range(blocks[j]):
            f = O.dense_run(p, f, 2)
        timed += time.perf_counter() - t
        updates += 2 * nf * blocks[j]
        del p, f
    v = updates / timed / 1e6 if timed > 0 else float("nan")
    sample = (f"dense FP64 push oracle; 2 LBM steps per benchmark step, the steps split in blocks of "
              f"{'/'.join(map(str, blocks))} over the {a.size}^3 domains of porosity "
              f"{'/'.join(str(p) for p in a.porosities)}")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(timed / max(a.steps, 1) * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": sample, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def serve_requests(n, max_steps):
    """The permeability-request stream: request i is a periodic Boolean sphere
    packing of edge in {64, 96, 128, 192}, porosity U(0.3, 0.8), radii
    U(6, 12), seed 41000 + i, D3Q19 TRT body-forced (F = 1e-6 x)."""
    import geometry as G
    from paper_2408_06880_gb300.serving import Request
    reqs = []
    for i in range(n):
        g = G.serving_request(i)
        reqs.append(Request(i, g.flags, force=FORCE, omega=OMEGA, trt_magic=MAGIC, max_steps=max_steps, tol=1e-6,
                            meta=dict(edge=g.meta["edge"], porosity=g.porosity)))
    return reqs


ORACLE_SERVING = os.path.join(ROOT, "tests", "golden", "serving16_oracle.json")


def oracle_permeability_errors(results):
    """Relative permeability error of served results against the FP64
    oracle's values stored in tests/golden/serving16_oracle.json (written by
    tests/golden/make_oracle_fixtures.py: the oracle's sum of u_x after every
    100 steps of the first 16 requests of edge 64 or 96), compared at the
    result's own step count (the oracle's last stored value when the result
    ran longer).  {} when the file is absent."""
    try:
        with open(ORACLE_SERVING) as f:
            ref = {r["rid"]: r for r in json.load(f)["requests"]}
    except Exception:
        return {}
    out = {}
    for r in results:
        o = ref.get(r.rid)
        if o is None or r.permeability is None or r.steps <= 0:
            continue
        j = min(r.steps // 100, len(o["sum_ux"])) - 1
        k_o = o["nu"] * (o["sum_ux"][j] / o["n_voxels"]) / 1e-6
        out[r.rid] = abs(r.permeability / k_o - 1)
    return out


def make_executor(a, P, storage, lanes_spec=None):
    from paper_2408_06880_gb300.serving import GpuExecutor, Precision
    spec = a.lanes if lanes_spec is None else lanes_spec
    lanes = None
    if spec != "none":
        cells, chunks = (int(x) for x in spec.split(":"))
        lanes = ((cells, chunks), (None, 1, a.large_cap or None))
    prec = Precision() if storage != P.FP32 and a.precision == "plan" else None
    return GpuExecutor(Q, storage, capacity=a.capacity, graph=bool(a.pool_graph),
                       group_bytes=None if a.group_mb is None else int(a.group_mb * 2 ** 20),
                       streams=a.pool_streams, lanes=lanes, precision=prec)


def bench_serve_summary(a, P, storages=("fp32", "fp16")):
    """Bounded serving measurement for the default line: the first
    `--serve-requests` requests of the stream as a closed batch through the
    continuous-batching server, and the same requests solved one at a time,
    per storage (16-bit storage with the FP32 hand-off plan), repeated
    `--serve-repeats` times; medians and the spread of the served /
    one-at-a-time ratio.  Accuracy: each 16-bit result against the FP32
    result of the same request, and against the FP64 oracle's stored values
    for the requests of the oracle subset."""
    import torch
    from paper_2408_06880_gb300.serving import Server, solve_alone
    reqs = serve_requests(a.requests if a.mode == "serve" else a.serve_requests, a.max_steps)
    budget = int(a.budget_gb * 2 ** 30)
    out = {"requests": len(reqs), "repeats": a.serve_repeats,
           "what": "closed batch of the first requests of the permeability stream (D3Q19 TRT, F = 1e-6, "
                   "converged to 1e-6 relative change of mean u_x per 100 steps), served with continuous "
                   "batching and solved one at a time; 16-bit storage handed off to FP32 (precision plan)"}
    k_by = {}
    for name in storages:
        storage = {"fp32": P.FP32, "fp16": P.FP16, "bf16": P.BF16}[name]
        served, seq, ratio = [], [], []
        for _ in range(max(1, a.serve_repeats)):
            ex = make_executor(a, P, storage)
            try:
                res, st = Server(ex, budget, chunk=100).run(reqs, realtime=False)
                ticks = {r.rid: ex.tick_chunks(r) for r in reqs}
            finally:
                ex.close()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            alone = [solve_alone(r, storage=storage, precision=ex.precision, tick=ticks[r.rid]) for r in reqs]
            wall = time.perf_counter() - t0
            lat = np.array([r.latency for r in alone])
            sq = {"solves_per_s": len(alone) / wall, "latency_p50_s": float(np.percentile(lat, 50)),
                  "latency_p99_s": float(np.percentile(lat, 99))}
            served.append(st)
            seq.append(sq)
            ratio.append(st["solves_per_s"] / sq["solves_per_s"])
        med = lambda xs, key: float(np.median([x[key] for x in xs]))  # noqa: E731
        k_alone = {r.rid: r.permeability for r in alone}
        row = {"served_solves_per_s": round(med(served, "solves_per_s"), 4),
               "served_p50_s": round(med(served, "latency_p50_s"), 4),
               "served_p99_s": round(med(served, "latency_p99_s"), 4),
               "one_at_a_time_solves_per_s": round(med(seq, "solves_per_s"), 4),
               "one_at_a_time_p50_s": round(med(seq, "latency_p50_s"), 4),
               "one_at_a_time_p99_s": round(med(seq, "latency_p99_s"), 4),
               "served_over_one_at_a_time": {"median": round(float(np.median(ratio)), 4),
                                             "min": round(min(ratio), 4), "max": round(max(ratio), 4)},
               "converged": int(sum(r.converged for r in res)), "solved": st["solved"],
               "served_equals_alone": all(r.permeability == k_alone[r.rid] and r.steps == a_.steps
                                          for r in res for a_ in alone if a_.rid == r.rid and r.error is None),
               "low_precision_step_share": round(st["low_precision_step_share"], 4)}
        k_by[name] = {r.rid: r.permeability for r in res if r.error is None}
        oerr = oracle_permeability_errors(res)
        if oerr:
            row["vs_fp64_oracle"] = {"requests": len(oerr), "max_rel_error": float(max(oerr.values())),
                                     "median_rel_error": float(np.median(list(oerr.values())))}
        out[name] = row
    if "fp32" in k_by:
        for name in storages:
            if name == "fp32":
                continue
            e = [abs(k_by[name][i] / k_by["fp32"][i] - 1) for i in k_by[name] if i in k_by["fp32"]]
            out[name]["vs_fp32_permeability"] = {"max_rel_error": float(max(e)), "median_rel_error":
                                                 float(np.median(e))}
            out[name]["served_vs_fp32_served"] = round(out[name]["served_solves_per_s"] /
                                                       out["fp32"]["served_solves_per_s"], 4)
    return out


def run_serve(a):
    """Serve mode: continuous batching of the request stream (closed batch or
    Poisson arrivals), optionally against one-at-a-time solves.  Under
    torchrun every rank serves its share of the requests on its own GPU
    (replicas, no exchange); rank 0 reports the whole job."""
    import torch
    import paper_2408_06880_gb300 as P
    from paper_2408_06880_gb300 import replicas
    from paper_2408_06880_gb300.serving import serve_replicas, solve_alone
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    rank, world = replicas.rank_world()
    storage = {"fp32": P.FP32, "fp16": P.FP16, "bf16": P.BF16}[a.storage]
    reqs = serve_requests(a.requests, a.max_steps)
    out = {"metric": "solves/s (continuous batching, permeability requests)", "unit": "solves/s",
           "n_gpus": world, "higher_is_better": True, "data": "synthetic", "storage": a.storage,
           "scaling": "strong" if world > 1 else "weak",
           "config": {"workload": f"{a.requests} permeability requests: periodic Boolean packings, edge "
                                  f"{{64,96,128,192}}, porosity U(0.3,0.8), D3Q19 TRT F=1e-6, converge to "
                                  f"1e-6 relative change of mean u_x per 100 steps or {a.max_steps} steps",
                      "budget_gb": a.budget_gb, "capacity": a.capacity, "arrivals": a.arrivals,
                      "pool_graph": bool(a.pool_graph), "group_mb": a.group_mb,
                      "pool_streams": a.pool_streams, "lanes": a.lanes, "large_cap": a.large_cap,
                      "parallelism": f"request replicas x{world}" if world > 1 else "single GPU"}}
    ex = make_executor(a, P, storage)
    out["config"]["precision"] = "fp32 hand-off plan" if ex.precision is not None else "none"
    budget = int(a.budget_gb * 2 ** 30)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", 0)))
    clocks.start()
    res, st = serve_replicas(ex, reqs, budget, realtime=False, chunk=100)
    out["clocks"] = clocks.stop()
    out["closed_batch"] = st
    out["value"] = round(st["solves_per_s"], 4)
    if a.arrivals == "poisson":
        # arrivals over the whole stream at `load` x the measured capacity
        rate = a.load * (st["solves_per_s"] if rank == 0 else 0.0)
        rate = replicas.job_rate(rate, 1.0)[1]              # rank 0's value, on every rank
        rng = np.random.default_rng(4100)
        t = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
        for r, ti in zip(reqs, t):
            r.arrival = float(ti)
        _, st_p = serve_replicas(ex, reqs, budget, realtime=True, chunk=100)
        out["poisson"] = dict(st_p, rate_per_s=rate)
    ticks = {r.rid: ex.tick_chunks(r) for r in reqs}
    prec = ex.precision
    ex.close()
    out["results"] = [{"rid": r.rid, "k": r.permeability, "steps": r.steps, "low_precision_steps": r.low_steps,
                       "converged": r.converged, "latency_s": round(r.latency, 4), "error": r.error}
                      for r in sorted(res, key=lambda r: r.rid)]
    oerr = oracle_permeability_errors(res)
    if oerr:
        out["vs_fp64_oracle"] = {"requests": len(oerr), "max_rel_error": float(max(oerr.values())),
                                 "median_rel_error": float(np.median(list(oerr.values()))),
                                 "per_request": {str(k): v for k, v in sorted(oerr.items())}}
    if a.sequential:
        mine = replicas.shard(reqs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        alone = [solve_alone(r, storage=storage, precision=prec, tick=ticks[r.rid]) for r in mine]
        wall = time.perf_counter() - t0
        sps, _, wall_max = replicas.job_rate(len(alone), wall)
        # service times and one-at-a-time FIFO latencies per rank (each rank
        # a FIFO server of its share under the same arrivals)
        done, fifo = 0.0, []
        lat = [r.latency for r in alone]
        for r, s_ in sorted(zip(mine, lat), key=lambda x: (x[0].arrival, x[0].rid)):
            done = max(done, r.arrival) + s_
            fifo.append(done - r.arrival)
        parts = replicas.gather((alone, lat, fifo))
        if parts is not None:
            alone = [r for p_ in parts for r in p_[0]]
            lat = np.array([x for p_ in parts for x in p_[1]])
            fifo = np.array([x for p_ in parts for x in p_[2]])
            seq = {"solves_per_s": sps, "wall_s": wall_max,
                   "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99))}
            if a.arrivals == "poisson":
                seq["poisson_fifo"] = {"latency_p50_s": float(np.percentile(fifo, 50)),
                                       "latency_p99_s": float(np.percentile(fifo, 99)),
                                       "latency_mean_s": float(np.mean(fifo))}
            out["one_at_a_time"] = seq
            k_alone = {r.rid: r.permeability for r in alone}
            out["served_equals_alone"] = all(r.permeability == k_alone[r.rid] for r in res if r.error is None)
            steps_alone = {r.rid: r.steps for r in alone}
            out["served_steps_equal_alone"] = all(r.steps == steps_alone[r.rid] for r in res if r.error is None)
    return out


def _time_pairs(P, d, stream, pairs):
    import torch
    d.step(4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.step(2 * pairs)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (2 * pairs)            # ms per LBM step


def full_bricks(flags):
    """Complete 8^3 bricks whose 512 voxels are all fluid (the cells the
    hybrid cell order steps as dense blocks)."""
    nz, ny, nx = flags.shape
    f = flags[:nz // 8 * 8, :ny // 8 * 8, :nx // 8 * 8] == 0
    f = f.reshape(nz // 8, 8, ny // 8, 8, nx // 8, 8)
    return int(np.count_nonzero(f.all(axis=(1, 3, 5))))


def run_workloads(a, pairs=10):
    """The application-shaped workloads (stand-ins for Sec. 6.2 and 6.3):
    the 512 x 256 x 256 particle bed (D3Q27 TRT, velocity inlet, pressure
    outlet, FP32 and FP16) and the 1024 x 512 x 512 artery tree (D3Q19 TRT,
    sparse, plus the dense comparator on the same voxels with the inlet and
    outlet voxels as walls -- it supports no open boundaries): MFLUPS, GB/s
    at the algorithmic bytes, memory per fluid cell, fluid fraction."""
    import torch
    import geometry as G
    import paper_2408_06880_gb300 as P
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.Stream()
    peak, _ = load_peaks()
    out = {"mode": "workloads", "data": "synthetic", "peak_gbs": peak, "rows": []}

    def row(name, g, q, storage, layout=P.SPARSE, flags=None, order=P.ORDER_LEX):
        b = 4 if storage == P.FP32 else 2
        d = P.Domain(g.flags if flags is None else flags, periodic=g.periodic,
                     inlet_u=g.inlet_u if flags is None else None, rho_out=g.rho_out, q=q, op=P.TRT, omega=OMEGA,
                     trt_magic=MAGIC, storage=storage, scale_exp=P.auto_scale_exp(0.06) if storage else 0,
                     layout=layout, stream=stream, cell_order=order)
        shapes = None
        mem = d.memory_bytes()              # before the tuner builds its candidates' optional tables
        if layout == P.SPARSE and order != P.ORDER_HYBRID:
            from paper_2408_06880_gb300 import tuner
            shapes = tuner.tune_domain(d, reps=5, use_cache=False, stream=stream)   # state restored
        ms = _time_pairs(P, d, stream, pairs)
        nf = int(np.count_nonzero(g.flags == 0))
        per = (2 * q * b + (q - 1) * B_IDX / 2) if layout == P.SPARSE else None
        extra = {}
        if order == P.ORDER_HYBRID:
            # index bytes of the odd step: every link of the sparse cells, the
            # face links of the full bricks
            n_full = full_bricks(g.flags)
            faces = {19: 1824, 27: 3176}[q]
            idx = ((nf - 512 * n_full) * (q - 1) + n_full * faces) * B_IDX
            per = 2 * q * b + idx / nf / 2
            extra = {"full_brick_cells": 512 * n_full, "full_brick_share": round(512 * n_full / nf, 4)}
        r = {"workload": name, "q": q, "storage": {P.FP32: "fp32", P.FP16: "fp16"}[storage],
             "cell_order": {P.ORDER_LEX: "lex", P.ORDER_BRICK8: "brick8", P.ORDER_HYBRID: "hybrid"}[order], **extra,
             "layout": {P.SPARSE: "sparse", P.DENSE: "dense"}[layout], "n_voxels": int(g.flags.size),
             "n_fluid": nf, "fluid_fraction": round(nf / g.flags.size, 5),
             "mflups": round(nf / (ms / 1e3) / 1e6, 1), "ms_per_step": round(ms, 4),
             "bytes_per_fluid_cell": round(mem / nf, 2)}
        if shapes:
            r["shapes"] = {"even": list(shapes["even"]), "odd": list(shapes["odd"]), "by": "autotuner"}
        if per is not None:
            gbs = nf * per / (ms / 1e3) / 1e9
            r.update({"gbs": round(gbs, 1), "frac": round(gbs / peak, 4)})
        d.close()
        out["rows"].append(r)
        print(json.dumps(r), file=sys.stderr, flush=True)

    bed = G.particle_bed()
    row("particle bed 512x256x256", bed, 27, P.FP32)
    row("particle bed 512x256x256", bed, 27, P.FP16)
    row("particle bed 512x256x256 (hybrid: full bricks dense)", bed, 27, P.FP32, order=P.ORDER_HYBRID)
    row("particle bed 512x256x256 (hybrid: full bricks dense)", bed, 27, P.FP16, order=P.ORDER_HYBRID)
    art = G.artery_tree()
    row("artery tree 1024x512x512", art, 19, P.FP32)
    walls = np.where(art.flags >= G.INLET, np.uint8(G.WALL), art.flags).astype(np.uint8)
    row("artery tree 1024x512x512 (inlet/outlet as walls)", art, 19, P.FP32, P.DENSE, flags=walls)
    return out


def run_case(a):
    """One domain stepped `--lbm-steps` times with its default launch shapes
    (the particle bed: the shapes the autotuner picks for it), no timing: the
    small cases the ncu summaries under profiles/ are captured on."""
    import torch
    import geometry as G
    import paper_2408_06880_gb300 as P
    stream = torch.cuda.Stream()
    if a.case in ("bed", "bed16"):
        g = G.particle_bed()
        storage = P.FP32 if a.case == "bed" else P.FP16
        d = P.Domain(g.flags, periodic=g.periodic, inlet_u=g.inlet_u, rho_out=g.rho_out, q=27, op=P.TRT,
                     omega=OMEGA, trt_magic=MAGIC, storage=storage,
                     scale_exp=P.auto_scale_exp(0.06) if storage else 0, stream=stream)
        even, odd = ((64, 4, 2), (64, 1, 2)) if a.case == "bed" else ((128, 2, 1), (128, 1, 2))
        d.set_launch(0, *even)
        d.set_launch(1, *odd)
    else:
        g = geometry_for(0.5, a.size)
        d = P.Domain(g.flags, periodic=7, q=27, op=P.CM if a.case == "cm" else P.CUMULANT, omega=OMEGA,
                     force=FORCE, stream=stream)
    d.step(a.lbm_steps)
    torch.cuda.synchronize()
    out = {"mode": "case", "case": a.case, "n_fluid": d.n_fluid, "lbm_steps": a.lbm_steps}
    d.close()
    return out


def main():
    a = parse()
    if a.mode == "case" and a.impl == "ours":
        print(json.dumps(run_case(a)), flush=True)
        return
    if a.mode == "workloads" and a.impl == "ours":
        print(json.dumps(run_workloads(a)), flush=True)
        return
    if a.mode == "serve" and a.impl == "ours":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
        out = run_serve(a)
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(out), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if a.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(a)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out = run_ours(a, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
