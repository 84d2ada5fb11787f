"""Writes the stored expected values of the long full-size parity tests and of
the serving accuracy report.  It calls only the FP64 oracle (``oracle/``) and
the seeded input generators (``geometry/``); nothing here touches the CUDA
library.  The oracle is compiled without FMA contraction and uses only IEEE
+, -, *, / , so the values are the same on x86 and Arm hosts.

    python tests/golden/make_oracle_fixtures.py sweep     # sweep256_phi05_trt_1000.npz
    python tests/golden/make_oracle_fixtures.py bed       # bed_full_q27_200.npz
    python tests/golden/make_oracle_fixtures.py serving   # serving16_oracle.json
    python tests/golden/make_oracle_fixtures.py packing   # packing32_srt_200.npz

sweep: the 256^3 periodic Boolean packing of porosity 0.5 (seed 12), D3Q19
  TRT (omega+ = 1.25, magic 3/16), body force 1e-6 along x, rest start, 1000
  steps of the oracle's sparse pull stepper.  Stored: the five FP64 domain
  sums over all fluid cells and (rho, u) of 32768 cells drawn without
  replacement (numpy PCG64 seed 2408), in the compacted lexicographic order.
bed: the full 512 x 256 x 256 particle bed (seed 21; inlet u = 0.05, outlet
  rho = 1), D3Q27 TRT, no body force, rest start, 200 steps; the same stored
  quantities.
serving: the first 16 requests of the permeability stream whose edge is 64 or
  96 (D3Q19 TRT, F = 1e-6 x): sum of u_x over the fluid cells after every 100
  steps, until the relative change of the mean u_x over 100 steps falls below
  1e-6 (the serving criterion) and then 1000 steps further, or 20000 steps;
  plus each request's voxel count, fluid cells and nu, so that the
  permeability at any of those steps is nu * (sum u_x / N) / F_x.
packing: the 32^3 relaxed packing (r = 4, porosity 0.5, seed 1), D3Q19 SRT
  (omega = 1.25), body force 1e-6 along x, rest start, 200 steps; stored:
  rho and u of every fluid cell in the compacted lexicographic order, and nu.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import geometry as G  # noqa: E402
import oracle as O  # noqa: E402

SAMPLE = 32768
SAMPLE_SEED = 2408


def _sample_fields(p, L, f, path, steps, extra):
    rho, u = O.sparse_macroscopic(p, L, f)
    nf = L.n_fluid
    sums = np.array([np.sum(rho - 1.0), np.sum(rho * u[:, 0]), np.sum(rho * u[:, 1]), np.sum(rho * u[:, 2]),
                     np.sum(u[:, 0])])
    cells = np.sort(np.random.default_rng(SAMPLE_SEED).choice(nf, size=min(SAMPLE, nf), replace=False))
    np.savez_compressed(path, cells=cells.astype(np.int32), rho=rho[cells], u=u[cells], sums=sums,
                        n_fluid=np.int64(nf), steps=np.int64(steps), u_norm=np.float64(np.linalg.norm(u)),
                        **extra)
    print(f"wrote {path}: N_F={nf}, sums={sums}", flush=True)


def sweep():
    g = G.boolean_spheres(256, 0.5, 12)
    p = O.Problem.from_geometry(g, q=19, op=O.TRT, omega_plus=1.25, magic=3 / 16, force=(1e-6, 0.0, 0.0))
    L = O.pull_list(p)
    t = time.time()
    f = O.sparse_run(p, L, O.sparse_rest(p, L), 1000)
    print(f"sweep: 1000 steps in {time.time() - t:.0f} s", flush=True)
    _sample_fields(p, L, f, os.path.join(HERE, "sweep256_phi05_trt_1000.npz"), 1000, {})


def bed():
    g = G.particle_bed()
    p = O.Problem.from_geometry(g, q=27, op=O.TRT, omega_plus=1.25, magic=3 / 16, force=(0.0, 0.0, 0.0))
    L = O.pull_list(p)
    t = time.time()
    f = O.sparse_run(p, L, O.sparse_rest(p, L), 200)
    print(f"bed: 200 steps in {time.time() - t:.0f} s", flush=True)
    _sample_fields(p, L, f, os.path.join(HERE, "bed_full_q27_200.npz"), 200, {})


def serving_subset(n=16):
    """Request ids of the first n requests of edge 64 or 96."""
    ids, i = [], 0
    while len(ids) < n:
        rng = np.random.default_rng(41000 + i)          # the stream's own first draw: the edge
        if int(rng.choice([64, 96, 128, 192])) in (64, 96):
            ids.append(i)
        i += 1
    return ids


def serving(tol=1e-6, max_steps=20000, chunk=100, after=1000):
    out = {"what": "FP64 oracle (sparse pull stepper) on the first 16 requests of edge 64 or 96 of the "
                   "permeability stream: sum of u_x over fluid cells after every 100 steps",
           "tol": tol, "chunk": chunk, "force_x": 1e-6, "omega": 1.25, "magic": 3 / 16, "requests": []}
    for rid in serving_subset():
        g = G.serving_request(rid)
        p = O.Problem.from_geometry(g, q=19, op=O.TRT, omega_plus=1.25, magic=3 / 16, force=(1e-6, 0.0, 0.0))
        L = O.pull_list(p)
        f = O.sparse_rest(p, L)
        t = time.time()
        sums, prev, conv_at, steps = [], None, None, 0
        while steps < max_steps:
            f = O.sparse_run(p, L, f, chunk)
            steps += chunk
            _, u = O.sparse_macroscopic(p, L, f)
            s = float(np.sum(u[:, 0]))
            sums.append(s)
            m = s / L.n_fluid
            if conv_at is None and prev is not None and m != 0.0 and abs(m - prev) / abs(m) < tol:
                conv_at = steps
            prev = m
            if conv_at is not None and steps >= conv_at + after:
                break
        k = O.permeability(p, sums[(conv_at or steps) // chunk - 1])
        out["requests"].append({"rid": rid, "edge": g.meta["edge"], "n_voxels": int(g.flags.size),
                                "n_fluid": int(L.n_fluid), "nu": p.nu, "converged_at": conv_at,
                                "permeability_at_convergence": k, "sum_ux": sums})
        print(f"request {rid}: N_F={L.n_fluid} converged at {conv_at} k={k:.6g} ({time.time() - t:.0f} s)",
              flush=True)
        with open(os.path.join(HERE, "serving16_oracle.json"), "w") as fh:
            json.dump(out, fh)


def packing():
    g = G.relaxed_spheres()
    p = O.Problem.from_geometry(g, q=19, op=O.SRT, omega_plus=1.25, force=(1e-6, 0.0, 0.0))
    L = O.pull_list(p)
    f = O.sparse_run(p, L, O.sparse_rest(p, L), 200)
    rho, u = O.sparse_macroscopic(p, L, f)
    path = os.path.join(HERE, "packing32_srt_200.npz")
    np.savez_compressed(path, rho=rho, u=u, nu=np.float64(p.nu), steps=np.int64(200), force_x=np.float64(1e-6))
    print(f"wrote {path}: N_F={L.n_fluid}", flush=True)


if __name__ == "__main__":
    what = sys.argv[1:] or ["sweep", "bed", "serving", "packing"]
    for w in what:
        {"sweep": sweep, "bed": bed, "serving": serving, "packing": packing}[w]()
