"""Shared helpers for the GPU-vs-oracle parity tests (test code only)."""
from __future__ import annotations

import numpy as np

import oracle as O

SRT, TRT = 0, 1


def oracle_problem(g, q=19, op=SRT, omega=1.25, magic=3 / 16, force=(0.0, 0.0, 0.0)):
    return O.Problem.from_geometry(g, q=q, op=op, omega_plus=omega, magic=magic, force=tuple(force))


def oracle_fields(g, steps, rho0=None, u0=None, **kw):
    """Dense FP64 oracle: (rho[N], u[N,3]) after `steps` steps."""
    p = oracle_problem(g, **kw)
    f = O.dense_init(p, rho0, u0)
    f = O.dense_run(p, f, steps)
    return O.dense_macroscopic(p, f), p, f


def gpu_domain(g, **kw):
    import paper_2408_06880_gb300 as P
    return P.Domain(g.flags, periodic=g.periodic, inlet_u=g.inlet_u, rho_out=g.rho_out, **kw)


def gpu_fields(dom):
    """(rho[N], u[N,3]) in voxel order from the GPU (zeros off fluid)."""
    import paper_2408_06880_gb300 as P
    rho, u = dom.macroscopic(P.ORDER_VOXELS)
    return rho.astype(np.float64), u.T.astype(np.float64)


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def fluid_mask(g):
    return g.flags.reshape(-1) == 0
