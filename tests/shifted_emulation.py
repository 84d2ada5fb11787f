"""Test instrument, not part of the library: the sparse two-grid pull stepper
of the oracle (TRT with the Guo source, halfway bounce-back through the pull
list, the inlet and outlet maps) written over shifted populations g = f - w,
vectorised with numpy in a chosen floating-point type.  In float64 it
reproduces the oracle (a CPU test holds it to 1e-11); in float32 it shows
what storing and updating the shifted populations in single precision alone
does to a run, independently of the CUDA kernels' order of operations.

The relations used: with f = g + w and f_eq - w = w (drho + rho (3 c.u +
4.5 (c.u)^2 - 1.5 u.u)), the collision keeps its form in g; the inlet map
f' = f* + 6 w c.u_w keeps its form; the outlet map f' = -f* + 2 w rho_out
(1 + 4.5 (c.u)^2 - 1.5 u.u) becomes g' = -g* + 2 w ((rho_out - 1) +
rho_out (4.5 (c.u)^2 - 1.5 u.u))."""
import numpy as np

import oracle as O


def run(p, lists, steps, dtype):
    """(rho, u[N_F, 3]) after `steps` steps from rest, computed in `dtype`;
    for a tuple of step counts, a list with the fields after each."""
    marks = tuple(steps) if isinstance(steps, (tuple, list)) else (steps,)
    dt = np.dtype(dtype).type
    c, w, inv = O.stencil(p.q)
    c = c.astype(dt)
    w = w.astype(dt)
    nf, S = lists.n_fluid, lists.stride
    P = lists.P[:, :nf]
    li, lk = np.nonzero(P < 0)                       # links: row i - 1, cell k
    b = -(P[li, lk].astype(np.int64)) - 1
    btype, bu = lists.bc_type[b], lists.bc_u[b].astype(dt)
    i_dir = li + 1
    src_row = inv[i_dir]
    slots = np.where(P >= 0, P, 0).astype(np.int64)
    rows, cols = slots // S, slots % S
    one, half = dt(1), dt(0.5)
    wp, wm = dt(p.omega_plus), dt(p.omega_minus)
    F = np.asarray(p.force, dt)
    inl, out = btype == 2, btype == 3
    ro = dt(p.rho_out)
    g = np.zeros((p.q, nf), dt)

    def moments(g):
        drho = g.sum(axis=0, dtype=dt)
        rho = one + drho
        return drho, rho, ((c.T @ g).astype(dt) + half * F[:, None]) / rho

    found = []
    for t in range(max(marks) + 1):
        if t in marks:
            _, rho, u = moments(g)
            found.append((rho.astype(np.float64), u.T.astype(np.float64)))
        if t == max(marks):
            break
        drho, rho, u = moments(g)
        cu = (c @ u).astype(dt)
        uu = (u * u).sum(axis=0, dtype=dt)
        e = w[:, None] * (drho[None, :] + rho[None, :] * (dt(3) * cu + dt(4.5) * cu * cu - dt(1.5) * uu[None, :]))
        cF = (c @ F).astype(dt)
        uF = (u * F[:, None]).sum(axis=0, dtype=dt)
        s = w[:, None] * (dt(3) * (cF[:, None] - uF[None, :]) + dt(9) * cu * cF[:, None])
        gp, gm = half * (g + g[inv]), half * (g - g[inv])
        ep, em = half * (e + e[inv]), half * (e - e[inv])
        sp, sm = half * (s + s[inv]), half * (s - s[inv])
        C = g - wp * (gp - ep) - wm * (gm - em) + (one - half * wp) * sp + (one - half * wm) * sm
        new = np.empty_like(g)
        new[0] = C[0]
        new[1:] = C[rows, cols]
        src = C[src_row, lk]
        ww, ci = w[i_dir], c[i_dir]
        val = src.copy()
        val[inl] = src[inl] + dt(6) * ww[inl] * (ci[inl] * bu[inl]).sum(axis=1, dtype=dt)
        uc = u[:, lk[out]].T
        cuc = (ci[out] * uc).sum(axis=1, dtype=dt)
        uuc = (uc * uc).sum(axis=1, dtype=dt)
        val[out] = -src[out] + dt(2) * ww[out] * ((ro - one) + ro * (dt(4.5) * cuc * cuc - dt(1.5) * uuc))
        new[i_dir, lk] = val
        g = new
    return found if isinstance(steps, (tuple, list)) else found[0]
