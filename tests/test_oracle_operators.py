"""Oracle pins for the D3Q27 central-moment (CM) and cumulant collisions:
the central-moment map against its definition written out here, cumulants
against the Taylor coefficients of the logarithm of the moment-generating
function (an independent route to the same numbers), the equilibrium fixed
point of the factorised equilibrium, every relaxed moment and cumulant of a
collision against its prescribed value, conservation and the force, full
relaxation (both operators then give the same equilibrium) and second-order
convergence of channel flow."""
import math
from itertools import product

import numpy as np
import pytest

import geometry as G
import oracle as O
from test_oracle_flows import poiseuille_error

C27, _, _ = O.stencil(27)
IDX = [(a, b, c) for c in range(3) for b in range(3) for a in range(3)]       # index a + 3b + 9c


def brute_central(f, u):
    d = C27 - np.asarray(u)[None, :]
    return np.array([np.sum(f * d[:, 0] ** a * d[:, 1] ** b * d[:, 2] ** c) for a, b, c in IDX])


def series_mul(x, y):
    """Product of two truncated power series in (xi_x, xi_y, xi_z), every
    exponent kept <= 2 (higher ones never feed an exponent <= 2)."""
    out = {}
    for (ka, va), (kb, vb) in product(x.items(), y.items()):
        k = tuple(p + q for p, q in zip(ka, kb))
        if max(k) <= 2:
            out[k] = out.get(k, 0.0) + va * vb
    return out


def log_mgf_cumulants(f, u):
    """Cumulants of f / rho about u: a! b! c! times the Taylor coefficients of
    ln sum_i (f_i / rho) exp(xi . (c_i - u)), from ln(1 + X) = sum_n
    (-1)^(n+1) X^n / n with the series truncated per exponent."""
    rho = f.sum()
    d = C27 - np.asarray(u)[None, :]
    X = {}
    for a, b, c in IDX:
        if a + b + c == 0:
            continue
        X[(a, b, c)] = np.sum(f / rho * d[:, 0] ** a * d[:, 1] ** b * d[:, 2] ** c) / (
            math.factorial(a) * math.factorial(b) * math.factorial(c))
    log = {}
    power = {(0, 0, 0): 1.0}
    for n in range(1, 7):
        power = series_mul(power, X)
        for k, v in power.items():
            log[k] = log.get(k, 0.0) + (-1) ** (n + 1) * v / n
    return np.array([log.get(k, 0.0) * math.factorial(k[0]) * math.factorial(k[1]) * math.factorial(k[2])
                     for k in IDX])


def factorised_equilibrium(rho, u):
    """D3Q27 equilibrium rho prod_a phi(c_a; u_a): phi(0) = 2/3 - u^2,
    phi(+-1) = (1/3 + u^2 +- u) / 2."""
    def phi(c, v):
        return 2.0 / 3.0 - v * v if c == 0 else (1.0 / 3.0 + v * v + c * v) / 2.0
    return np.array([rho * phi(cx, u[0]) * phi(cy, u[1]) * phi(cz, u[2]) for cx, cy, cz in C27])


def random_cell(seed, amp=0.02):
    rng = np.random.default_rng(seed)
    rho = 1.0 + rng.uniform(-0.03, 0.03)
    u = rng.uniform(-0.05, 0.05, 3)
    return factorised_equilibrium(rho, u) * (1.0 + amp * rng.standard_normal(27))


def problem(op, w=1.25, wb=1.0, wh=1.0, force=(0.0, 0.0, 0.0)):
    g = G.Geometry(np.zeros((1, 1, 1), np.uint8), 7)
    return O.Problem.from_geometry(g, q=27, op=op, omega_plus=w, force=force, cm_bulk=wb, cm_high=wh)


def guo_velocity(f, force):
    return (C27.T @ f + 0.5 * np.asarray(force)) / f.sum()


def test_central_moment_map_and_its_inverse():
    for seed in range(5):
        f = random_cell(seed, 0.1)
        u = np.random.default_rng(100 + seed).uniform(-0.3, 0.3, 3)
        kap = O.central_moments(f, u)
        assert np.allclose(kap, brute_central(f, u), rtol=1e-13, atol=1e-15)
        assert np.allclose(O.from_central(kap, u), f, rtol=1e-12, atol=1e-14)


def test_cumulants_are_the_log_mgf_coefficients():
    for seed in range(5):
        f = random_cell(seed, 0.05)
        p = problem(O.CUMULANT)                                  # F = 0: u = j / rho, zero first moments
        got = O.cumulants(p, f)
        want = log_mgf_cumulants(f, guo_velocity(f, (0, 0, 0)))
        order = np.array([sum(k) for k in IDX])
        assert np.allclose(got[order >= 2], want[order >= 2], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("op", [O.CM, O.CUMULANT])
def test_factorised_equilibrium_is_a_fixed_point(op):
    rng = np.random.default_rng(3)
    for w, wb, wh in ((1.25, 1.0, 1.0), (0.7, 1.6, 1.3), (1.9, 0.5, 0.8)):
        rho = 1.0 + rng.uniform(-0.05, 0.05)
        u = rng.uniform(-0.1, 0.1, 3)
        feq = factorised_equilibrium(rho, u)
        assert np.allclose(O.collide(problem(op, w, wb, wh), feq), feq, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("op", [O.CM, O.CUMULANT])
def test_conservation_and_the_force(op):
    F = (2e-4, -1e-4, 5e-5)
    for seed in range(4):
        f = random_cell(seed)
        fs = O.collide(problem(op, 1.4, 1.2, 0.9, F), f)
        assert abs(fs.sum() - f.sum()) < 1e-14
        assert np.allclose(C27.T @ fs, C27.T @ f + np.asarray(F), rtol=0, atol=1e-15)


def relaxed_second(v, eq, w, wb):
    """The prescribed second-order relaxation, written out again (moment
    indexing): trace towards 3 eq with wb, normal differences and
    off-diagonal entries towards 0 with w."""
    xx, yy, zz, xy, xz, yz = 2, 6, 18, 4, 10, 12
    v = v.copy()
    T = v[xx] + v[yy] + v[zz]
    T = T - wb * (T - 3 * eq)
    d1, d2 = (1 - w) * (v[xx] - v[yy]), (1 - w) * (v[xx] - v[zz])
    v[xx], v[yy], v[zz] = (T + d1 + d2) / 3, (T - 2 * d1 + d2) / 3, (T + d1 - 2 * d2) / 3
    for m in (xy, xz, yz):
        v[m] *= 1 - w
    return v


def test_central_moment_collision_relaxes_every_moment():
    w, wb, wh = 1.3, 1.1, 0.7
    F = (1e-4, 3e-5, -2e-5)
    order = np.array([sum(k) for k in IDX])
    for seed in range(4):
        f = random_cell(seed)
        rho, u = f.sum(), guo_velocity(f, F)
        kap = brute_central(f, u)
        fs = O.collide(problem(O.CM, w, wb, wh, F), f)
        got = brute_central(fs, u)                               # about the input's Guo velocity
        want = relaxed_second(kap, rho / 3, w, wb)
        for m, (a, b, c) in enumerate(IDX):
            if order[m] >= 3:
                eq = rho * np.prod([(1.0, 0.0, 1.0 / 3.0)[e] for e in (a, b, c)])
                want[m] = kap[m] - wh * (kap[m] - eq)
        want[0] = rho
        want[[1, 3, 9]] = 0.5 * np.asarray(F)
        assert np.allclose(got, want, rtol=1e-11, atol=1e-15)


def test_cumulant_collision_relaxes_every_cumulant():
    w, wb, wh = 1.2, 0.9, 0.6
    order = np.array([sum(k) for k in IDX])
    for seed in range(4):
        f = random_cell(seed)
        u = guo_velocity(f, (0, 0, 0))
        c0 = log_mgf_cumulants(f, u)
        fs = O.collide(problem(O.CUMULANT, w, wb, wh), f)
        c1 = log_mgf_cumulants(fs, u)
        want = relaxed_second(np.where(order >= 2, c0, 0.0), 1.0 / 3.0, w, wb)
        want[order >= 3] = (1 - wh) * c0[order >= 3]
        assert np.allclose(c1[order >= 2], want[order >= 2], rtol=1e-8, atol=1e-14)
        assert abs(fs.sum() - f.sum()) < 1e-14


def test_full_relaxation_gives_the_same_equilibrium():
    F = (1e-4, 0.0, -3e-5)
    for seed in range(3):
        f = random_cell(seed, 0.05)
        a = O.collide(problem(O.CM, 1.0, 1.0, 1.0, F), f)
        b = O.collide(problem(O.CUMULANT, 1.0, 1.0, 1.0, F), f)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-16)
        if seed == 0:                                            # F = 0: exactly the equilibrium
            g = O.collide(problem(O.CM, 1.0, 1.0, 1.0), f)
            assert np.allclose(g, factorised_equilibrium(f.sum(), guo_velocity(f, (0, 0, 0))), rtol=1e-12)


@pytest.mark.parametrize("op", [O.CM, O.CUMULANT])
def test_channel_flow_second_order(op):
    # measured slopes -1.998 and -2.000 (the same profile as SRT's at the
    # same omega for this unidirectional flow)
    hs = [4, 8, 16]
    errs = [poiseuille_error(h, op, q=27)[0] for h in hs]
    slopes = [math.log(errs[i + 1] / errs[i]) / math.log(hs[i + 1] / hs[i]) for i in range(2)]
    for s in slopes:
        assert -2.3 < s < -1.7, (errs, slopes)
