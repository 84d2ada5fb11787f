"""Oracle pins for the D3Q19 MRT operator (moment space of d'Humieres et al.
2002; the paper lists MRT among its operators, Sec. 4, and benchmarks it in
Sec. 5.1): the basis against its defining properties, and the operator
against closed forms it must reduce to -- SRT at uniform rates, TRT at
even/odd rates, conservation, the equilibrium fixed point, and the exact
Poiseuille profile at the TRT magic combination."""
import math

import numpy as np

import geometry as G
import oracle as O
from test_oracle_flows import _run_to_steady

ODD = [3, 4, 5, 6, 7, 8, 16, 17, 18]          # rows odd in c (j, q, m)
EVEN = [a for a in range(19) if a not in ODD]


def test_basis_is_orthogonal_with_the_defining_rows():
    M = O.mrt_matrix()
    c, _, inv = O.stencil(19)
    G2 = M @ M.T
    assert np.array_equal(G2, np.diag(np.diag(G2)))           # rows mutually orthogonal
    assert np.all(np.diag(G2) > 0)
    assert np.array_equal(M[0], np.ones(19))                  # density
    assert np.array_equal(M[[3, 5, 7]], c.T)                  # momentum
    # every row is even or odd under c -> -c, as classified
    for a in range(19):
        sign = -1 if a in ODD else 1
        assert np.array_equal(M[a, inv], sign * M[a])
    # the second-order rows span the traceless stress: 3xx - |c|^2, yy - zz, xy, yz, xz
    n = (c ** 2).sum(1)
    assert np.array_equal(M[9], 3 * c[:, 0] ** 2 - n)
    assert np.array_equal(M[13], c[:, 0] * c[:, 1])


def _random_cell(rng, rho=1.02, u=(0.03, -0.02, 0.01)):
    f = O.equilibrium(19, rho, np.array(u)) * (1 + 0.05 * rng.standard_normal(19))
    return f


def _collide(f, op, force, omega=1.25, rates=None, magic=3 / 16):
    g = G.channel(1, 1, 1)
    p = O.Problem.from_geometry(g, q=19, op=op, omega_plus=omega, magic=magic, force=force, mrt_rates=rates)
    return O.collide(p, f)


def test_uniform_rates_reduce_to_srt():
    rng = np.random.default_rng(1)
    for _ in range(5):
        f = _random_cell(rng)
        F = tuple(rng.uniform(-1e-4, 1e-4, 3))
        for w in (0.7, 1.25, 1.9):
            got = _collide(f, O.MRT, F, omega=w, rates=(w,) * 19)
            want = _collide(f, O.SRT, F, omega=w)
            assert np.max(np.abs(got - want)) < 1e-15


def test_even_odd_rates_reduce_to_trt():
    rng = np.random.default_rng(2)
    wp = 1.25
    wm = O.trt_omega_minus(wp, 3 / 16)
    rates = tuple(wm if a in ODD else wp for a in range(19))
    for _ in range(5):
        f = _random_cell(rng)
        F = tuple(rng.uniform(-1e-4, 1e-4, 3))
        got = _collide(f, O.MRT, F, omega=wp, rates=rates)
        want = _collide(f, O.TRT, F, omega=wp)
        assert np.max(np.abs(got - want)) < 1e-15


def test_conservation_and_fixed_point_with_default_rates():
    rng = np.random.default_rng(3)
    c, _, _ = O.stencil(19)
    F = np.array([2e-5, -1e-5, 5e-6])
    for _ in range(5):
        f = _random_cell(rng)
        fs = _collide(f, O.MRT, tuple(F))
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.max(np.abs(c.T @ fs - (c.T @ f + F))) < 1e-15
        # not SRT: the ghost moments relax at their own rates
        assert np.max(np.abs(fs - _collide(f, O.SRT, tuple(F)))) > 1e-6
    feq = O.equilibrium(19, 0.97, np.array([0.02, 0.01, -0.03]))
    assert np.max(np.abs(_collide(feq, O.MRT, (0.0, 0.0, 0.0)) - feq)) < 1e-16


def _poiseuille_mrt(h, rates, force=1e-6):
    g = G.channel(1, 1, h)
    p = O.Problem.from_geometry(g, q=19, op=O.MRT, force=(force, 0, 0), mrt_rates=rates)
    f, _ = _run_to_steady(p, O.dense_init(p), 2000, 400000, 1e-13)
    _, u = O.dense_macroscopic(p, f)
    ux = u[:, 0].reshape(h + 2)[1:-1]
    z = np.arange(1, h + 1)
    exact = force / (2 * p.nu) * (z - 0.5) * (h + 0.5 - z)
    return float(np.linalg.norm(ux - exact) / np.linalg.norm(exact))


def test_poiseuille_exact_at_the_magic_odd_rate():
    # halfway bounce-back sits exactly mid-link when the odd non-conserved
    # moments relax at omega- with (1/omega+ - 1/2)(1/omega- - 1/2) = 3/16,
    # whatever the even ghost rates
    w = 1.25
    wm = O.trt_omega_minus(w, 3 / 16)
    rates = list(O.mrt_default_rates(w))
    for a in (4, 6, 8, 16, 17, 18):
        rates[a] = wm
    assert _poiseuille_mrt(12, tuple(rates)) < 1e-9


def test_poiseuille_second_order_with_default_rates():
    hs = [8, 16, 32]
    rates = O.mrt_default_rates(1.25)
    errs = [_poiseuille_mrt(h, rates) for h in hs]
    slopes = [math.log(errs[i + 1] / errs[i]) / math.log(hs[i + 1] / hs[i]) for i in range(2)]
    assert errs[0] > 1e-6
    for s in slopes:
        assert -2.3 < s < -1.7, (errs, slopes)
