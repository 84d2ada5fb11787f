"""Oracle pins, per cell: the velocity sets, the equilibrium (Eq. 6), the Guo
source, and the collision (Eq. 3 with Eq. 5 / TRT) against closed-form moment
identities.  A wrong weight, sign, index or a dropped term breaks one of these.
"""
import itertools

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("q", [19, 27])
def test_velocity_set_isotropy(q):
    c, w, inv = O.stencil(q)
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), d / 3.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(fourth, iso, atol=1e-16)
    # inverse directions
    assert np.array_equal(c[inv], -c)
    assert inv[0] == 0
    # the set is exactly the vectors of {-1,0,1}^3 with |c|^2 <= 2 (Q19) or all (Q27)
    allv = {v for v in itertools.product((-1, 0, 1), repeat=3)
            if q == 27 or sum(x * x for x in v) <= 2}
    assert {tuple(v) for v in c} == allv and len(c) == q


def test_d3q19_is_prefix_of_d3q27():
    c19, _, inv19 = O.stencil(19)
    c27, _, inv27 = O.stencil(27)
    assert np.array_equal(c19, c27[:19])
    assert np.array_equal(inv19, inv27[:19])


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_moments(q):
    c, w, _ = O.stencil(q)
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        feq = O.equilibrium(q, rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
        pi = np.einsum("ia,ib,i->ab", c, c, feq)
        assert np.allclose(pi, rho * (np.outer(u, u) + np.eye(3) / 3.0), atol=1e-14)
    # at rest the equilibrium is the weights
    assert np.allclose(O.equilibrium(q, 1.0, [0, 0, 0]), w, atol=0)


@pytest.mark.parametrize("q", [19, 27])
def test_guo_source_moments(q):
    c, _, _ = O.stencil(q)
    rng = np.random.default_rng(4)
    u = rng.uniform(-0.1, 0.1, 3)
    F = rng.uniform(-1e-3, 1e-3, 3)
    S = O.guo_source(q, u, F)
    assert abs(S.sum()) < 1e-17
    assert np.allclose(c.T @ S, F, atol=1e-18)
    second = np.einsum("ia,ib,i->ab", c, c, S)
    assert np.allclose(second, np.outer(u, F) + np.outer(F, u), atol=1e-17)


def _prob(q, op, F=(0, 0, 0), omega=1.25, magic=3 / 16):
    return O.Problem(flags=np.zeros((1, 1, 1), np.uint8), q=q, op=op, force=F,
                     omega_plus=omega, magic=magic)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("op", [O.SRT, O.TRT])
def test_collision_conservation_and_momentum_kick(q, op):
    c, _, _ = O.stencil(q)
    rng = np.random.default_rng(5)
    F = np.array([1e-4, -2e-4, 3e-5])
    p = _prob(q, op, F)
    f = O.equilibrium(q, 1.02, [0.03, -0.01, 0.02]) + rng.uniform(-1e-3, 1e-3, q)
    fs = O.collide(p, f)
    assert abs(fs.sum() - f.sum()) < 1e-15
    # Guo: post-collision momentum = pre-collision momentum + F
    assert np.allclose(c.T @ fs, c.T @ f + F, atol=1e-16)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("op", [O.SRT, O.TRT])
def test_equilibrium_is_fixed_point(q, op):
    p = _prob(q, op)
    feq = O.equilibrium(q, 0.97, [0.02, 0.01, -0.03])
    assert np.allclose(O.collide(p, feq), feq, atol=1e-16)


@pytest.mark.parametrize("q", [19, 27])
def test_trt_with_equal_rates_is_srt(q):
    omega = 1.25
    magic = (1.0 / omega - 0.5) ** 2            # makes omega- == omega+
    assert abs(O.trt_omega_minus(omega, magic) - omega) < 1e-14
    rng = np.random.default_rng(6)
    f = O.equilibrium(q, 1.0, [0.05, 0, 0]) + rng.uniform(-1e-3, 1e-3, q)
    F = (1e-4, 0, 2e-5)
    srt = O.collide(_prob(q, O.SRT, F, omega), f)
    trt = O.collide(_prob(q, O.TRT, F, omega, magic), f)
    assert np.allclose(srt, trt, atol=1e-16, rtol=0)


def test_trt_magic_parameter():
    wp = 1.25
    wm = O.trt_omega_minus(wp, 3 / 16)
    assert abs((1 / wp - 0.5) * (1 / wm - 0.5) - 3 / 16) < 1e-15
    assert abs(1 / wm - 1.125) < 1e-14


@pytest.mark.parametrize("q", [19, 27])
def test_srt_relaxes_nonequilibrium_by_one_minus_omega(q):
    # SRT (Eq. 5) without force: f_i - f_i^eq is scaled by (1 - omega)
    omega = 1.25
    p = _prob(q, O.SRT, omega=omega)
    c, w, _ = O.stencil(q)
    rng = np.random.default_rng(7)
    # a non-equilibrium part with zero mass and momentum keeps rho, u fixed
    g = rng.uniform(-1e-3, 1e-3, q)
    A = np.vstack([np.ones(q), c.T.astype(float)])
    g -= A.T @ np.linalg.solve(A @ A.T, A @ g)
    feq = O.equilibrium(q, 1.0, [0.01, 0.02, 0.0])
    fs = O.collide(p, feq + g)
    assert np.allclose(fs - feq, (1 - omega) * g, atol=1e-16)
