"""Oracle pins on whole flows: closed-form solutions (Poiseuille, Couette,
Taylor-Green decay), invariants (rest state, mass, momentum balance) and a
plug-flow flux invariant for the inlet/outlet maps."""
import math

import numpy as np
import pytest

import geometry as G
import oracle as O


def _run_to_steady(p, f, chunk, max_steps, tol):
    steps = 0
    prev = None
    while steps < max_steps:
        f = O.dense_run(p, f, chunk)
        steps += chunk
        _, u = O.dense_macroscopic(p, f)
        if prev is not None and np.max(np.abs(u - prev)) <= tol * np.max(np.abs(u)):
            return f, steps
        prev = u
    return f, steps


def poiseuille_error(h, op, q=19, force=1e-6):
    g = G.channel(1, 1, h)
    p = O.Problem.from_geometry(g, q=q, op=op, force=(force, 0, 0))
    f, _ = _run_to_steady(p, O.dense_init(p), 2000, 400000, 1e-13)
    _, u = O.dense_macroscopic(p, f)
    ux = u[:, 0].reshape(h + 2)[1:-1]
    z = np.arange(1, h + 1)
    exact = force / (2 * p.nu) * (z - 0.5) * (h + 0.5 - z)
    return float(np.linalg.norm(ux - exact) / np.linalg.norm(exact)), ux, exact


@pytest.mark.parametrize("q", [19, 27])
def test_poiseuille_trt_magic_is_exact(q):
    # TRT with Lambda = 3/16 places the halfway bounce-back wall exactly,
    # so the parabola is reproduced to round-off.
    err, _, _ = poiseuille_error(12, O.TRT, q)
    assert err < 1e-9


def test_poiseuille_srt_second_order():
    hs = [8, 16, 32]
    errs = [poiseuille_error(h, O.SRT)[0] for h in hs]
    slopes = [math.log(errs[i + 1] / errs[i]) / math.log(hs[i + 1] / hs[i]) for i in range(2)]
    assert errs[0] > 1e-6          # SRT at tau = 0.8 is not exact
    for s in slopes:
        assert -2.2 < s < -1.8, (errs, slopes)


@pytest.mark.parametrize("op", [O.SRT, O.TRT])
def test_couette_moving_wall_linear_profile(op):
    # moving top wall (inlet flag = Ladd velocity wall), fixed bottom wall:
    # the steady profile is linear between the halfway walls
    h, U = 10, 1e-3
    g = G.channel(2, 2, h, top=G.INLET, top_u=(U, 0, 0))
    p = O.Problem.from_geometry(g, q=19, op=op)
    f, _ = _run_to_steady(p, O.dense_init(p), 2000, 200000, 1e-13)
    _, u = O.dense_macroscopic(p, f)
    ux = u[:, 0].reshape(h + 2, 2, 2)[1:-1, 0, 0]
    z = np.arange(1, h + 1)
    exact = U * (z - 0.5) / h
    assert np.max(np.abs(ux - exact)) < 1e-10 * U / 1e-3
    assert np.max(np.abs(u[:, 1:])) < 1e-13


def test_plug_flow_inlet_outlet_flux():
    # inlet u_in at x = 0, pressure outlet at x = L-1, periodic in y,z: the
    # steady state is the uniform plug u = u_in, rho = rho_out, which the
    # moving-wall inlet and the anti-bounce-back outlet (towards the
    # equilibrium at rho_out and the cell's velocity) reproduce exactly; the
    # exact discrete mass flux through every interface x+1/2 equals u_in.
    u_in, L = 0.01, 12
    g = G.plug_duct(L, 1, 1, u_in, rho_out=1.0)
    p = O.Problem.from_geometry(g, q=19, op=O.TRT)
    f = O.dense_run(p, O.dense_init(p), 50000)
    rho, u = O.dense_macroscopic(p, f)
    rho, ux = rho[1:-1], u[1:-1, 0]
    c, _, _ = O.stencil(19)
    plus, minus = c[:, 0] == 1, c[:, 0] == -1
    J = f[plus, 2:-1].sum(0) - f[minus, 1:-2].sum(0)
    assert np.max(np.abs(J - u_in)) < 1e-13
    assert np.max(np.abs(rho - 1.0)) < 1e-13
    assert np.max(np.abs(ux - u_in)) < 1e-13


@pytest.mark.parametrize("u_in", [0.02, 0.05])
def test_inlet_outlet_stable_at_bed_velocity(u_in):
    # an impulsively started channel with walls, inlet and outlet settles
    # (the outlet's velocity-dependent equilibrium keeps it stable at the
    # particle-bed inlet speed)
    nz, ny, nx = 18, 2, 40
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[0] = G.WALL
    fl[-1] = G.WALL
    fl[1:-1, :, 0] = G.INLET
    fl[1:-1, :, -1] = G.OUTLET
    n_in = int(np.count_nonzero(fl == G.INLET))
    g = G.Geometry(fl, 2, inlet_u=np.tile([u_in, 0.0, 0.0], (n_in, 1)), rho_out=1.0)
    p = O.Problem.from_geometry(g, q=27, op=O.TRT)
    f = O.dense_run(p, O.dense_init(p), 4000)
    _, u = O.dense_macroscopic(p, f)
    assert np.all(np.isfinite(u)) and np.max(np.abs(u)) < 3 * u_in


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("op", [O.SRT, O.TRT])
def test_rest_state_is_invariant(q, op):
    g = G.random_solids(8, 0.3, 3, periodic=0b011, walls_z=True)
    p = O.Problem.from_geometry(g, q=q, op=op)
    f0 = O.dense_init(p)
    f = O.dense_run(p, f0, 50)
    assert np.max(np.abs(f - f0)) < 1e-15


def test_mass_conserved_with_bounce_back_and_force():
    g = G.relaxed_spheres()         # the 32^3 sphere packing, periodic + walls
    p = O.Problem.from_geometry(g, q=19, op=O.SRT, force=(1e-6, 0, 0))
    f0 = O.dense_init(p)
    m0 = f0.sum()
    f = O.dense_run(p, f0, 200)
    assert abs(f.sum() - m0) / m0 < 1e-12
    assert np.max(np.abs(O.dense_macroscopic(p, f)[1][:, 0])) > 1e-5   # it did flow


@pytest.mark.parametrize("q", [19, 27])
def test_momentum_grows_by_force_in_periodic_box(q):
    # no walls: each step adds exactly F of momentum per fluid cell
    c, _, _ = O.stencil(q)
    F = np.array([2e-5, -1e-5, 5e-6])
    g = G.Geometry(np.zeros((6, 5, 4), np.uint8), 7)
    p = O.Problem.from_geometry(g, q=q, op=O.TRT, force=tuple(F))
    n = 7
    f = O.dense_run(p, O.dense_init(p), n)
    mom = c.T.astype(float) @ f.sum(axis=1)
    # exact up to the rounding of summing O(1) populations
    assert np.allclose(mom, n * p.n * F, rtol=0, atol=64 * 2.2e-16 * p.n * n)


def tg_decay_error(L, op):
    U = 0.02 * 16 / L
    nz = 2
    rho, u = G.taylor_green_fields(L, nz, U)
    g = G.Geometry(np.zeros((nz, L, L), np.uint8), 7)
    p = O.Problem.from_geometry(g, q=19, op=op)
    f = O.dense_init(p, rho, u)
    t1, t2 = int(20 * (L / 16) ** 2), int(120 * (L / 16) ** 2)
    f = O.dense_run(p, f, t1)
    e1 = np.sum(O.dense_macroscopic(p, f)[1] ** 2)
    f = O.dense_run(p, f, t2 - t1)
    e2 = np.sum(O.dense_macroscopic(p, f)[1] ** 2)
    k = 2 * math.pi / L
    rate = math.log(e1 / e2) / (t2 - t1)
    return abs(rate / (4 * p.nu * k * k) - 1.0)


@pytest.mark.parametrize("op", [O.SRT, O.TRT])
def test_taylor_green_decay_second_order(op):
    errs = [tg_decay_error(L, op) for L in (16, 32, 64)]
    assert errs[0] < 2e-2
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.5, errs


def test_permeability_of_slit_closed_form():
    # slit of height h between halfway walls, N counts the wall planes too:
    # the discrete parabola sums to F/(2 nu) * h(2h^2+1)/12 over the h fluid
    # planes, so k = nu U_D / F = h(2h^2+1) / (24 (h+2))
    h = 12
    g = G.channel(1, 1, h)
    p = O.Problem.from_geometry(g, q=19, op=O.TRT, force=(1e-6, 0, 0))
    f, _ = _run_to_steady(p, O.dense_init(p), 2000, 400000, 1e-13)
    red = O.reductions(p, f)
    k = O.permeability(p, red[4])
    assert abs(k / (h * (2 * h * h + 1) / (24 * (h + 2))) - 1) < 1e-8
