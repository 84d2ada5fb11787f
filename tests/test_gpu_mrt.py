"""The D3Q19 MRT operator on the GPU (Sec. 4's operator family, Sec. 5.1's
benchmark): parity with the FP64 oracle's MRT (default and custom rates,
periodic, walled and inlet/outlet domains), FP16 storage, launch shapes and
the pull layout bit-identical, and the refusals."""
import numpy as np
import pytest

import geometry as G
import oracle as O
from helpers import gpu_domain, rel_l2

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2408_06880_gb300")


def _mixed_bc(seed, shape):
    g = G.random_solids(shape, 0.25, seed, periodic=0b010)
    f = g.flags
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    g.inlet_u = np.random.default_rng(seed).uniform(-0.02, 0.04, (int((f == G.INLET).sum()), 3))
    return g


CASES = [
    ("periodic_spheres", lambda: G.boolean_spheres(24, 0.5, 31), (1e-5, -2e-6, 3e-6)),
    ("walled", lambda: G.random_solids((20, 17, 15), 0.3, 7, periodic=0b011, walls_z=True), (1e-5, 0, 0)),
    ("inlet_outlet", lambda: _mixed_bc(13, (24, 15, 13)), (0.0, 0.0, 0.0)),
]


def _oracle(g, steps, force, rates=None, omega=1.25):
    p = O.Problem.from_geometry(g, q=19, op=O.MRT, omega_plus=omega, force=force, mrt_rates=rates)
    L = O.pull_list(p)
    return O.sparse_macroscopic(p, L, O.sparse_run(p, L, O.sparse_rest(p, L), steps))


@pytest.mark.parametrize("name,make,force", CASES)
def test_mrt_matches_oracle(name, make, force):
    g = make()
    steps = 200
    with gpu_domain(g, q=19, op=P.MRT, omega=1.25, force=force) as d:
        d.step(steps)
        rho, u = d.macroscopic(P.ORDER_CELLS)
    rho_o, u_o = _oracle(g, steps, force)
    assert rel_l2(u.T, u_o) <= 1e-5
    assert np.max(np.abs(rho - rho_o)) <= 1e-6


def test_mrt_custom_rates_match_oracle():
    g = G.boolean_spheres(24, 0.6, 32)
    force = (2e-5, 0.0, 1e-6)
    rates = np.array([0, 1.5, 1.1, 0, 1.7, 0, 1.7, 0, 1.7, 1.6, 1.3, 1.6, 1.3, 1.6, 1.6, 1.6, 1.9, 1.9, 1.9])
    with gpu_domain(g, q=19, op=P.MRT, omega=1.6, force=force) as d:
        d.set_mrt_rates(rates)
        d.step(150)
        rho, u = d.macroscopic(P.ORDER_CELLS)
    rho_o, u_o = _oracle(g, 150, force, rates=tuple(rates), omega=1.6)
    assert rel_l2(u.T, u_o) <= 1e-5
    assert np.max(np.abs(rho - rho_o)) <= 1e-6


def test_mrt_fp16_storage_close_to_the_oracle():
    g = G.boolean_spheres(24, 0.5, 33)
    force = (1e-5, 0.0, 0.0)
    with gpu_domain(g, q=19, op=P.MRT, force=force, storage=P.FP16, scale_exp=P.auto_scale_exp(2e-3)) as d:
        d.step(200)
        _, u = d.macroscopic(P.ORDER_CELLS)
    _, u_o = _oracle(g, 200, force)
    assert rel_l2(u.T, u_o) <= 5e-3


@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
def test_mrt_shapes_and_pull_layout_are_bitwise_identical(storage):
    g = G.boolean_spheres(32, 0.55, 34)
    kw = dict(q=19, op=P.MRT, force=(2e-5, 1e-6, 0.0), storage=storage, scale_exp=16)
    with gpu_domain(g, **kw) as ref:
        ref.step(7)
        want = ref.macroscopic(P.ORDER_CELLS)
        state, _ = ref.get_state()
    for even, odd in (((128, 1, 0), (128, 1, 0)), ((64, 2, 0), (256, 2, 2)), ((256, 1, 0), (64, 1, 2)),
                      ((64, 2, 2), (128, 1, 2)), ((256, 2, 2), (128, 2, 0)), ((128, 1, 5), (128, 1, 5)),
                      ((64, 2, 2), (128, 1, 3))):
        with gpu_domain(g, **kw) as d:
            d.set_launch(0, *even)
            d.set_launch(1, *odd)
            d.step(7)
            assert np.array_equal(d.get_state()[0], state)
    with gpu_domain(g, layout=P.SPARSE_PULL, **kw) as d:
        d.step(7)
        got = d.macroscopic(P.ORDER_CELLS)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_mrt_paired_collision_on_a_random_state():
    # one even step from random populations: the paired MRT collision gives
    # the scalar one's bits
    g = G.boolean_spheres(39, 0.5, 9)
    kw = dict(q=19, op=P.MRT, force=(1e-5, 2e-6, -1e-6))
    rng = np.random.default_rng(5)
    with gpu_domain(g, **kw) as ref:
        S = ref.info["stride"]
        x = (rng.standard_normal(19 * S) * 1e-2).astype(np.float32).view(np.uint8)
        ref.set_state(x, 0)
        ref.set_launch(0, 64, 1)
        ref.step(1)
        want, _ = ref.get_state()
    with gpu_domain(g, **kw) as d:
        d.set_state(x, 0)
        d.set_launch(0, 64, 2, 2)
        d.step(1)
        assert np.array_equal(d.get_state()[0], want)


def test_mrt_refusals():
    g = G.boolean_spheres(16, 0.5, 2)
    with pytest.raises(P.SlbmError):
        gpu_domain(g, q=27, op=P.MRT)
    with pytest.raises(P.SlbmError):
        gpu_domain(g, q=19, op=P.MRT, layout=P.DENSE)
    with gpu_domain(g, q=19, op=P.MRT) as d:
        with pytest.raises(P.SlbmError):
            d.set_launch(1, 128, 2, 1)
        with pytest.raises(P.SlbmError):
            d.set_launch(0, 128, 4, 2)     # MRT pairs: 2 cells per thread
        with pytest.raises(P.SlbmError):
            d.set_launch(0, 128, 2, 3)     # no staged MRT kernel
        with pytest.raises(P.SlbmError):
            d.set_mrt_rates(np.full(19, 2.5))
        with P.Pool(19, P.FP32, capacity=2) as pool:
            with pytest.raises(P.SlbmError):
                pool.add(d)
    with gpu_domain(g, q=19, op=P.TRT) as d:
        with pytest.raises(P.SlbmError):
            d.set_mrt_rates(np.full(19, 1.0))
