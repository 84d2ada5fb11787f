"""The D3Q27 central-moment (CM) and cumulant operators on the GPU (two of the
operators of Sec. 4, benchmarked in Sec. 5.1): parity with the FP64 oracle
(default and custom rates; periodic, walled and inlet/outlet domains), the
rest state kept at exactly zero, FP16 storage, launch shapes and the pull
layout bit-identical, and the refusals."""
import numpy as np
import pytest

import geometry as G
import oracle as O
from helpers import gpu_domain, rel_l2

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2408_06880_gb300")

OPS = [(P.CM, O.CM), (P.CUMULANT, O.CUMULANT)]


def _mixed_bc(seed, shape):
    g = G.random_solids(shape, 0.25, seed, periodic=0b010)
    f = g.flags
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    g.inlet_u = np.random.default_rng(seed).uniform(-0.02, 0.04, (int((f == G.INLET).sum()), 3))
    return g


CASES = [
    ("periodic_spheres", lambda: G.boolean_spheres(24, 0.5, 41), (1e-5, -2e-6, 3e-6)),
    ("walled", lambda: G.random_solids((20, 17, 15), 0.3, 8, periodic=0b011, walls_z=True), (1e-5, 0, 0)),
    ("inlet_outlet", lambda: _mixed_bc(14, (24, 15, 13)), (0.0, 0.0, 0.0)),
]


def _oracle(g, op, steps, force, omega=1.25, bulk=1.0, high=1.0):
    p = O.Problem.from_geometry(g, q=27, op=op, omega_plus=omega, force=force, cm_bulk=bulk, cm_high=high)
    L = O.pull_list(p)
    return O.sparse_macroscopic(p, L, O.sparse_run(p, L, O.sparse_rest(p, L), steps))


@pytest.mark.parametrize("gop,oop", OPS, ids=["cm", "cumulant"])
@pytest.mark.parametrize("name,make,force", CASES)
def test_central_operators_match_oracle(gop, oop, name, make, force):
    g = make()
    steps = 200
    with gpu_domain(g, q=27, op=gop, omega=1.25, force=force) as d:
        d.step(steps)
        rho, u = d.macroscopic(P.ORDER_CELLS)
    rho_o, u_o = _oracle(g, oop, steps, force)
    assert rel_l2(u.T, u_o) <= 1e-5
    assert np.max(np.abs(rho - rho_o)) <= 1e-6


@pytest.mark.parametrize("gop,oop,bulk,high", [(P.CM, O.CM, 1.3, 0.8), (P.CUMULANT, O.CUMULANT, 0.7, 1.0)],
                         ids=["cm", "cumulant"])
def test_central_custom_rates_match_oracle(gop, oop, bulk, high):
    g = G.boolean_spheres(24, 0.6, 42)
    force = (2e-5, 0.0, 1e-6)
    with gpu_domain(g, q=27, op=gop, omega=1.6, force=force) as d:
        d.set_cm_rates(bulk, high)
        d.step(150)
        rho, u = d.macroscopic(P.ORDER_CELLS)
    rho_o, u_o = _oracle(g, oop, 150, force, omega=1.6, bulk=bulk, high=high)
    assert rel_l2(u.T, u_o) <= 1e-5
    assert np.max(np.abs(rho - rho_o)) <= 1e-6


@pytest.mark.parametrize("gop", [P.CM, P.CUMULANT], ids=["cm", "cumulant"])
def test_central_rest_state_stays_exactly_at_rest(gop):
    g = G.boolean_spheres(20, 0.5, 43)
    with gpu_domain(g, q=27, op=gop) as d:
        d.step(6)
        x = d.get_state()[0].view(np.float32)
    assert np.all(x == 0.0)


@pytest.mark.parametrize("gop,oop", OPS, ids=["cm", "cumulant"])
def test_central_fp16_storage_close_to_the_oracle(gop, oop):
    g = G.boolean_spheres(24, 0.5, 44)
    force = (1e-5, 0.0, 0.0)
    with gpu_domain(g, q=27, op=gop, force=force, storage=P.FP16, scale_exp=P.auto_scale_exp(2e-3)) as d:
        d.step(200)
        _, u = d.macroscopic(P.ORDER_CELLS)
    _, u_o = _oracle(g, oop, 200, force)
    assert rel_l2(u.T, u_o) <= 5e-3


@pytest.mark.parametrize("gop", [P.CM, P.CUMULANT], ids=["cm", "cumulant"])
@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
def test_central_shapes_and_pull_layout_are_bitwise_identical(gop, storage):
    g = G.boolean_spheres(32, 0.55, 45)
    kw = dict(q=27, op=gop, force=(2e-5, 1e-6, 0.0), storage=storage, scale_exp=16)
    with gpu_domain(g, **kw) as ref:
        ref.step(7)
        want = ref.macroscopic(P.ORDER_CELLS)
        state, _ = ref.get_state()
    for even, odd in (((128, 1, 0), (128, 1, 0)), ((64, 2, 0), (256, 2, 2)), ((256, 1, 0), (64, 1, 2)),
                      ((32, 2, 0), (128, 2, 0)), ((128, 1, 5), (128, 1, 5)), ((64, 1, 0), (128, 1, 3)),
                      ((128, 1, 5), (256, 1, 3))):
        with gpu_domain(g, **kw) as d:
            d.set_launch(0, *even)
            d.set_launch(1, *odd)
            d.step(7)
            assert np.array_equal(d.get_state()[0], state)
    with gpu_domain(g, layout=P.SPARSE_PULL, **kw) as d:
        d.step(7)
        got = d.macroscopic(P.ORDER_CELLS)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


@pytest.mark.parametrize("gop", [P.CM, P.CUMULANT], ids=["cm", "cumulant"])
def test_central_register_bounded_kernels_with_links(gop):
    # variant 5 (128 x 1, at most 102 registers) of both steps, with the
    # even step's link maps and the odd step's, gives the plain kernels' bits
    g = _mixed_bc(16, (24, 19, 17))
    kw = dict(q=27, op=gop, force=(0.0, 0.0, 0.0))
    with gpu_domain(g, **kw) as ref:
        ref.set_launch(0, 128, 1)
        ref.set_launch(1, 128, 1)
        ref.step(9)
        want = ref.get_state()[0]
    with gpu_domain(g, **kw) as d:
        d.set_launch(0, 128, 1, 5)
        d.set_launch(1, 128, 1, 5)
        d.step(9)
        assert np.array_equal(d.get_state()[0], want)
        assert d.device_error() == 0
        with pytest.raises(P.SlbmError):
            d.set_launch(1, 128, 1, 3)            # slots re-read: domains without links only


def test_central_checked_mode_matches_unchecked():
    g = _mixed_bc(15, (20, 14, 12))
    kw = dict(q=27, op=P.CUMULANT, force=(0.0, 0.0, 0.0))
    with gpu_domain(g, **kw) as ref:
        ref.step(9)
        want = ref.get_state()[0]
    with gpu_domain(g, **kw) as d:
        d.set_checked(True)
        d.step(9)
        assert np.array_equal(d.get_state()[0], want)


def test_central_refusals():
    g = G.boolean_spheres(16, 0.5, 2)
    for op in (P.CM, P.CUMULANT):
        with pytest.raises(P.SlbmError):
            gpu_domain(g, q=19, op=op)
        with pytest.raises(P.SlbmError):
            gpu_domain(g, q=27, op=op, layout=P.DENSE)
    with gpu_domain(g, q=27, op=P.CM) as d:
        for parity, shape in ((0, (128, 2, 2)), (0, (128, 2, 3)), (0, (64, 4, 0)), (1, (128, 2, 1)),
                              (1, (128, 1, 4)), (1, (128, 1, 6)), (0, (64, 1, 5)), (1, (128, 2, 5)),
                              (0, (128, 1, 1))):
            with pytest.raises(P.SlbmError):
                d.set_launch(parity, *shape)
        for bulk, high in ((0.0, 1.0), (1.0, 2.5), (float("nan"), 1.0)):
            with pytest.raises(P.SlbmError):
                d.set_cm_rates(bulk, high)
        d.set_cm_rates(1.5, 0.5)
        with P.Pool(27, P.FP32, capacity=2) as pool:
            with pytest.raises(P.SlbmError):
                pool.add(d)
    with gpu_domain(g, q=27, op=P.CUMULANT) as d:
        with pytest.raises(P.SlbmError):
            d.set_cm_rates(1.0, 0.9)           # the cumulant collision takes the higher rate 1
        d.set_cm_rates(0.8, 1.0)
    with gpu_domain(g, q=27, op=P.TRT) as d:
        with pytest.raises(P.SlbmError):
            d.set_cm_rates(1.0, 1.0)
