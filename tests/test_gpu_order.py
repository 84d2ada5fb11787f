"""The brick-8 cell order (8^3 bricks lexicographic, voxels lexicographic
inside): device lists bit-exact against the oracle's, and every field, in
voxel order, bitwise identical to the lexicographic order's at both
parities, in FP32 and FP16, for the AA and pull layouts."""
import numpy as np
import pytest

import geometry as G
import oracle as O
from helpers import gpu_domain

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2408_06880_gb300")


def _mixed_bc(seed, shape):
    g = G.random_solids(shape, 0.25, seed, periodic=0b010)
    f = g.flags
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    g.inlet_u = np.random.default_rng(seed).uniform(-0.02, 0.04, (int((f == G.INLET).sum()), 3))
    return g


GEOMS = [
    ("partial_bricks", lambda: G.random_solids((37, 20, 27), 0.3, 5, periodic=7)),
    ("spheres", lambda: G.boolean_spheres(40, 0.5, 9)),
    ("inlet_outlet", lambda: _mixed_bc(13, (30, 17, 21))),
]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name,make", GEOMS)
def test_brick_lists_match_oracle(name, make, q):
    g = make()
    with gpu_domain(g, q=q, cell_order=P.ORDER_BRICK8) as d:
        got = d.export_lists()
    L = O.pull_list(O.Problem.from_geometry(g, q=q, order=1))
    assert got["n_fluid"] == L.n_fluid and got["stride"] == L.stride
    assert np.array_equal(got["cell_voxel"], L.cell_voxel)
    assert np.array_equal(got["P"], L.P)
    assert np.array_equal(got["link_cell"], L.bc_cell)
    assert np.array_equal(got["link_dir"], L.bc_dir)
    assert not np.array_equal(L.cell_voxel, O.pull_list(O.Problem.from_geometry(g, q=q)).cell_voxel)


@pytest.mark.parametrize("layout", [P.SPARSE, P.SPARSE_PULL])
@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
@pytest.mark.parametrize("name,make", GEOMS)
def test_brick_order_fields_equal_lexicographic(name, make, storage, layout):
    g = make()
    if layout == P.SPARSE_PULL and name == "inlet_outlet":
        pytest.skip("the pull layout has no inlet/outlet links")
    kw = dict(q=19, op=P.TRT, force=(1e-5, -2e-6, 0.0), storage=storage, scale_exp=16, layout=layout)
    with gpu_domain(g, **kw) as lex, gpu_domain(g, cell_order=P.ORDER_BRICK8, **kw) as brk:
        for n in (1, 6, 3):                       # odd, odd, even step counts
            lex.step(n)
            brk.step(n)
            rl, ul = lex.macroscopic(P.ORDER_VOXELS)
            rb, ub = brk.macroscopic(P.ORDER_VOXELS)
            assert np.array_equal(rl, rb) and np.array_equal(ul, ub)


@pytest.mark.parametrize("order", [P.ORDER_LEX, P.ORDER_BRICK8])
@pytest.mark.parametrize("name,make", GEOMS)
def test_device_lists_pass_the_host_validator(name, make, order):
    with gpu_domain(make(), q=27, cell_order=order) as d:
        d.validate_lists()


# ------------------------------------------------ hybrid order (full bricks first)
def _bed_like(seed=3):
    # 96 x 40 x 48: a random porous layer below z = 16, free flow above,
    # walls at z = 0 and z = 47, inlet x = 0, outlet x = 95, y periodic:
    # the complete all-fluid bricks of the free-flow part take the dense
    # odd step, the porous layer and the boundary bricks the sparse one
    g = G.random_solids((96, 40, 48), 0.0, seed, periodic=0b010)
    f = g.flags
    rng = np.random.default_rng(seed)
    f[1:16] = np.where(rng.random(f[1:16].shape) < 0.45, G.WALL, G.FLUID)
    f[0] = G.WALL
    f[-1] = G.WALL
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    g.inlet_u = np.tile([0.03, 0.0, 0.0], (int((f == G.INLET).sum()), 1))
    return g


HYBRID_GEOMS = GEOMS + [
    ("all_fluid_periodic", lambda: G.Geometry(np.zeros((24, 16, 40), np.uint8), 7)),
    ("bed_like", _bed_like),
]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name,make", HYBRID_GEOMS)
def test_hybrid_lists_match_oracle(name, make, q):
    g = make()
    with gpu_domain(g, q=q, cell_order=P.ORDER_HYBRID) as d:
        got = d.export_lists()
        d.validate_lists()
    L = O.pull_list(O.Problem.from_geometry(g, q=q, order=2))
    assert got["n_fluid"] == L.n_fluid and got["stride"] == L.stride
    assert np.array_equal(got["cell_voxel"], L.cell_voxel)
    assert np.array_equal(got["P"], L.P)
    assert np.array_equal(got["link_cell"], L.bc_cell)
    assert np.array_equal(got["link_dir"], L.bc_dir)


@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name,make", HYBRID_GEOMS)
def test_hybrid_order_fields_equal_lexicographic(name, make, q, storage):
    # full bricks step with neighbours by arithmetic and compact face lists,
    # the rest with the plain odd kernel: every field, in voxel order, is the
    # lexicographic order's bit for bit, at both parities
    g = make()
    kw = dict(q=q, op=P.TRT, force=(1e-5, -2e-6, 0.0), storage=storage, scale_exp=16)
    with gpu_domain(g, **kw) as lex, gpu_domain(g, cell_order=P.ORDER_HYBRID, **kw) as hyb:
        for n in (1, 6, 3):
            lex.step(n)
            hyb.step(n)
            rl, ul = lex.macroscopic(P.ORDER_VOXELS)
            rh, uh = hyb.macroscopic(P.ORDER_VOXELS)
            assert np.array_equal(rl, rh) and np.array_equal(ul, uh)
        assert hyb.device_error() == 0


def test_hybrid_bed_vs_oracle_and_shape_refusals():
    g = _bed_like(4)
    kw = dict(q=27, op=P.TRT, omega=1.25, trt_magic=3 / 16, force=(0.0, 0.0, 0.0))
    p = O.Problem.from_geometry(g, q=27, op=O.TRT, omega_plus=1.25, magic=3 / 16, order=2)
    L = O.pull_list(p)
    f = O.sparse_run(p, L, O.sparse_rest(p, L), 400)
    rho_o, u_o = O.sparse_macroscopic(p, L, f)
    with gpu_domain(g, cell_order=P.ORDER_HYBRID, **kw) as d:
        d.step(400)
        rho, u = d.macroscopic(P.ORDER_CELLS)
        with pytest.raises(P.SlbmError):
            d.set_launch(1, 128, 1, 0)
        d.set_launch(1, 128, 1, 2)
    # velocity within the FP32 target; the density, pressurised by the inlet
    # over 400 steps, drifts from FP64 by 1.04e-6 (measured), ~9 ulps of FP32
    # at rho ~ 1.003
    u = u.T.astype(np.float64)
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) <= 1e-5
    assert np.max(np.abs(rho - rho_o)) <= 2e-6
