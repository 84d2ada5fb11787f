"""GPU parity through the C ABI against the FP64 oracle.

Bit-exact for the integer work (compaction order, pull index-list, link
table); for FP32 storage the velocity relative L2 over all fluid cells and
components must be <= 1e-5 (the stated tolerance), density within 1e-6."""
import numpy as np
import pytest

import geometry as G
import oracle as O
from helpers import gpu_domain, gpu_fields, oracle_fields, rel_l2, fluid_mask

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2408_06880_gb300")

U_TOL = 1e-5
RHO_TOL = 1e-6


def _mixed_bc(seed=5, shape=(12, 9, 10)):
    g = G.random_solids(shape, 0.25, seed, periodic=0b010)
    f = g.flags
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    n_in = int(np.count_nonzero(f == G.INLET))
    g.inlet_u = np.random.default_rng(seed).uniform(-0.02, 0.05, (n_in, 3))
    g.rho_out = 1.001
    return g


LIST_CASES = {
    "periodic8": lambda: G.random_solids(8, 0.3, 1, periodic=7),
    "walled": lambda: G.random_solids((9, 7, 5), 0.3, 2, periodic=0),
    "mixed_bc": _mixed_bc,
    "spheres32": lambda: G.relaxed_spheres(),
    "boolean64": lambda: G.boolean_spheres(64, 0.5, 3),
    "all_fluid": lambda: G.Geometry(np.zeros((5, 6, 7), np.uint8), 7),
}


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("case", list(LIST_CASES))
def test_lists_bit_exact(q, case):
    g = LIST_CASES[case]()
    ref = O.pull_list(O.Problem.from_geometry(g, q=q))
    with gpu_domain(g, q=q) as d:
        got = d.export_lists()
    assert got["n_fluid"] == ref.n_fluid and got["stride"] == ref.stride
    assert np.array_equal(got["cell_voxel"], ref.cell_voxel)
    assert np.array_equal(got["P"], ref.P)
    assert np.array_equal(got["link_cell"], ref.bc_cell)
    assert np.array_equal(got["link_dir"], ref.bc_dir)
    assert np.array_equal(got["link_type"], ref.bc_type)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("storage", [P.FP32, P.FP16, P.BF16])
@pytest.mark.parametrize("op", [P.SRT, P.TRT])
def test_rest_state_bitwise_zero(q, storage, op):
    g = G.random_solids(12, 0.3, 4, periodic=0b011, walls_z=True)
    with gpu_domain(g, q=q, storage=storage, op=op, scale_exp=10) as d:
        d.step(11)
        buf, step = d.get_state()
        assert step == 11
        assert not buf.any()
        rho, u = gpu_fields(d)
        m = fluid_mask(g)
        assert np.all(rho[m] == 1.0) and not u.any()


def test_small_case_parity_srt_d3q19():
    # the 32^3 sphere packing, SRT tau = 0.8, F = 1e-6 x, 200 steps, FP32
    g = G.relaxed_spheres()
    kw = dict(q=19, op=P.SRT, omega=1.25, force=(1e-6, 0.0, 0.0))
    (rho_o, u_o), _, _ = oracle_fields(g, 200, **kw)
    with gpu_domain(g, **kw) as d:
        d.step(200)
        rho_g, u_g = gpu_fields(d)
    m = fluid_mask(g)
    assert rel_l2(u_g[m], u_o[m]) <= U_TOL
    assert np.max(np.abs(rho_g[m] - rho_o[m])) <= RHO_TOL
    assert np.max(np.abs(u_o[m])) > 1e-5


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("op", [P.SRT, P.TRT])
def test_parity_forced_with_walls(q, op):
    g = G.random_solids((24, 20, 18), 0.2, 7, periodic=0b011, walls_z=True)
    kw = dict(q=q, op=op, omega=1.6, force=(2e-6, -1e-6, 5e-7))
    (rho_o, u_o), _, _ = oracle_fields(g, 60, **kw)
    with gpu_domain(g, **kw) as d:
        d.step(60)
        rho_g, u_g = gpu_fields(d)
    m = fluid_mask(g)
    assert rel_l2(u_g[m], u_o[m]) <= U_TOL
    assert np.max(np.abs(rho_g[m] - rho_o[m])) <= RHO_TOL


@pytest.mark.parametrize("q", [19, 27])
def test_parity_inlet_outlet_links(q):
    g = _mixed_bc()
    kw = dict(q=q, op=P.TRT, omega=1.25, force=(0.0, 0.0, 0.0))
    (rho_o, u_o), _, _ = oracle_fields(g, 40, **kw)
    with gpu_domain(g, **kw) as d:
        assert d.info["n_bc_links"] > 0
        d.step(40)
        rho_g, u_g = gpu_fields(d)
    m = fluid_mask(g)
    assert rel_l2(u_g[m], u_o[m]) <= U_TOL
    assert np.max(np.abs(rho_g[m] - rho_o[m])) <= RHO_TOL


@pytest.mark.parametrize("steps", [1, 7, 33])
def test_odd_parity_readout(steps):
    # after an odd number of steps the state is read through the odd-step slots
    g = _mixed_bc(9)
    kw = dict(q=19, op=P.TRT, omega=1.4, force=(1e-5, 0.0, 0.0))
    (rho_o, u_o), _, _ = oracle_fields(g, steps, **kw)
    with gpu_domain(g, **kw) as d:
        d.step(steps)
        rho_g, u_g = gpu_fields(d)
        s = d.reduce()
    m = fluid_mask(g)
    assert rel_l2(u_g[m], u_o[m]) <= U_TOL
    assert np.max(np.abs(rho_g[m] - rho_o[m])) <= RHO_TOL
    assert abs(s[4] - u_o[m, 0].sum()) <= 1e-5 * np.abs(u_o[m, 0]).sum() + 1e-12


def test_taylor_green_initialisation_parity():
    L, nz, U = 32, 4, 0.02
    rho0, u0 = G.taylor_green_fields(L, nz, U)
    g = G.Geometry(np.zeros((nz, L, L), np.uint8), 7)
    kw = dict(q=19, op=P.SRT, omega=1.25)
    (rho_o, u_o), _, _ = oracle_fields(g, 100, rho0, u0, **kw)
    with gpu_domain(g, **kw) as d:
        d.init_equilibrium(rho0, u0.T.copy(), order=P.ORDER_VOXELS)
        d.step(100)
        rho_g, u_g = gpu_fields(d)
    assert rel_l2(u_g, u_o) <= U_TOL
    assert np.max(np.abs(rho_g - rho_o)) <= RHO_TOL


def test_reductions_match_fields_and_are_deterministic():
    g = G.boolean_spheres(48, 0.5, 8)
    kw = dict(q=19, op=P.TRT, force=(1e-5, 0.0, 0.0))
    with gpu_domain(g, **kw) as d:
        d.step(50)
        s1, s2 = d.reduce(), d.reduce()
        rho, u = d.macroscopic()
    assert np.array_equal(s1, s2)
    assert abs(s1[4] - np.sum(u[0].astype(np.float64))) <= 1e-6 * np.abs(u[0]).sum()
    # momentum sum = sum rho u with the same fields
    assert abs(s1[1] - np.sum(rho.astype(np.float64) * u[0])) <= 1e-5 * np.abs(rho * u[0]).sum()
    # mass is conserved (periodic + bounce-back): sum(rho-1) stays at FP32 rounding level
    assert abs(s1[0]) < 1e-6


SHAPES = [(64, 1, 0), (128, 1, 0), (256, 1, 0), (64, 2, 0), (256, 2, 0), (128, 4, 0), (256, 4, 0),
          (64, 2, 1), (64, 4, 1), (128, 2, 1), (128, 4, 1), (64, 1, 2), (128, 1, 2), (128, 1, 3), (64, 1, 3), (128, 2, 2),
          (128, 1, 4), (64, 1, 4), (128, 2, 4), (256, 2, 4), (128, 1, 5), (256, 1, 5), (64, 1, 5),
          (128, 2, 6), (128, 3, 6), (128, 4, 6)]


@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("shape", SHAPES)
def test_launch_shapes_are_bitwise_identical(shape, q, storage):
    # every launch shape, including the bulk-staged persistent kernels, gives
    # the same bits; mixed inlet/outlet links exercise the link maps too
    g = _mixed_bc(13, (40, 33, 29)) if q == 27 else G.boolean_spheres(40, 0.5, 9)
    kw = dict(q=q, op=P.TRT, force=(1e-5, 2e-6, 0.0), storage=storage, scale_exp=20)
    with gpu_domain(g, **kw) as ref:
        ref.set_launch(0, 128, 1)
        ref.set_launch(1, 128, 1)
        ref.step(7)
        want, _ = ref.get_state()
    threads, cells, variant = shape
    with gpu_domain(g, **kw) as d:
        if variant < 2:
            d.set_launch(0, threads, cells, variant)
        d.set_launch(1, threads, cells if variant else min(cells, 2), variant)
        d.step(7)
        got, _ = d.get_state()
        assert d.device_error() == 0
    assert np.array_equal(got, want)


def _mixed_bc_residue(residue, seed=13, shape=(40, 33, 29)):
    """_mixed_bc with the last fluid voxels turned to walls until N_F mod 128
    equals `residue`: the 64-cell tiles of the padded PDF-list then end in a
    tile of padding columns only (residue <= 64), whose link range must stay
    empty without reading past the first-link table (residue <= 32)."""
    g = _mixed_bc(seed, shape)
    flat = g.flags.reshape(-1)
    fluid = np.flatnonzero(flat == G.FLUID)
    drop = (len(fluid) - residue) % 128
    flat[fluid[len(fluid) - drop:]] = G.WALL
    assert int(np.count_nonzero(flat == G.FLUID)) % 128 == residue
    return g


@pytest.mark.parametrize("residue", [1, 17, 32, 33, 64, 65])
@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
def test_even_links_with_ragged_last_tiles(residue, storage):
    # the even step's link maps, applied inside the plain, paired and
    # bulk-staged kernels, give the same bits whatever the remainder of N_F
    g = _mixed_bc_residue(residue)
    kw = dict(q=27, op=P.TRT, force=(1e-5, 2e-6, 0.0), storage=storage, scale_exp=20)
    with gpu_domain(g, **kw) as ref:
        ref.set_launch(0, 128, 1)
        ref.step(5)
        want, _ = ref.get_state()
    for shape in ((64, 1, 0), (64, 2, 1), (64, 4, 1), (128, 2, 1), (64, 2, 2), (64, 2, 3), (64, 4, 3),
                  (128, 4, 3)):
        with gpu_domain(g, **kw) as d:
            d.set_launch(0, *shape)
            d.step(5)
            got, _ = d.get_state()
            assert d.device_error() == 0
        assert np.array_equal(got, want), shape


def _all_boundary_slab(q_seed=3):
    """A 3-voxel-thick slab between a velocity inlet (x = 0) and a pressure
    outlet (x = 2), periodic in y and z: every fluid cell has links, so a
    block of the even kernels holds more links than threads."""
    nz, ny, nx = 40, 33, 3
    f = np.zeros((nz, ny, nx), np.uint8)
    f[:, :, 0] = G.INLET
    f[:, :, 2] = G.OUTLET
    rng = np.random.default_rng(q_seed)
    f[:, :, 1][rng.random((nz, ny)) < 0.2] = G.WALL
    n_in = int(np.count_nonzero(f == G.INLET))
    return G.Geometry(f, 0b110, rng.uniform(0.0, 0.03, (n_in, 3)), 1.002, {})


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
def test_even_links_more_links_than_threads(q, storage):
    # every cell a boundary cell: the even kernels' link pass walks several
    # links per thread; all even shapes give the bits of 128 x 1, and FP32
    # stays within the FP64 oracle's tolerance
    g = _all_boundary_slab()
    kw = dict(q=q, op=P.TRT, force=(0.0, 0.0, 0.0), storage=storage, scale_exp=18)
    with gpu_domain(g, **kw) as ref:
        assert ref.info["n_bc_links"] > 4 * ref.n_fluid
        ref.set_launch(0, 128, 1)
        ref.step(6)
        want, _ = ref.get_state()
        rho, u = ref.macroscopic(P.ORDER_CELLS)
    for shape in ((32, 1, 0), (64, 2, 0), (32, 4, 0), (64, 2, 2), (64, 4, 2), (64, 2, 1), (128, 2, 1), (64, 2, 3)):
        with gpu_domain(g, **kw) as d:
            d.set_launch(0, *shape)
            d.step(6)
            got, _ = d.get_state()
            assert d.device_error() == 0
        assert np.array_equal(got, want), shape
    if storage == P.FP32:
        p = O.Problem.from_geometry(g, q=q, op=O.TRT, omega_plus=1.25, magic=3 / 16, force=(0.0, 0.0, 0.0))
        L = O.pull_list(p)
        rho_o, u_o = O.sparse_macroscopic(p, L, O.sparse_run(p, L, O.sparse_rest(p, L), 6))
        assert rel_l2(u.T, u_o) <= 1e-5
        assert np.max(np.abs(rho - rho_o)) <= 1e-6


@pytest.mark.parametrize("stages", [2, 3, 4])
@pytest.mark.parametrize("case", ["sweep96_lex", "sweep96_brick", "dense96", "bed_links", "bf16"])
def test_window_staged_odd_step_over_many_tiles(case, stages):
    # odd variant 6 (index rows, own rows and neighbour windows bulk-copied
    # into a ring of shared-memory stages) on domains with many more 128-cell
    # tiles than resident CTAs, so every CTA cycles through its ring; brick-8
    # order and the near-all-fluid packing send more links outside the
    # windows (read from global memory); the bed carries inlet/outlet links
    q, storage, order = 19, P.FP32, P.ORDER_LEX
    if case == "sweep96_lex":
        g = G.boolean_spheres(96, 0.5, 9)
    elif case == "sweep96_brick":
        g, order, storage = G.boolean_spheres(96, 0.5, 9), P.ORDER_BRICK8, P.FP16
    elif case == "dense96":
        g, storage = G.boolean_spheres(96, 0.9, 14), P.FP16
    elif case == "bf16":
        g, storage = G.boolean_spheres(80, 0.7, 4), P.BF16
    else:
        g, q = G.particle_bed(96, 64, 64, bed_top=32, radius=5.0, seed=23), 27
    kw = dict(q=q, op=P.TRT, force=(1e-5, 2e-6, 0.0), storage=storage, scale_exp=20, cell_order=order)
    with gpu_domain(g, **kw) as ref:
        ref.step(9)
        want, _ = ref.get_state()
    with gpu_domain(g, **kw) as d:
        d.set_launch(1, 128, stages, 6)
        assert d.n_fluid > 400 * 128                   # many tiles per CTA
        d.step(9)
        got, _ = d.get_state()
        assert d.device_error() == 0
    assert np.array_equal(got, want)


def test_window_staged_shape_refusals():
    g = G.boolean_spheres(16, 0.5, 2)
    with gpu_domain(g, q=19, op=P.TRT) as d:
        for bad in ((64, 2, 6), (128, 1, 6), (128, 5, 6), (128, 1, 7)):
            with pytest.raises(P.SlbmError):
                d.set_launch(1, *bad)
        with pytest.raises(P.SlbmError):
            d.set_launch(0, 128, 2, 6)                  # odd step only
    with gpu_domain(g, q=19, op=P.TRT, layout=P.SPARSE_PULL) as d:
        with pytest.raises(P.SlbmError):
            d.set_launch(1, 128, 2, 6)


EVEN_PAIRED = [(64, 2, 2), (128, 2, 2), (256, 2, 2), (64, 4, 2), (256, 4, 2), (64, 2, 3), (64, 4, 3), (128, 2, 3),
               (128, 4, 3)]


@pytest.mark.parametrize("storage", [P.FP32, P.FP16, P.BF16])
@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("shape", EVEN_PAIRED)
def test_paired_collision_is_bitwise_identical(shape, q, storage):
    # the even step with cells collided in pairs (paired FP32 instructions)
    # gives the scalar collision's bits; both geometries have an odd N_F, so
    # the last pair is ragged; the D3Q27 case carries inlet/outlet links
    g = _mixed_bc(13, (40, 33, 29)) if q == 27 else G.boolean_spheres(39, 0.5, 9)
    assert int((g.flags == 0).sum()) % 2 == 1
    kw = dict(q=q, op=P.TRT, force=(1e-5, 2e-6, -1e-6), storage=storage, scale_exp=20)
    with gpu_domain(g, **kw) as ref:
        ref.set_launch(0, 128, 1)
        ref.step(9)
        want, _ = ref.get_state()
    with gpu_domain(g, **kw) as d:
        if storage == P.BF16 and shape[2] == 3:
            with pytest.raises(P.SlbmError):
                d.set_launch(0, *shape)
            return
        d.set_launch(0, *shape)
        d.step(9)
        got, _ = d.get_state()
        assert d.device_error() == 0
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape", [(64, 2, 2), (64, 4, 2), (64, 2, 3)])
def test_paired_collision_srt_and_tiny_domain(shape):
    # SRT (omega- = omega+) and a 3-cell channel: one pair plus a lone cell
    for g, q, op in ((G.boolean_spheres(24, 0.6, 4), 19, P.SRT), (G.channel(1, 1, 3), 27, P.TRT)):
        kw = dict(q=q, op=op, force=(3e-5, 0.0, 1e-6))
        with gpu_domain(g, **kw) as ref:
            ref.set_launch(0, 64, 1)
            ref.step(11)
            want, _ = ref.get_state()
        with gpu_domain(g, **kw) as d:
            d.set_launch(0, *shape)
            d.step(11)
            got, _ = d.get_state()
        assert np.array_equal(got, want)


@pytest.mark.parametrize("q", [19, 27])
def test_paired_collision_on_a_random_state(q):
    # far from equilibrium every rounding of the collision shows: one even
    # step from random populations, paired shapes against the scalar kernel
    g = G.boolean_spheres(39, 0.5, 9)
    kw = dict(q=q, op=P.TRT, force=(1e-5, 2e-6, -1e-6))
    rng = np.random.default_rng(q)
    with gpu_domain(g, **kw) as ref:
        S = ref.info["stride"]
        x = (rng.standard_normal(q * S) * 1e-2).astype(np.float32).view(np.uint8)
        ref.set_state(x, 0)
        ref.set_launch(0, 64, 1)
        ref.step(1)
        want, _ = ref.get_state()
    for shape in ((64, 2, 2), (64, 4, 2), (128, 4, 3)):
        with gpu_domain(g, **kw) as d:
            d.set_state(x, 0)
            d.set_launch(0, *shape)
            d.step(1)
            assert np.array_equal(d.get_state()[0], want), shape


def test_paired_even_shape_refusals():
    g = G.boolean_spheres(16, 0.5, 2)
    with gpu_domain(g, q=19, op=P.TRT) as d:
        for bad in ((64, 1, 2), (64, 8, 2), (96, 2, 3), (128, 3, 3), (64, 2, 5)):
            with pytest.raises(P.SlbmError):
                d.set_launch(0, *bad)


def test_graph_replay_and_checked_mode_match_plain_steps():
    g = _mixed_bc(11)
    kw = dict(q=27, op=P.TRT, force=(1e-5, 0.0, 0.0))
    with gpu_domain(g, **kw) as a:
        a.step(10)
        want, _ = a.get_state()
    with gpu_domain(g, **kw) as b:
        b.step(4, graph=True)
        b.step(3, graph=True)
        b.step(3, graph=True)
        got, _ = b.get_state()
    assert np.array_equal(got, want)
    with gpu_domain(g, **kw) as c:
        c.set_checked(True)
        c.step(10)
        assert c.device_error() == 0
        got, _ = c.get_state()
    assert np.array_equal(got, want)


def test_checkpoint_resume_is_bitwise():
    g = G.boolean_spheres(32, 0.6, 10)
    kw = dict(q=19, op=P.TRT, force=(1e-5, 0.0, 0.0))
    with gpu_domain(g, **kw) as a:
        a.step(21)
        want, _ = a.get_state()
    with gpu_domain(g, **kw) as b:
        b.step(13)
        buf, step = b.get_state()
    with gpu_domain(g, **kw) as c:
        c.set_state(buf, step)
        c.step(8)
        got, s = c.get_state()
    assert s == 21 and np.array_equal(got, want)


def test_edge_cases_empty_and_single_cell():
    solid = G.Geometry(np.ones((4, 4, 4), np.uint8), 7)
    with gpu_domain(solid) as d:
        assert d.n_fluid == 0
        d.step(5)
        assert np.array_equal(d.reduce(), np.zeros(5))
    one = np.ones((3, 3, 3), np.uint8)
    one[1, 1, 1] = 0
    g = G.Geometry(one, 7)
    kw = dict(q=19, op=P.SRT, force=(1e-4, 0, 0))
    (rho_o, u_o), _, _ = oracle_fields(g, 9, **kw)
    with gpu_domain(g, **kw) as d:
        assert d.n_fluid == 1 and d.info["stride"] == 128
        d.step(9)
        rho_g, u_g = gpu_fields(d)
    m = fluid_mask(g)
    assert np.allclose(u_g[m], u_o[m], atol=1e-9, rtol=1e-5)


def test_dense_comparator_parity():
    g = G.random_solids((20, 16, 12), 0.3, 12, periodic=0b011, walls_z=True)
    kw = dict(q=19, op=P.TRT, force=(1e-6, 0.0, 0.0))
    (rho_o, u_o), _, _ = oracle_fields(g, 50, **kw)
    with gpu_domain(g, layout=P.DENSE, **kw) as d:
        d.step(50)
        rho_g, u_g = gpu_fields(d)
        s = d.reduce()
    m = fluid_mask(g)
    assert rel_l2(u_g[m], u_o[m]) <= U_TOL
    assert np.max(np.abs(rho_g[m] - rho_o[m])) <= RHO_TOL
    assert abs(s[4] - u_o[m, 0].sum()) <= 1e-5 * np.abs(u_o[m, 0]).sum()


def _dense_vs_sparse(g, steps_list, storage=P.FP32, q=19):
    kw = dict(q=q, op=P.TRT, force=(1e-5, -2e-6, 0.0), storage=storage, scale_exp=16)
    m = fluid_mask(g)
    with gpu_domain(g, layout=P.DENSE, **kw) as dn, gpu_domain(g, **kw) as sp:
        for n in steps_list:
            dn.step(n)
            sp.step(n)
            rd, ud = dn.macroscopic(P.ORDER_VOXELS)
            rs, us = sp.macroscopic(P.ORDER_VOXELS)
            assert np.array_equal(rd[m], rs[m]) and np.array_equal(ud[:, m], us[:, m])


@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
def test_dense_comparator_is_bitwise_the_sparse_result(storage):
    # the same collision on the same values, whatever the addressing: every
    # fluid voxel's fields agree bit for bit at odd and even step counts
    # (odd box width: a thread's voxel pair straddles rows and the tail)
    g = G.random_solids((21, 16, 13), 0.35, 15, periodic=0b011, walls_z=True)
    _dense_vs_sparse(g, (1, 4, 3), storage)


def test_dense_comparator_64_bit_slots():
    # Q * N >= 2^31: the dense kernels switch to 64-bit slot offsets
    g = G.random_solids((512, 512, 440), 0.5, 16, periodic=7)
    assert 19 * g.flags.size >= 2 ** 31
    _dense_vs_sparse(g, (1, 2))


def test_invalid_calls_report_status():
    g = G.random_solids(8, 0.3, 1)
    with gpu_domain(g) as d:
        with pytest.raises(P.SlbmError):
            d.set_launch(0, 100, 1)
        with pytest.raises(P.SlbmError):
            d.set_launch(1, 128, 4)
        with pytest.raises(P.SlbmError):
            d.step(-1)


def _flip_rows(Pc, S, inv):
    """The odd-step slot R from the canonical pull list: each non-negative
    entry's row swapped between i and inverse(i)."""
    R = Pc.astype(np.int64).copy()
    for r in range(Pc.shape[0]):
        i = r + 1
        e = R[r]
        m = e >= 0
        row = e[m] // S
        R[r, m] = np.where(row == i, inv[i], i) * S + (e[m] - row * S)
    return R


@pytest.mark.parametrize("case", ["periodic_64", "mixed_bc_q27", "walled_sparse"])
def test_link_codes_decode_to_the_slot_list(case):
    # the 16-bit codes plus bases reproduce every odd-step slot exactly
    # (escapes read the int32 entry), and stepping through them (variant 4)
    # gives the same bits as the int32 list
    if case == "periodic_64":        # 131k cells: tiles at the z wrap span too wide
        g, q = G.boolean_spheres(64, 0.5, 3), 19
    elif case == "mixed_bc_q27":     # inlet/outlet links escape
        g, q = _mixed_bc(13, (40, 33, 29)), 27
    else:
        g, q = G.random_solids((96, 80, 72), 0.9, 5, periodic=0), 19
    _, _, inv = O.stencil(q)
    kw = dict(q=q, op=P.TRT, force=(1e-5, 2e-6, 0.0))
    with gpu_domain(g, **kw) as d:
        lists = d.export_lists()
        codes, bases = d.export_codes()
        S, nf = lists["stride"], lists["n_fluid"]
        R = _flip_rows(lists["P"], S, inv)
        k = np.arange(S)
        n_fluid_codes = n_escape = 0
        for r in range(q - 1):
            i = r + 1
            c = codes[r].astype(np.int64)
            b = bases[k // 128, r].astype(np.int64)
            dec = np.where((b < 0) | (c == 0xFFFE), R[r], np.where(c == 0xFFFF, i * S + k, inv[i] * S + b + c))
            assert np.array_equal(dec[:nf], R[r, :nf])
            assert np.all((c[nf:] == 0xFFFF) | (b[nf:] < 0))
            assert np.all(c[b < 0] == 0xFFFE)
            # escapes in narrow tiles are exactly the inlet/outlet links
            assert np.array_equal((c[:nf] == 0xFFFE) & (b[:nf] >= 0), (R[r, :nf] < 0) & (b[:nf] >= 0))
            n_fluid_codes += int(np.count_nonzero((c[:nf] < 0xFFFE) & (b[:nf] >= 0)))
            n_escape += int(np.count_nonzero(c[:nf] == 0xFFFE))
        assert n_fluid_codes > 0
        if case != "walled_sparse":
            assert n_escape > 0
        assert n_escape < 0.05 * nf * (q - 1)
        d.set_launch(1, 128, 1, 0)
        d.step(6)
        want, _ = d.get_state()
    with gpu_domain(g, **kw) as d:
        m0 = d.memory_bytes()
        d.set_launch(1, 128, 1, 4)              # builds the codes on first use
        assert d.memory_bytes() > m0
        d.step(6)
        got, _ = d.get_state()
    assert np.array_equal(got, want)
