"""The synthetic inputs on CPU: every generator follows its stated recipe
(boundary planes, periodic axes, porosity targets, inlet profiles) and is
deterministic for its seed, and the workloads have the fluid-cell counts the
measurements quote.  numpy's PCG64 stream is the same on every platform, so
these counts hold on any host."""
import numpy as np
import pytest

import geometry as G


def test_small_packing_is_the_documented_case():
    g = G.relaxed_spheres()                                   # 32^3, r = 4, porosity 0.5, seed 1
    assert g.flags.shape == (32, 32, 32) and g.periodic == 7
    assert g.meta["spheres"] == 61
    assert int(np.count_nonzero(g.flags == G.FLUID)) == 16393
    assert abs(g.porosity - 0.5) < 1e-3
    assert set(np.unique(g.flags)) == {G.FLUID, G.WALL}


@pytest.mark.parametrize("phi,seed,n_fluid", [(0.3, 11, 5031367), (0.5, 12, 8388390), (0.7, 13, 11742029),
                                              (0.9, 14, 15098365)])
def test_sweep_domains_have_the_quoted_cell_counts(phi, seed, n_fluid):
    g = G.boolean_spheres(256, phi, seed)
    nf = int(np.count_nonzero(g.flags == G.FLUID))
    assert nf == n_fluid
    assert g.porosity <= phi
    # the last sphere took the porosity below the target: at most one sphere of r = 12 below it
    assert g.porosity > phi - (4.0 / 3.0 * np.pi * 12.0 ** 3 + 1) / 256 ** 3
    assert g.periodic == 7 and set(np.unique(g.flags)) == {G.FLUID, G.WALL}


def test_boolean_model_is_deterministic_and_seeded():
    a = G.boolean_spheres(48, 0.6, 5)
    b = G.boolean_spheres(48, 0.6, 5)
    c = G.boolean_spheres(48, 0.6, 6)
    assert np.array_equal(a.flags, b.flags)
    assert not np.array_equal(a.flags, c.flags)
    assert a.meta["rmin"] == 6.0 and a.meta["rmax"] == 12.0


def test_particle_bed_follows_its_recipe():
    g = G.particle_bed()
    f = g.flags
    nz, ny, nx = f.shape
    assert (nx, ny, nz) == (512, 256, 256) and g.periodic == 2          # periodic in y only
    assert int(np.count_nonzero(f == G.FLUID)) == 23121575
    assert np.all(f[0] == G.WALL) and np.all(f[-1] == G.WALL)           # no-slip planes z = 0, 255
    inner = f[1:-1]
    assert set(np.unique(inner[:, :, 0])) <= {G.INLET, G.WALL}          # inlet plane x = 0
    assert set(np.unique(inner[:, :, -1])) <= {G.OUTLET, G.WALL}        # outlet plane x = 511
    assert not np.any(inner[:, :, 1:-1] == G.INLET) and not np.any(inner[:, :, 1:-1] == G.OUTLET)
    free = f[129:-1, :, 1:-1]                                             # above the bed: open channel
    assert np.all(free == G.FLUID)
    slab = f[1:129]
    assert np.count_nonzero(slab != G.WALL) / slab.size <= 0.4           # bed slab porosity
    n_in = int(np.count_nonzero(f == G.INLET))
    assert g.inlet_u.shape == (n_in, 3)
    assert np.all(g.inlet_u == np.array([0.05, 0.0, 0.0])) and g.rho_out == 1.0


def test_artery_tree_follows_its_recipe():
    g = G.artery_tree(256, 128, 128, r0=10.0, r_leaf=2.0)
    f = g.flags
    nz, ny, nx = f.shape
    assert g.periodic == 0 and g.meta["segments"] == 2 ** 7 - 1       # binary tree of depth 6
    assert set(np.unique(f)) == {G.FLUID, G.WALL, G.INLET, G.OUTLET}
    inlet = np.argwhere(f == G.INLET)
    assert np.all(inlet[:, 2] == 0)                                      # only on the x = 0 face
    r2 = (inlet[:, 1] - ny / 2.0) ** 2 + (inlet[:, 0] - nz / 2.0) ** 2
    assert np.all(r2 <= 10.0 ** 2)                                       # inside the root disc
    # parabolic profile along +x with peak u_max = 0.01, in ascending voxel order
    assert g.inlet_u.shape == (len(inlet), 3)
    assert np.allclose(g.inlet_u[:, 0], 0.01 * (1.0 - r2 / 100.0)) and np.all(g.inlet_u[:, 1:] == 0)
    assert np.all(np.diff(inlet[:, 0] * ny * nx + inlet[:, 1] * nx + inlet[:, 2]) > 0)
    # no fluid on a box face: every face voxel of the tree is an inlet or an outlet
    for face in (f[:, :, -1], f[:, 0, :], f[:, -1, :], f[0], f[-1], f[:, :, 0]):
        assert not np.any(face == G.FLUID)
    assert np.count_nonzero(f == G.OUTLET) > 0
    assert abs(g.meta["fluid_fraction"] - np.count_nonzero(f == G.FLUID) / f.size) < 1e-12


def test_serving_requests_follow_the_stream_recipe():
    edges = set()
    for i in range(8):
        g = G.serving_request(i)
        n = g.meta["edge"]
        edges.add(n)
        assert n in (64, 96, 128, 192) and g.flags.shape == (n, n, n) and g.meta["request"] == i
        assert g.periodic == 7 and 0.3 - 0.03 < g.porosity <= g.meta["target_porosity"] <= 0.8
        assert np.array_equal(g.flags, G.serving_request(i).flags)            # seeded by the request id
    assert len(edges) > 1
