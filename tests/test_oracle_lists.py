"""Oracle pins for the sparse data structure (Sec. 3.1, 3.1.1): the compacted
cell order and the pull index-list, against brute force written here in pure
Python and against structural invariants; plus bitwise equality of the sparse
pull stepper with the dense push stepper on tiny domains."""
import numpy as np
import pytest

import geometry as G
import oracle as O

# Directions written out again for the brute force (independent of the
# oracle's C table); the test checks the two agree.
DIRS19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
          (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
          (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
DIRS27 = DIRS19 + [(1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1), (1, -1, 1), (-1, 1, -1),
                   (-1, 1, 1), (1, -1, -1)]


def visiting_order(nx, ny, nz, brick, flags=None):
    """Voxels (x, y, z) in cell-numbering order: lexicographic (0), brick-8
    (1: 8^3 bricks lexicographic, voxels lexicographic inside each brick), or
    full bricks first (2: the bricks of 512 fluid voxels in brick-8 order,
    then every other voxel in brick-8 order)."""
    if not brick:
        return [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
    bricks = []
    for bz in range(0, nz, 8):
        for by in range(0, ny, 8):
            for bx in range(0, nx, 8):
                vox = [(x, y, z) for z in range(bz, min(bz + 8, nz)) for y in range(by, min(by + 8, ny))
                       for x in range(bx, min(bx + 8, nx))]
                bricks.append(vox)
    if brick == 1:
        return [v for b in bricks for v in b]
    full = [len(b) == 512 and all(flags[z, y, x] == G.FLUID for x, y, z in b) for b in bricks]
    return [v for b, f in zip(bricks, full) if f for v in b] + [v for b, f in zip(bricks, full) if not f for v in b]


def brute_force_lists(g, q, brick=0):
    dirs = DIRS19 if q == 19 else DIRS27
    nz, ny, nx = g.flags.shape
    fl = g.flags
    order = [(x, y, z) for x, y, z in visiting_order(nx, ny, nz, brick, fl) if fl[z, y, x] == G.FLUID]
    index = {v: k for k, v in enumerate(order)}
    nf = len(order)
    S = (nf + 127) // 128 * 128
    P = np.full((q - 1, S), np.iinfo(np.int32).min, np.int64)
    links = []
    for k, (x, y, z) in enumerate(order):
        for i in range(1, q):
            cx, cy, cz = dirs[i]
            nbr = [x - cx, y - cy, z - cz]
            outside = False
            for a, n in enumerate((nx, ny, nz)):
                if nbr[a] < 0 or nbr[a] >= n:
                    if g.periodic >> a & 1:
                        nbr[a] %= n
                    else:
                        outside = True
            inv = dirs.index((-cx, -cy, -cz))
            t = G.WALL if outside else fl[nbr[2], nbr[1], nbr[0]]
            if t == G.FLUID:
                P[i - 1, k] = i * S + index[tuple(nbr)]
            elif t == G.WALL:
                P[i - 1, k] = inv * S + k
            else:
                P[i - 1, k] = -(len(links) + 1)
                links.append((k, i, int(t)))
    return order, S, P, links


def _mixed_geometry(seed):
    g = G.random_solids((5, 4, 6), 0.3, seed, periodic=0b010)
    f = g.flags
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    n_in = int(np.count_nonzero(f == G.INLET))
    g.inlet_u = np.random.default_rng(seed).uniform(-0.05, 0.05, (n_in, 3))
    return g


CASES = [
    ("periodic", lambda s: G.random_solids(4, 0.35, s, periodic=7)),
    ("walled", lambda s: G.random_solids((4, 5, 3), 0.3, s, periodic=0)),
    ("mixed_bc", _mixed_geometry),
]


BRICK_CASES = [
    ("brick_periodic", lambda s: G.random_solids((19, 10, 17), 0.35, s, periodic=7)),
    ("brick_mixed_bc", lambda s: _mixed_geometry(s)),
]


def _half_solid(seed):
    # 24 x 17 x 20 box: solids only in the lower z layers and in one corner,
    # so some complete bricks are all fluid (full) and others not; partial
    # bricks at the high faces; inlet/outlet planes at x = 0 and x = 23
    g = G.random_solids((24, 17, 20), 0.0, seed, periodic=0b010)
    f = g.flags
    rng = np.random.default_rng(seed)
    f[:6] = np.where(rng.random(f[:6].shape) < 0.4, G.WALL, G.FLUID)
    f[14:, 10:, 16:] = G.WALL
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    g.inlet_u = rng.uniform(-0.05, 0.05, (int(np.count_nonzero(f == G.INLET)), 3))
    return g


HYBRID_CASES = [
    ("hybrid_periodic", lambda s: G.random_solids((16, 24, 17), 0.0 if s == 0 else 0.004, s, periodic=7)),
    ("hybrid_half_solid", _half_solid),
]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name,make,brick", [c + (0,) for c in CASES] + [c + (1,) for c in BRICK_CASES] +
                         [c + (2,) for c in HYBRID_CASES])
def test_lists_match_brute_force(q, name, make, brick):
    c, _, _ = O.stencil(q)
    assert [tuple(v) for v in c] == (DIRS19 if q == 19 else DIRS27)
    for seed in range(3):
        g = make(seed)
        p = O.Problem.from_geometry(g, q=q, order=brick)
        L = O.pull_list(p)
        order, S, P, links = brute_force_lists(g, q, brick)
        nz, ny, nx = g.flags.shape
        assert L.n_fluid == len(order) and L.stride == S
        assert np.array_equal(L.cell_voxel, [x + nx * (y + ny * z) for x, y, z in order])
        assert np.array_equal(L.P, P)
        assert [(int(a), int(b), int(t)) for a, b, t in zip(L.bc_cell, L.bc_dir, L.bc_type)] == links
        # cell_id is the inverse of cell_voxel
        assert np.array_equal(L.cell_id[L.cell_voxel], np.arange(L.n_fluid))
        assert np.count_nonzero(L.cell_id >= 0) == L.n_fluid


def _aa_read_slot(P, i, k, S, inv):
    """AA odd-step read slot R(i,k): the pull entry with its row flipped
    between i and inverse(i)."""
    e = int(P[i - 1, k])
    row = e // S
    other = inv[i] if row == i else i
    return other * S + (e - row * S)


@pytest.mark.parametrize("q", [19, 27])
def test_list_invariants_on_sphere_packing(q):
    g = G.relaxed_spheres()          # 32^3, r = 4, phi ~ 0.5
    p = O.Problem.from_geometry(g, q=q)
    L = O.pull_list(p)
    S, nf, P = L.stride, L.n_fluid, L.P
    _, _, inv = O.stencil(q)
    assert nf == np.count_nonzero(g.flags == G.FLUID)
    assert P.shape == (q - 1, S)                       # N_F (Q-1) entries + padding
    assert np.all(P[:, nf:] == O.PAD)
    rows = P[:, :nf] // S
    cols = P[:, :nf] - rows * S
    for i in range(1, q):
        r, cc = rows[i - 1], cols[i - 1]
        fluid = r == i
        wall = r == inv[i]
        assert np.all(fluid | wall)
        # no-slip links pull the same cell's inverse direction (Sec. 3.1.1)
        assert np.array_equal(cc[wall], np.arange(nf)[wall])
        # reciprocity: if k pulls direction i from n, n pulls inverse(i) from k
        ks = np.arange(nf)[fluid]
        ns = cc[fluid]
        back = P[inv[i] - 1, ns]
        assert np.array_equal(back, inv[i] * S + ks)
    # the AA odd-step read slots of all cells and directions 1..Q-1 are a
    # permutation of the non-centre slots: every slot read (and written) once
    slots = np.concatenate([[_aa_read_slot(P, i, k, S, inv) for k in range(nf)]
                            for i in range(1, q)])
    expect = np.concatenate([i * S + np.arange(nf) for i in range(1, q)])
    assert np.array_equal(np.sort(slots), np.sort(expect))


SPARSE_DENSE = [
    ("periodic_srt", lambda: G.random_solids(8, 0.3, 11, periodic=7), O.SRT),
    ("walled_trt", lambda: G.random_solids(8, 0.25, 12, periodic=0b011, walls_z=True), O.TRT),
    ("mixed_bc_trt", lambda: _mixed_geometry(13), O.TRT),
    ("partial_bricks_trt", lambda: G.random_solids((19, 10, 17), 0.3, 14, periodic=0b101), O.TRT),
    ("full_bricks_trt", lambda: _half_solid(15), O.TRT),
]


@pytest.mark.parametrize("brick", [0, 1, 2])
@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name,make,op", SPARSE_DENSE)
def test_sparse_equals_dense_bitwise(q, name, make, op, brick):
    g = make()
    p = O.Problem.from_geometry(g, q=q, op=op, force=(1e-5, -2e-6, 3e-6), order=brick)
    rng = np.random.default_rng(5)
    n = p.n
    rho = 1.0 + rng.uniform(-0.01, 0.01, n)
    u = rng.uniform(-0.02, 0.02, (n, 3))
    f0 = O.dense_init(p, rho, u)
    L = O.pull_list(p)
    fd = O.dense_run(p, f0, 10)
    fs = O.sparse_run(p, L, O.sparse_from_dense(L, f0), 10)
    got = fs[:, :L.n_fluid]
    want = fd[:, L.cell_voxel]
    assert np.array_equal(got, want)          # bit for bit
    assert not np.array_equal(want, f0[:, L.cell_voxel])
    # the PDF-list readout equals the dense readout on the fluid voxels
    rs, us = O.sparse_macroscopic(p, L, fs)
    rd, ud = O.dense_macroscopic(p, fd)
    assert np.array_equal(rs, rd[L.cell_voxel]) and np.array_equal(us, ud[L.cell_voxel])


def test_sparse_rest_state_is_the_dense_rest_state():
    g = G.random_solids(6, 0.3, 4)
    p = O.Problem.from_geometry(g, q=27)
    L = O.pull_list(p)
    assert np.array_equal(O.sparse_rest(p, L), O.sparse_from_dense(L, O.dense_init(p)))


def test_host_list_validator_accepts_valid_and_rejects_planted_mistakes():
    # the package's host-side validator on the oracle's lists; mistakes are
    # planted in copies of the oracle's list
    from paper_2408_06880_gb300.domain import validate_pull_list
    for q in (19, 27):
        g = _mixed_geometry(7)
        L = O.pull_list(O.Problem.from_geometry(g, q=q))
        nl = int(L.bc_cell.size)
        validate_pull_list(L.P, L.n_fluid, nl)
        S = L.stride
        for r, k, v in ((0, 0, (q + 3) * S),            # beyond the list
                        (2, 1, 3 * S + L.n_fluid),       # fluid column past N_F
                        (4, 2, -(nl + 1)),               # link id out of range
                        (1, 0, 1 * S + 0 + 5 * S)):      # wall slot of another row
            bad = L.P.copy()
            bad[r, k] = v
            with pytest.raises(ValueError):
                validate_pull_list(bad, L.n_fluid, nl)
        bad = L.P.copy()
        bad[0, -1] = 0                                     # padding overwritten
        if L.n_fluid < S:
            with pytest.raises(ValueError):
                validate_pull_list(bad, L.n_fluid, nl)


# ------------------------------------------- stored oracle values (tests/golden)
def test_stored_oracle_fixtures_match_their_recipes():
    # the fixtures the long GPU parity tests compare with were written by
    # tests/golden/make_oracle_fixtures.py from the oracle: their sizes and
    # seeded cell samples follow the recipe, and the first chunk of a stored
    # serving trajectory is what the oracle computes now
    import json
    import os
    import geometry as G
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    for name, nf in (("sweep256_phi05_trt_1000.npz", 8388390), ("bed_full_q27_200.npz", 23121575)):
        fx = np.load(os.path.join(here, name))
        assert int(fx["n_fluid"]) == nf
        want = np.sort(np.random.default_rng(2408).choice(nf, size=32768, replace=False))
        assert np.array_equal(fx["cells"], want)
        assert fx["u"].shape == (32768, 3) and np.all(np.isfinite(fx["u"]))
    with open(os.path.join(here, "serving16_oracle.json")) as f:
        ref = json.load(f)
    assert [r["rid"] for r in ref["requests"]] == [2, 3, 7, 8, 10, 12, 14, 15, 16, 20, 21, 25, 26, 29, 31, 34]
    o = next(r for r in ref["requests"] if r["rid"] == 26)         # the smallest request
    g = G.serving_request(26)
    p = O.Problem.from_geometry(g, q=19, op=O.TRT, omega_plus=1.25, magic=3 / 16, force=(1e-6, 0.0, 0.0))
    L = O.pull_list(p)
    f = O.sparse_run(p, L, O.sparse_rest(p, L), 100)
    _, u = O.sparse_macroscopic(p, L, f)
    assert float(np.sum(u[:, 0])) == o["sum_ux"][0]
    # the packing fixture (the storage-accuracy report) is the oracle's run, bit for bit
    fx = np.load(os.path.join(here, "packing32_srt_200.npz"))
    g = G.relaxed_spheres()
    p = O.Problem.from_geometry(g, q=19, op=O.SRT, omega_plus=1.25, force=(1e-6, 0.0, 0.0))
    L = O.pull_list(p)
    rho, u = O.sparse_macroscopic(p, L, O.sparse_run(p, L, O.sparse_rest(p, L), int(fx["steps"])))
    assert np.array_equal(fx["rho"], rho) and np.array_equal(fx["u"], u) and float(fx["nu"]) == p.nu
