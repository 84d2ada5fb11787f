"""GPU test of sparse_lbm_compact_noalloc, the compaction entry point that
allocates nothing.

It exists for callers that own all device memory themselves (a framework with
one pre-reserved arena that forbids other allocations, or a latency-critical
loop that cannot afford cudaMalloc/cudaFree and the device-wide
synchronisation they may cause).  Such a caller passes device buffers in; the
library uses only its own fixed scratch array.

The test calls the entry point through the C ABI twice in a row, on two
different geometries (so the shared scratch holds the first call's contents
when the second starts), and checks both results against the compaction of the
existing path (sparse_lbm_create + sparse_lbm_export_lists), bit for bit, as
all integer outputs in this suite are compared; checks voxel counts that end
in a partial scan tile against a sequential scan; checks that a call leaves the
device's free memory unchanged; and checks that a size above the stated
maximum is refused before anything is launched.  The file is
named to be collected last so a failing run that stops at the first failure
has run every other test first; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import geometry as G

pytestmark = pytest.mark.gpu


def _reference_compaction(g):
    import paper_2408_06880_gb300 as P
    with P.Domain(g.flags, periodic=g.periodic, inlet_u=g.inlet_u) as d:
        lists = d.export_lists()
    return lists["n_fluid"], lists["cell_voxel"]


def _noalloc(torch, capi, flags_np, stream):
    n = flags_np.size
    flags = torch.from_numpy(flags_np.reshape(-1)).to("cuda")
    cell_id = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    cell_voxel = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    n_fluid = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    st = capi.lib().sparse_lbm_compact_noalloc(flags.data_ptr(), n, cell_id.data_ptr(), cell_voxel.data_ptr(),
                                               n_fluid.data_ptr(), stream.cuda_stream)
    capi.check(st)
    stream.synchronize()
    nf = int(n_fluid.item())
    return nf, cell_id.cpu().numpy(), cell_voxel.cpu().numpy()[:nf]


def test_noalloc_compaction_matches_existing_path_twice_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_2408_06880_gb300 import _capi as capi
    stream = torch.cuda.Stream()
    geoms = [G.boolean_spheres(96, 0.45, 21),      # 884,736 voxels: 216 scan tiles
             G.relaxed_spheres()]                   # 32^3: 8 tiles, fewer than the first call
    for g in geoms:
        nf, cid, cvx = _noalloc(torch, capi, g.flags, stream)
        ref_nf, ref_cvx = _reference_compaction(g)
        assert nf == ref_nf
        assert np.array_equal(cvx, ref_cvx)
        # cell_id is the inverse map: -1 off fluid, k at cell_voxel[k]
        fluid = g.flags.reshape(-1) == 0
        assert np.all(cid[~fluid] == -1)
        assert np.array_equal(cid[cvx], np.arange(nf))


def test_noalloc_ragged_last_tile_matches_a_sequential_scan():
    # voxel counts that are not whole 4096-voxel scan tiles: the partial last
    # tile of this path, compared with the plain sequential numbering
    torch = pytest.importorskip("torch")
    from paper_2408_06880_gb300 import _capi as capi
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(7)
    for n in (33 * 31 * 29, 4096 * 3 + 17, 4095, 1):
        flags = (rng.random(n) < 0.4).astype(np.uint8)      # 60 % fluid (flag 0)
        nf, cid, cvx = _noalloc(torch, capi, flags, stream)
        ref = np.flatnonzero(flags == 0)
        assert nf == ref.size
        assert np.array_equal(cvx, ref)
        want = np.full(n, -1, np.int64)
        want[ref] = np.arange(ref.size)
        assert np.array_equal(cid, want)


def test_noalloc_call_allocates_no_device_memory():
    # the defining property: a call (after a first one has loaded the kernels)
    # changes neither the device's free memory nor PyTorch's allocations
    torch = pytest.importorskip("torch")
    from paper_2408_06880_gb300 import _capi as capi
    stream = torch.cuda.Stream()
    g = G.boolean_spheres(64, 0.5, 5)
    n = g.flags.size
    flags = torch.from_numpy(g.flags.reshape(-1)).to("cuda")
    cell_id = torch.empty(n, dtype=torch.int32, device="cuda")
    cell_voxel = torch.empty(n, dtype=torch.int32, device="cuda")
    n_fluid = torch.empty(1, dtype=torch.int32, device="cuda")
    args = (flags.data_ptr(), n, cell_id.data_ptr(), cell_voxel.data_ptr(), n_fluid.data_ptr(), stream.cuda_stream)
    capi.check(capi.lib().sparse_lbm_compact_noalloc(*args))
    stream.synchronize()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    capi.check(capi.lib().sparse_lbm_compact_noalloc(*args))
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert int(n_fluid.item()) == int(np.count_nonzero(g.flags == 0))


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_2408_06880_gb300 import _capi as capi
    one = C.c_int32()
    dummy = C.addressof(one)
    st = capi.lib().sparse_lbm_compact_noalloc(dummy, capi.NOALLOC_MAX_VOXELS + 1, dummy, dummy, dummy, None)
    assert st == capi.EINVAL
    assert b"SLBM_NOALLOC_MAX_VOXELS" in capi.lib().sparse_lbm_last_error()
    assert capi.lib().sparse_lbm_compact_noalloc(None, 16, None, None, None, None) == capi.EINVAL
