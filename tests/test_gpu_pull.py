"""The two-grid pull layout (the comparison scheme of Sec. 5.1): against the
FP64 oracle's sparse pull stepper, bit for bit against the AA layout at every
step count and storage, under graph replay and checkpoint/resume, and its
refusals."""
import numpy as np
import pytest

import geometry as G
import oracle as O
from helpers import gpu_domain, rel_l2

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2408_06880_gb300")

CASES = [
    ("periodic_spheres", lambda: G.boolean_spheres(24, 0.5, 31)),
    ("walled", lambda: G.random_solids((20, 17, 15), 0.3, 7, periodic=0b011, walls_z=True)),
]


@pytest.mark.parametrize("q,op", [(19, P.TRT), (27, P.SRT)])
@pytest.mark.parametrize("name,make", CASES)
def test_pull_matches_oracle(name, make, q, op):
    g = make()
    force = (1e-5, -2e-6, 3e-6)
    steps = 200
    with gpu_domain(g, q=q, op=op, omega=1.25, trt_magic=3 / 16, force=force, layout=P.SPARSE_PULL) as d:
        d.step(steps)
        rho, u = d.macroscopic(P.ORDER_CELLS)
    p = O.Problem.from_geometry(g, q=q, op=O.TRT if op == P.TRT else O.SRT, omega_plus=1.25, magic=3 / 16,
                                force=force)
    L = O.pull_list(p)
    rho_o, u_o = O.sparse_macroscopic(p, L, O.sparse_run(p, L, O.sparse_rest(p, L), steps))
    assert rel_l2(u.T, u_o) <= 1e-5
    assert np.max(np.abs(rho - rho_o)) <= 1e-6


@pytest.mark.parametrize("storage", [P.FP32, P.FP16, P.BF16])
def test_pull_is_bitwise_the_aa_result(storage):
    # the same collision on the same inputs at every step: identical fields
    # and sums after any number of steps, including the first (in-place) one
    g = G.boolean_spheres(32, 0.6, 5)
    kw = dict(q=19, op=P.TRT, force=(2e-5, 0.0, 1e-6), storage=storage, scale_exp=16)
    with gpu_domain(g, **kw) as aa, gpu_domain(g, layout=P.SPARSE_PULL, **kw) as pl:
        for n in (0, 1, 1, 2, 3, 7):
            aa.step(n)
            pl.step(n)
            ra, ua = aa.macroscopic(P.ORDER_CELLS)
            rp, up = pl.macroscopic(P.ORDER_CELLS)
            assert np.array_equal(ra, rp) and np.array_equal(ua, up)
            assert np.array_equal(aa.reduce(), pl.reduce())
        assert np.array_equal(aa.export_lists()["P"], pl.export_lists()["P"])


def test_pull_graph_replay_and_checkpoint():
    g = G.random_solids((20, 17, 15), 0.3, 8, periodic=0b011, walls_z=True)
    kw = dict(q=19, op=P.TRT, force=(1e-5, 0, 0), layout=P.SPARSE_PULL)
    with gpu_domain(g, **kw) as ref:
        ref.step(9)
        want = ref.macroscopic(P.ORDER_CELLS)
    with gpu_domain(g, **kw) as d:
        d.step(4, graph=True)                  # from step 0 (in-place first collision)
        d.step(1, graph=True)
        state, step = d.get_state()
        assert step == 5
    with gpu_domain(g, **kw) as r:
        r.set_state(state, step)
        r.step(4, graph=True)                  # from an odd step: the other field
        got = r.macroscopic(P.ORDER_CELLS)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_pull_refusals():
    g = G.random_solids((10, 9, 8), 0.3, 3, periodic=0b010)
    f = g.flags
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    with pytest.raises(P.SlbmError):
        gpu_domain(g, q=19, layout=P.SPARSE_PULL)
    with gpu_domain(G.boolean_spheres(16, 0.5, 2), q=19, layout=P.SPARSE_PULL) as d:
        with pytest.raises(P.SlbmError):
            d.set_launch(1, 128, 1, 2)
        with pytest.raises(P.SlbmError):
            d.export_codes()
