"""Continuous batching on the GPU: every served result equals the same request
solved alone (bit for bit: same kernels, deterministic sums), FP16 storage
stays within the permeability tolerance of FP32, and the FP32 permeability
matches the FP64 oracle run for the same number of steps."""
import numpy as np
import pytest

import geometry as G
import oracle as O

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2408_06880_gb300")
from paper_2408_06880_gb300.serving import GpuExecutor, Request, Server, solve_alone  # noqa: E402


def small_requests(n=6, tol=1e-5, max_steps=6000):
    reqs = []
    for i in range(n):
        edge = (24, 32, 40)[i % 3]
        g = G.boolean_spheres(edge, 0.45 + 0.05 * (i % 4), 500 + i)
        reqs.append(Request(i, g.flags, force=(1e-5, 0.0, 0.0), max_steps=max_steps, tol=tol,
                            arrival=0.0))
    return reqs


@pytest.mark.parametrize("lanes", [None, ((20000, 3), (None, 1))])
@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
def test_served_results_equal_alone(storage, lanes):
    # lanes: requests under 20000 cells (the 24^3 and 32^3 samples) advance
    # three chunks per tick in their own pool, the others one
    reqs = small_requests()
    alone = {r.rid: solve_alone(r, storage=storage, scale_exp=24) for r in reqs}
    ex = GpuExecutor(19, storage, capacity=3, scale_exp=24, lanes=lanes)     # fewer slots than requests
    try:
        res, st = Server(ex, budget_bytes=1 << 34, chunk=100).run(reqs, realtime=False)
    finally:
        ex.close()
    assert st["solved"] == len(reqs)
    for r in res:
        a = alone[r.rid]
        assert r.error is None
        assert r.steps == a.steps and r.converged == a.converged
        assert r.permeability == a.permeability          # bit for bit
    assert any(r.converged for r in res)


def test_fp16_permeability_close_to_fp32():
    # FP16 keeps 11 significant bits per stored population (relative rounding
    # 2^-12 per store).  On these small, strongly forced samples the measured
    # permeability error against FP32 was 1.3e-5 .. 1.5e-3; the bound below is
    # that of this test case, the stream workload's error is reported by
    # bench.py --mode serve.
    reqs = small_requests(4, tol=1e-6, max_steps=8000)
    errs = []
    for r in reqs:
        k32 = solve_alone(r, storage=P.FP32).permeability
        k16 = solve_alone(r, storage=P.FP16, scale_exp=24).permeability
        errs.append(abs(k16 / k32 - 1))
    assert max(errs) <= 3e-3, errs
    assert float(np.median(errs)) <= 5e-4, errs


def test_fp32_permeability_matches_oracle():
    g = G.boolean_spheres(24, 0.5, 777)
    req = Request(0, g.flags, force=(1e-5, 0.0, 0.0), max_steps=4000, tol=1e-6)
    r = solve_alone(req, storage=P.FP32)
    p = O.Problem.from_geometry(g, q=19, op=O.TRT, omega_plus=req.omega, magic=req.trt_magic, force=req.force)
    f = O.dense_run(p, O.dense_init(p), r.steps)
    k_oracle = O.permeability(p, O.reductions(p, f)[4])
    assert abs(r.permeability / k_oracle - 1) <= 1e-5
