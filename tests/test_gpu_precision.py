"""GPU tests of the reduced-precision support: the extended domain reduction
(sums plus max |f_i - w_i| and max |u|), the in-place storage change
(FP16/BF16 -> FP32 hand-off, exact power-of-two rescale, FP32 -> FP16/BF16
rounding), and the BF16 storage form against the FP64 oracle with its error
stated, like the FP16 rows of test_gpu_configs.py."""
import numpy as np
import pytest

import geometry as G
import oracle as O
from helpers import gpu_domain, rel_l2

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2408_06880_gb300")
from paper_2408_06880_gb300 import _capi as A  # noqa: E402

TRT = dict(op=P.TRT, omega=1.25, trt_magic=3 / 16)


def _stored(d):
    """Stored populations (Q, S) as float64 in unscaled units, and N_F."""
    buf, _ = d.get_state()
    inf = d.info
    q, S, st, s = inf["q"], inf["stride"], inf["storage"], inf["scale_exp"]
    if st == P.FP32:
        x = buf.view(np.float32).astype(np.float64)
    elif st == P.FP16:
        x = buf.view(np.float16).astype(np.float64) * 2.0 ** -s
    else:
        x = (buf.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64) * 2.0 ** -s
    return x.reshape(q, S), inf["n_fluid"]


def _forced(storage=P.FP32, scale_exp=0, steps=40):
    g = G.boolean_spheres(32, 0.5, 3)
    d = gpu_domain(g, q=19, force=(1e-5, 2e-6, 0.0), storage=storage, scale_exp=scale_exp, **TRT)
    d.step(steps)
    return g, d


@pytest.mark.parametrize("steps", [40, 41])          # natural and odd-step (gathered) parity
@pytest.mark.parametrize("storage", [P.FP32, P.FP16, P.BF16])
def test_reduce_ext_sums_and_maxima(storage, steps):
    _, d = _forced(storage, 0 if storage == P.FP32 else 24, steps)
    with d:
        ext = d.reduce_ext()
        assert np.array_equal(ext[:5], d.reduce())                   # the same bits as the plain sums
        x, nf = _stored(d)
        assert ext[5] == np.max(np.abs(x[:, :nf]))                   # every stored slot, exact
        _, u = d.macroscopic(P.ORDER_CELLS)
        sp = np.sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2])        # float32, the kernel's order
        assert ext[6] == pytest.approx(float(np.max(sp)), rel=1e-6)
        assert ext[6] > 0


def test_reduce_ext_reports_a_nan_and_the_stability_bound():
    _, d = _forced()
    with d:
        buf, step = d.get_state()
        x = buf.view(np.float32).copy()
        x[3 * d.info["stride"] + 5] = np.nan
        d.set_state(x.view(np.uint8), step)
        out = d.reduce_ext(check=False)
        assert np.isnan(out[5])
        with pytest.raises(P.SlbmError, match="EDIVERGED"):
            d.reduce_ext()


def test_pool_reduce_ext_matches_members():
    doms = [_forced(P.FP16, 24, 40 + 2 * j)[1] for j in range(3)]
    with P.Pool(19, P.FP16, capacity=4) as pool:
        slots = [pool.add(d) for d in doms]
        pool.step(2)
        ext = pool.reduce_ext()
        for d, s in zip(doms, slots):
            pool.remove(s)
            assert np.array_equal(ext[s], d.reduce_ext())
    for d in doms:
        d.close()


@pytest.mark.parametrize("src", [P.FP16, P.BF16])
def test_handoff_to_fp32_is_exact_and_keeps_the_step(src):
    _, d = _forced(src, 24, 41)                                     # odd parity: slots mid-pair
    with d:
        before, nf = _stored(d)
        step = d.step_count
        d.set_storage(P.FP32)
        after, _ = _stored(d)
        assert d.info["storage"] == P.FP32 and d.step_count == step
        assert np.array_equal(after, before)                        # raw * 2^-s, exactly
        # stepping on continues exactly like an FP32 domain given that state
        g = G.boolean_spheres(32, 0.5, 3)
        with gpu_domain(g, q=19, force=(1e-5, 2e-6, 0.0), **TRT) as ref:
            ref.set_state(after.astype(np.float32).view(np.uint8).reshape(-1), step)
            d.step(9)
            ref.step(9)
            assert np.array_equal(_stored(d)[0], _stored(ref)[0])


def test_rescale_is_exact_and_overflow_is_refused():
    _, d = _forced(P.FP16, 24, 40)
    with d:
        x0, nf = _stored(d)
        d.set_storage(P.FP16, 26)
        x1, _ = _stored(d)
        big = np.abs(x0) * 2.0 ** 24 >= 2.0 ** -14                   # FP16 normal range before and after
        assert np.array_equal(x1[big], x0[big])
        assert d.info["scale_exp"] == 26
        gmax = d.reduce_ext()[5]
        s_over = int(np.ceil(np.log2(65504.0 / gmax))) + 1           # would overflow FP16
        with pytest.raises(P.SlbmError, match="EINVAL"):
            d.set_storage(P.FP16, s_over)
        assert d.info["scale_exp"] == 26 and np.array_equal(_stored(d)[0], x1)


def test_fp32_to_fp16_rounds_to_nearest_even():
    _, d = _forced(P.FP32, 0, 40)
    with d:
        x32, nf = _stored(d)
        d.set_storage(P.FP16, 20)
        buf, _ = d.get_state()
        want = (x32.astype(np.float32) * np.float32(2.0 ** 20)).astype(np.float16)
        assert np.array_equal(buf.view(np.float16).reshape(want.shape), want)


def test_storage_change_of_a_pool_member_is_refused():
    _, d = _forced(P.FP16, 24, 40)
    with d, P.Pool(19, P.FP16, capacity=2) as pool:
        s = pool.add(d)
        with pytest.raises(P.SlbmError, match="EINVAL"):
            d.set_storage(P.FP32)
        pool.remove(s)
        d.set_storage(P.FP32)
        assert d.info["storage"] == P.FP32


def test_freed_member_leaves_its_pool():
    _, d = _forced(P.FP32, 0, 40)
    _, e = _forced(P.FP32, 0, 40)
    with P.Pool(19, P.FP32, capacity=2) as pool:
        pool.add(d)
        se = pool.add(e)
        d.close()                                    # the pool loses the member, keeps stepping the other
        pool.step(2)
        assert pool.reduce()[se][4] == pytest.approx(e.reduce()[4])
        pool.remove(se)
    e.close()


# --------------------------------------------- BF16 storage vs the FP64 oracle
def _oracle_cells(g, steps, q, op, force):
    p = O.Problem.from_geometry(g, q=q, op=op, omega_plus=1.25, magic=3 / 16, force=force)
    L = O.pull_list(p)
    f = O.sparse_run(p, L, O.sparse_rest(p, L), steps)
    return O.sparse_macroscopic(p, L, f)


def test_bf16_packing_32_srt_200_steps_vs_oracle():
    # the 32^3 relaxed packing, SRT, F = 1e-6 x, 200 steps.  BF16 keeps 8
    # significant bits (relative rounding 2^-9 per store): measured velocity
    # relative L2 1.74e-3 and sum of u_x 1.97e-4 against the FP64 oracle
    # (FP16: 2.2e-4 and 2.7e-5; FP32: 7.9e-7)
    g = G.relaxed_spheres()
    force = (1e-6, 0.0, 0.0)
    rho_o, u_o = _oracle_cells(g, 200, 19, O.SRT, force)
    with gpu_domain(g, q=19, op=P.SRT, omega=1.25, force=force, storage=P.BF16,
                    scale_exp=P.auto_scale_exp(1e-3)) as d:
        d.step(200)
        rho, u = d.macroscopic(P.ORDER_CELLS)
    u = u.T.astype(np.float64)
    assert rel_l2(u, u_o) <= 3e-3
    assert abs(np.sum(u[:, 0]) / np.sum(u_o[:, 0]) - 1) <= 5e-4
    assert np.max(np.abs(rho - rho_o)) <= 2e-6


def test_bf16_scaled_bed_5000_steps_vs_oracle():
    # the particle bed at 64 x 32 x 32 (inlet 0.05, outlet rho 1), D3Q27 TRT,
    # 5000 steps: measured velocity relative L2 6.1e-3 (FP16 1.4e-3, FP32
    # 7.7e-7)
    g = G.particle_bed(64, 32, 32, bed_top=16, radius=4.0, seed=22)
    rho_o, u_o = _oracle_cells(g, 5000, 27, O.TRT, (0.0, 0.0, 0.0))
    with gpu_domain(g, q=27, force=(0.0, 0.0, 0.0), storage=P.BF16, scale_exp=P.auto_scale_exp(0.06, 0.01),
                    **TRT) as d:
        d.step(5000)
        rho, u = d.macroscopic(P.ORDER_CELLS)
    assert rel_l2(u.T.astype(np.float64), u_o) <= 1e-2
    assert np.max(np.abs(rho - rho_o)) <= 5e-3
