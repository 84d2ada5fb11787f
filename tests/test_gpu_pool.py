"""Batched persistent stepping (slbm_pool_*): a member evolves bit for bit as
it would alone, at any parity, under graph replay and membership changes;
per-slot sums equal the single-domain sums; the host abort flag stops the
kernel without harming the context."""
import numpy as np
import pytest

import geometry as G
from helpers import gpu_domain

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2408_06880_gb300")


def _bc_geom(seed):
    g = G.random_solids((14, 11, 9), 0.25, seed, periodic=0b010)
    f = g.flags
    f[:, :, 0] = np.where(f[:, :, 0] == G.FLUID, G.INLET, f[:, :, 0])
    f[:, :, -1] = np.where(f[:, :, -1] == G.FLUID, G.OUTLET, f[:, :, -1])
    g.inlet_u = np.random.default_rng(seed).uniform(-0.02, 0.04, (int((f == G.INLET).sum()), 3))
    return g


def _cases(storage=0):
    kw = dict(q=19, op=P.TRT, storage=storage, scale_exp=18)
    return [
        (G.boolean_spheres(24, 0.5, 31), dict(kw, force=(1e-5, 0, 0))),
        (G.boolean_spheres(40, 0.7, 32), dict(kw, force=(2e-6, 1e-6, 0), omega=1.6)),
        (_bc_geom(33), dict(kw, force=(0, 0, 0), omega=1.1)),
        (G.relaxed_spheres(), dict(kw, op=P.SRT, force=(1e-6, 0, 0))),
    ]


def _alone(g, kw, steps):
    with gpu_domain(g, **kw) as d:
        d.step(steps)
        return d.get_state()[0], d.reduce()


# (split, group bytes, streams): split 10000 -- the larger members step with
# their own kernels, the smaller ones share the batched launch; group 0 -- one
# group of all batched members per launch; group 1 -- every member a group of
# its own, all k steps of it before the next; None -- the default grouping;
# streams 3 -- graph steps spread the large members over three streams
SPLIT_GROUP = [(0, 0, 1), (0, 1, 1), (10000, 1, 1), (10000, None, 1), (10000, None, 3), (0, None, 2)]


def _configure(pool, split, group, streams=1):
    pool.set_split(split)
    if group is not None:
        pool.set_group_bytes(group)
    if streams > 1:
        pool.set_streams(streams)


@pytest.mark.parametrize("split,group,streams", SPLIT_GROUP)
@pytest.mark.parametrize("storage", [P.FP32, P.FP16])
@pytest.mark.parametrize("graph", [False, True])
def test_pool_members_match_alone_bitwise(storage, graph, split, group, streams):
    cases = _cases(storage)
    steps = 9
    want = [_alone(g, kw, steps) for g, kw in cases]
    doms = [gpu_domain(g, **kw) for g, kw in cases]
    with P.Pool(19, storage, capacity=8) as pool:
        _configure(pool, split, group, streams)
        slots = [pool.add(d) for d in doms]
        pool.step(4, graph=graph)
        pool.step(5, graph=graph)
        sums = pool.reduce()
        for d, s, (ws, wr) in zip(doms, slots, want):
            got, step = d.get_state()
            assert step == steps
            assert np.array_equal(got, ws)
            assert np.array_equal(sums[s], wr)
            assert np.array_equal(d.reduce(), wr)
        assert not sums[len(doms):].any()
    for d in doms:
        d.close()


@pytest.mark.parametrize("split,group,streams", SPLIT_GROUP)
def test_mixed_parities_and_membership_changes_under_graph_replay(split, group, streams):
    cases = _cases()
    (ga, ka), (gb, kb), (gc, kc), _ = cases
    a, b, c = gpu_domain(ga, **ka), gpu_domain(gb, **kb), gpu_domain(gc, **kc)
    a.step(3)                                  # a joins at odd parity
    with P.Pool(19, 0, capacity=4) as pool:
        _configure(pool, split, group, streams)
        sa, sb = pool.add(a), pool.add(b)
        pool.step(4, graph=True)               # a: 7, b: 4
        pool.remove(sa)
        sc = pool.add(c)                       # same graph, new table
        pool.step(4, graph=True)               # b: 8, c: 4
        pool.step(1, graph=False)              # b: 9, c: 5
        pool.reduce()
        pool.remove(sb)                        # with split 10000 b steps alone: the
        pool.step(2, graph=True)               # batched table stays as it was; c: 7
        pool.reduce()
        for d, (g, kw), n in ((a, (ga, ka), 7), (b, (gb, kb), 9), (c, (gc, kc), 7)):
            got, step = d.get_state()
            want, _ = _alone(g, kw, n)
            assert step == n and np.array_equal(got, want)
    for d in (a, b, c):
        d.close()


def test_abort_flag_stops_kernels_and_context_stays_usable():
    cases = _cases()
    doms = [gpu_domain(g, **kw) for g, kw in cases]
    with P.Pool(19, 0, capacity=8) as pool:
        pool.set_split(0)                      # every member in the batched launch
        for d in doms:
            pool.add(d)
        pool.abort(True)
        pool.step(6, graph=True)
        with pytest.raises(P.SlbmError) as ei:
            pool.reduce()
        assert "EABORTED" in str(ei.value)
        pool.abort(False)                      # clear: the pool and context keep working
        fresh = gpu_domain(*cases[0][:1], **cases[0][1])
        s = pool.add(fresh)
        pool.step(2, graph=False)
        sums = pool.reduce()
        want = _alone(cases[0][0], cases[0][1], 2)[1]
        assert np.array_equal(sums[s], want)
        fresh.close()
    for d in doms:
        d.close()


def test_pool_launch_shapes_agree():
    cases = _cases()
    ref = [_alone(g, kw, 6)[0] for g, kw in cases]
    for threads, ctas in ((64, 0), (128, 2), (96, 1), (64, 8)):
        doms = [gpu_domain(g, **kw) for g, kw in cases]
        with P.Pool(19, 0, capacity=4) as pool:
            pool.set_launch(threads, ctas)
            for d in doms:
                pool.add(d)
            pool.step(6)
            pool.reduce()
            for d, w in zip(doms, ref):
                assert np.array_equal(d.get_state()[0], w)
        for d in doms:
            d.close()


def test_autotuner_keeps_results_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("SLBM_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2408_06880_gb300 import tuner
    g, kw = _cases()[1]
    want, _ = _alone(g, kw, 10)
    with gpu_domain(g, **kw) as d:
        d.step(4)
        chosen = tuner.tune_domain(d, reps=3)
        assert d.step_count == 4                       # state restored after timing
        d.step(6)
        got, _ = d.get_state()
    assert np.array_equal(got, want)
    assert set(chosen) == {"even", "odd"}
    assert (tmp_path / "tune.json").exists()
    with gpu_domain(g, **kw) as d2:                    # second domain: from the cache
        assert tuner.tune_domain(d2) == chosen
    doms = [gpu_domain(g2, **kw2) for g2, kw2 in _cases()]
    with P.Pool(19, 0, capacity=4) as pool:
        for d3 in doms:
            pool.add(d3)
        shape = tuner.tune_pool(pool, steps=2, reps=1)
        assert shape in tuner.POOL_SHAPES
        pool.step(6)
        pool.reduce()
        ref = [_alone(g3, kw3, 6)[0] for g3, kw3 in _cases()]
        for d3, w in zip(doms, ref):
            assert np.array_equal(d3.get_state()[0], w)
    for d3 in doms:
        d3.close()
