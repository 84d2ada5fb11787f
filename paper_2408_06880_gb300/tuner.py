"""Autotuner for launch shapes.

For a domain, every candidate shape of the even and of the odd kernel is
timed with CUDA events on the domain's own stream (median of several
launches, after warm-up), the fastest is applied, and the choice is cached in
a JSON file keyed by GPU name, stencil, storage, parity and a size class, so
later domains of the same kind reuse it without timing.  Shapes never change
results (every shape computes the same bits), only speed.

For a pool, the persistent kernel's threads per CTA (cells per tile) and
CTAs per SM are tuned the same way over the pool's current members."""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from . import _capi as A

EVEN_SHAPES = [(64, 1, 0), (64, 2, 0), (128, 2, 0), (64, 4, 0), (128, 2, 1), (128, 4, 1), (64, 2, 1),
               (64, 2, 2), (128, 2, 2), (64, 4, 2), (128, 2, 3), (128, 4, 3), (64, 2, 3), (128, 1, 0),
               (128, 1, 5)]
ODD_SHAPES = [(128, 1, 2), (64, 1, 2), (256, 1, 2), (128, 1, 3), (256, 1, 3), (128, 1, 4), (64, 1, 4), (128, 1, 0),
              (128, 2, 1), (256, 1, 5), (128, 1, 5), (64, 2, 2), (128, 2, 2), (256, 2, 2)]
POOL_SHAPES = [(64, 0), (64, 8), (128, 4), (96, 4)]

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("SLBM_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sparse_lbm", "tune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def size_class(n_fluid: int) -> int:
    """log2 bucket of the cell count (shapes matter by grid size)."""
    return int(math.log2(max(n_fluid, 1)))


def _valid(info: dict, parity: int, shape) -> bool:
    """Shapes the library accepts for this domain: no bulk-staged BF16 (even
    variants 1 and 3, odd variant 1); the moment-space operators (MRT,
    central moments, cumulants) run even variants 0 and 5 (MRT also 2) and odd
    variants 0, 2, 3 (without links) and 5, at most 2 cells per thread,
    variant 5 as 128 x 1; even variant 5 exists for them only."""
    staged = shape[2] == 1 or (parity == 0 and shape[2] == 3)
    if staged and info["storage"] == A.BF16:
        return False
    if info["op"] in (A.MRT, A.CM, A.CUMULANT):
        if shape[2] == 5:
            return tuple(shape[:2]) == (128, 1)
        if parity == 0:
            return shape[1] <= 2 and (shape[2] == 0 or (info["op"] == A.MRT and shape[2] == 2))
        return shape[1] <= 2 and (shape[2] in (0, 2) or (shape[2] == 3 and info.get("n_bc_links", 0) == 0))
    return shape[2] != 5 or parity == 1


def _time_parity(dom, parity: int, shape, reps: int, stream) -> float:
    import torch
    dom.set_launch(parity, *shape)
    for _ in range(2):
        dom.step(2)
    times = []
    for _ in range(reps):
        if dom.step_count % 2 != parity:
            dom.step(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dom.step(1)
        e1.record(stream)
        times.append((e0, e1))
        dom.step(1)
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in times]))


def tune_domain(dom, reps: int = 9, use_cache: bool = True, stream=None) -> dict:
    """Pick and apply the fastest even and odd shapes for `dom`.  The domain's
    state is saved before timing and restored afterwards."""
    import torch
    info = dom.info
    if info["layout"] != A.SPARSE:
        return {}                      # the pull and dense layouts have one launch shape
    key_base = (f"{_gpu_name()}|q{info['q']}|op{info['op']}|st{info['storage']}"
                f"|n{size_class(info['n_fluid'])}")
    with _lock:
        cache = _load() if use_cache else {}
    chosen = {}
    todo = []
    for parity in (0, 1):
        key = f"{key_base}|p{parity}"
        if key in cache:
            chosen[parity] = tuple(cache[key]["shape"])
        else:
            todo.append((parity, key))
    if todo:
        st = stream if stream is not None else getattr(dom, "_stream", None)
        if st is None:
            st = torch.cuda.current_stream()
        state, step = dom.get_state()
        for parity, key in todo:
            shapes = EVEN_SHAPES if parity == 0 else ODD_SHAPES
            res = {}
            for s in shapes:
                if not _valid(info, parity, s):
                    continue
                try:
                    res[s] = _time_parity(dom, parity, s, reps, st)
                except A.SlbmError as e:          # a shape this domain refuses (cell order, layout)
                    if e.status not in (A.EINVAL, A.EUNSUPPORTED):
                        raise
            best = min(res, key=res.get)
            chosen[parity] = best
            cache[key] = {"shape": list(best), "ms": res[best],
                          "all_ms": {",".join(map(str, s)): round(v, 5) for s, v in res.items()}}
        dom.set_state(state, step)
        if use_cache:
            with _lock:
                merged = _load()
                merged.update(cache)
                _store(merged)
    for parity, shape in chosen.items():
        dom.set_launch(parity, *shape)
    return {"even": chosen[0], "odd": chosen[1]}


def tune_pool(pool, steps: int = 4, reps: int = 3, use_cache: bool = True) -> tuple:
    """Pick and apply the pool kernel shape (threads, ctas_per_sm) by timing
    `steps` pool steps over the current members (their states are restored)."""
    import time
    import torch
    key = f"{_gpu_name()}|pool|q{pool.q}|st{pool.storage}|m{len(pool.members)}"
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        best = tuple(cache[key]["shape"])
        pool.set_launch(*best)
        return best
    saved = {s: d.get_state() for s, d in pool.members.items()}
    res = {}
    for shape in POOL_SHAPES:
        pool.set_launch(*shape)
        pool.step(steps, graph=False)
        pool.reduce()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pool.step(steps, graph=False)
            pool.reduce()
            ts.append(time.perf_counter() - t0)
        res[shape] = float(np.median(ts))
    for s, (state, step) in saved.items():
        pool.members[s].set_state(state, step)
    best = min(res, key=res.get)
    pool.set_launch(*best)
    if use_cache:
        with _lock:
            merged = _load()
            merged[key] = {"shape": list(best), "s": res[best]}
            _store(merged)
    return best
