"""Request-level replicas across ranks (one process per GPU).

Domains are independent, so the multi-GPU form of this library is a set of
replicas with no exchange on the data path: every rank steps its own domains
(or serves its own share of a request stream) on its own GPU, and the host
only combines timings and results at the end.  These helpers work with any
initialised `torch.distributed` process group (NCCL on GPUs, gloo on CPU);
with no process group they reduce to the single-process case.
"""
from __future__ import annotations


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def rank_world() -> tuple[int, int]:
    d = _dist()
    return (d.get_rank(), d.get_world_size()) if d else (0, 1)


def shard(items: list, rank: int | None = None, world: int | None = None) -> list:
    """This rank's share of `items`: every world-th item starting at rank
    (so each item lands on exactly one rank)."""
    if rank is None or world is None:
        rank, world = rank_world()
    return items[rank::world]


def _tensor(values):
    import torch
    d = _dist()
    dev = "cuda" if d and d.get_backend() == "nccl" else "cpu"
    return torch.tensor(values, dtype=torch.float64, device=dev)


def job_rate(units_local: float, seconds_local: float) -> tuple[float, float, float]:
    """Whole-job throughput over all ranks: (sum of units) / (max of times).
    Returns (rate, total units, max seconds).  Call after every rank has
    finished its timed work; it synchronises the ranks."""
    d = _dist()
    if d is None:
        return (units_local / seconds_local if seconds_local > 0 else float("nan"), float(units_local),
                float(seconds_local))
    units = _tensor([float(units_local)])
    secs = _tensor([float(seconds_local)])
    d.all_reduce(units, op=d.ReduceOp.SUM)
    d.all_reduce(secs, op=d.ReduceOp.MAX)
    u, s = float(units.item()), float(secs.item())
    return (u / s if s > 0 else float("nan"), u, s)


def gather(obj) -> list | None:
    """Every rank's `obj`, in rank order, on rank 0 (None elsewhere)."""
    d = _dist()
    if d is None:
        return [obj]
    out = [None] * d.get_world_size() if d.get_rank() == 0 else None
    d.gather_object(obj, out, dst=0)
    return out


def barrier() -> None:
    d = _dist()
    if d is not None:
        d.barrier()
