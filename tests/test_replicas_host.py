"""The multi-rank form (request-level replicas, no data-path exchange) on CPU:
two gloo ranks shard a request stream, combine the whole-job rate (sum of
work over the slowest rank's time) and gather results on rank 0; the served
results equal a single-process run."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2408_06880_gb300 import replicas  # noqa: E402
from paper_2408_06880_gb300.serving import Server, serve_replicas  # noqa: E402
from test_serving_host import FakeExecutor, req  # noqa: E402

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reqs():
    return [req(i, T=150.0 + 60 * i) for i in range(9)]


def _worker(rank, port, outdir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=WORLD)
    try:
        assert replicas.rank_world() == (rank, WORLD)
        assert replicas.shard(list(range(9))) == list(range(rank, 9, WORLD))
        rate, total, secs = replicas.job_rate(rank + 1, rank + 2.0)
        assert (rate, total, secs) == (1.0, 3.0, 3.0)          # (1 + 2) units / max(2, 3) s
        got = replicas.gather({"rank": rank})
        if rank == 0:
            assert got == [{"rank": 0}, {"rank": 1}]
        else:
            assert got is None
        res, st = serve_replicas(FakeExecutor(capacity=3), _reqs(), 10 ** 9, realtime=False)
        if rank == 0:
            assert st["ranks"] == WORLD and st["solved"] == 9
            with open(os.path.join(outdir, "served.txt"), "w") as f:
                for r in sorted(res, key=lambda r: r.rid):
                    f.write(f"{r.rid} {r.steps} {r.permeability!r}\n")
        else:
            assert sorted(r.rid for r in res) == list(range(1, 9, 2))   # its own share only
        replicas.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_combine_and_match_one_process(tmp_path):
    mp.spawn(_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    res, _ = Server(FakeExecutor(capacity=3), 10 ** 9).run(_reqs(), realtime=False)
    want = [f"{r.rid} {r.steps} {r.permeability!r}" for r in sorted(res, key=lambda r: r.rid)]
    assert (tmp_path / "served.txt").read_text().split("\n")[:-1] == want


def test_single_process_helpers_reduce_to_local_values():
    assert replicas.rank_world() == (0, 1)
    assert replicas.shard([1, 2, 3]) == [1, 2, 3]
    assert replicas.job_rate(6.0, 2.0) == (3.0, 6.0, 2.0)
    assert replicas.gather("x") == ["x"]
