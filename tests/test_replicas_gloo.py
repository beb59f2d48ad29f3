"""The N > 1 benchmark path on CPU: two gloo ranks run independent replicas
(no data-path collective); the whole-job rate is the units all ranks
processed over the slowest rank's time, and only the timing reductions
cross ranks."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        bench.barrier(ws)
        # rank r processed 100 (r + 1) units in 10 (r + 1) ms
        value, ms_max = bench.replica_rate(100 * (rank + 1), 10.0 * (rank + 1), ws)
        m = bench.max_over_ranks(float(rank) * 3.0, ws)
        bench.barrier(ws)
        q.put((rank, value, ms_max, m))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, value, ms_max, m in got:
        assert ms_max == 20.0                      # the slowest replica
        assert value == pytest.approx(300 / 0.020)  # all units over the max time
        assert m == 3.0


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(4.5, 1) == 4.5
    assert bench.replica_rate(50, 10.0, 1) == (50 / 0.010, 10.0)
