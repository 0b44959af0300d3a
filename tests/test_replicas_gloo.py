"""The N > 1 path of bench.py (replicas, no data-path collective) on CPU:
two gloo ranks agree on the barrier, take the slowest rank's time and draw
different read batches."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world)
    rate = bench.whole_job_rate(1000, world, 2, slowest)
    q.put((rank, slowest, rate, bench.replica_seed(rank)))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]                  # both see the slowest rank
    assert out[0][2] == out[1][2] == 2 * 1000 * 2 / 0.020       # all ranks' reads / slowest time
    assert out[0][3] != out[1][3]                                # different batches per replica
