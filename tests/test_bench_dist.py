"""The multi-rank path of bench.py (replicas): step time is the maximum over
ranks and the converged count the sum, over a world_size-2 gloo group."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, conv = bench.aggregate(dist, torch, torch.device("cpu"), 10.0 + 5 * rank, 100 + rank)
    q.put((rank, ms, conv))
    dist.destroy_process_group()


def test_aggregate_max_time_sum_converged():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, conv in out:
        assert ms == 15.0 and conv == 201


def test_single_process_passthrough():
    import bench
    assert bench.aggregate(None, torch, torch.device("cpu"), 3.5, 7) == (3.5, 7)
