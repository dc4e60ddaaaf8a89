"""The bench's multi-rank path on the CPU: two gloo ranks, each with its own
batch (weak scaling, no collective on the data path). The job time is the
slowest rank's and the bytes are summed over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, b = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), world)
    q.put((rank, t, b))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, b in res:
        assert t == 15.0 and b == 3000


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(3.0, 7, 1) == (3.0, 7)
