"""bench.py's multi-rank path on CPU: two gloo ranks agree on the max timed
milliseconds (the barrier + max-over-ranks rule), and the JSON aggregation uses it."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 100.0 + 50.0 * rank
    out = bench.aggregate(local, world)
    bench.barrier(world)
    q.put((rank, out, bench.dist_env()))
    dist.destroy_process_group()


def test_two_rank_max_aggregation():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    assert [r[2][:2] for r in res] == [(0, 2), (1, 2)]


def test_single_rank_aggregation_is_identity():
    import bench
    assert bench.aggregate(12.5, 1) == 12.5
