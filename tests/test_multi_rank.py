"""The bench's multi-rank path on CPU: two gloo ranks, each a replica with its
own work, aggregated as total units over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    # rank r processed (r + 1) * 100 units in (r + 1) seconds
    value, t_max = bench.aggregate(float(r + 1), float((r + 1) * 100), w)
    q.put((r, w, lr, value, t_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, lr, value, t_max in out:
        assert w == 2 and lr == r
        assert t_max == pytest.approx(2.0)
        assert value == pytest.approx(300.0 / 2.0)


def test_single_rank_aggregate_is_local():
    import bench
    v, t = bench.aggregate(2.0, 50.0, 1)
    assert v == 25.0 and t == 2.0
