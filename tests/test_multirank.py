"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1). Multi-GPU runs are
independent replicas of the solve; the only exchange is the timing, reduced to the slowest
rank's, which every rank receives."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        env = bench.dist_env()
        v = bench.max_over_ranks(1.0 + 0.5 * rank, "cpu")
        w = bench.max_over_ranks(7.0 - rank, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    q.put((rank, env, v, w))


def test_max_over_ranks_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, v, w in out:
        assert env == (rank, rank, 2)
        assert v == 1.5 and w == 7.0


def test_max_over_ranks_without_a_process_group_is_the_value():
    import bench
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
