"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks run
disjoint batch ranges of one seed and the reported time is the slowest rank's."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    slow = bench.slowest_ms(ms, world)
    firsts = [None] * world
    dist.all_gather_object(firsts, bench.rank_first_batch(rank, 16))
    q.put((rank, slow, firsts))
    dist.destroy_process_group()


def test_two_rank_timing_and_batch_ranges():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, firsts in out:
        assert slow == pytest.approx(15.0)
        # rank r runs batches [16 r, 16 r + 16): disjoint histories of one seed
        assert sorted(firsts) == [0, 16]
