"""The data-parallel path on CPU ranks (gloo, world size 2): disjoint batch
ranges of one seed, reduced by one sum, equal the one-rank run.

Each rank runs the oracle over its own batch range (the histories one rank
would have drawn for those batches) and hands its tally state to the product's
reduction (paper_1503_01725_b300.dist); the reduced state must equal the
oracle's single run over all batches: integer counters bit for bit, the FP64
sums up to the order of addition.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1503_01725_b300 import dist as D

N_BATCHES = 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    from paper_1503_01725_b300 import workloads as W
    wl = W.workload_full_10x10(1500)
    wl.phantom = W.water_phantom(20, 20, 24, 0.5)
    return wl


def _oracle_state(first, count):
    from oracle import oracle as O
    wl = _case()
    plan = O.Plan(wl.model, wl.beams, wl.n_hist)
    r = O.run(plan, wl.phantom, wl.seed, n_batches=count, electron_mode=1, first_batch=first)
    stats = dict(r["stats"], cap_hits=int(r["cap_hits"]), overflows=0)
    return r["s1"].ravel(), r["s2"].ravel(), count, r["ledger"], stats


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = D.batch_shard(N_BATCHES, rank, world)
    s1, s2, nb, led, st = _oracle_state(first, count)
    r1, r2, nbt, ledt, stt = D.reduce_sums(s1, s2, nb, led, st)
    q.put((rank, (first, count), r1.numpy(), r2.numpy(), nbt, ledt, stt))
    dist.destroy_process_group()


def test_batch_shards_cover_the_run_once():
    for n in (5, 16, 17, 255):
        for world in (1, 2, 3, 4, 8):
            if world > n:
                continue
            spans = [D.batch_shard(n, r, world) for r in range(world)]
            covered = [b for first, count in spans for b in range(first, first + count)]
            assert covered == list(range(n))
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        D.batch_shard(2, 0, 3)


def test_two_ranks_reduced_equal_one_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs], key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s1, s2, nb, led, st = _oracle_state(0, N_BATCHES)
    assert [o[1] for o in out] == [(0, 3), (3, 2)]
    for rank, _, r1, r2, nbt, ledt, stt in out:
        assert nbt == nb == N_BATCHES
        assert stt == st                                  # integer counters bit for bit
        np.testing.assert_allclose(r1, s1, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(r2, s2, rtol=1e-12, atol=1e-300)
        for k in D.LEDGER_KEYS:
            assert ledt[k] == pytest.approx(led[k], rel=1e-12)
    # the two ranks hold the same reduced state
    np.testing.assert_array_equal(out[0][2], out[1][2])
    # and a rank alone holds only its own batches
    a1 = _oracle_state(0, 3)[0]
    assert not np.allclose(a1, s1)
