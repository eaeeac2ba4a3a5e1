"""Data-parallel dose calculation over ranks, one GPU each.

The method's only parallelism is over independent histories (Sec. 2.1.3: the
plan is sampled M histories at a time, and every history's particles depend
only on its own random stream). A run of B batches therefore splits into
disjoint batch ranges: rank r of N runs batches [b_r, b_r + n_r) of the same
plan with the same seed (lsm_run_opts.first_batch = b_r), so that the ranks
together draw exactly the histories one rank would have drawn, and the one
exchange step is a sum over ranks of the tally's batch sums S1 and S2 (FP64),
of its folded-batch count, its energy ledger and its statistics. The dose,
its batch sigma and the basis matrix of commissioning (Sec. 2.2.2) are then
computed from the reduced tally on any rank, and the Eq. 8 fit runs replicated
on every rank (it is milliseconds). Batched commissioning shards the same way:
every rank runs every PSR's histories of its own batches, so the (PSR,
history) work items are divided without changing any history's identity.

The reduction uses torch.distributed (NCCL between GPUs, gloo on CPU): sums of
FP64 and int64 tensors. Nothing here does any of the method's arithmetic.
"""
from __future__ import annotations

LEDGER_KEYS = ("source", "rejected", "escaped", "deposited")
STAT_KEYS = ("histories", "photons", "electrons", "rejected", "missed", "flights", "real", "esteps",
             "cap_hits", "overflows", "secondaries")


def batch_shard(n_batches: int, rank: int, world: int) -> tuple[int, int]:
    """(first batch, batch count) of `rank`: contiguous ranges covering
    [0, n_batches), sizes differing by at most one."""
    if not (0 <= rank < world) or n_batches < world:
        raise ValueError("need 0 <= rank < world <= n_batches")
    q, r = divmod(n_batches, world)
    first = rank * q + min(rank, r)
    return first, q + (1 if rank < r else 0)


def allreduce_sum(tensors, group=None):
    """In-place sum over ranks of every tensor (FP64 or int64)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return tensors
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def reduce_sums(s1, s2, n_batches: int, ledger: dict, stats: dict, group=None, device=None):
    """Sum one rank's tally state over all ranks. s1, s2: FP64 arrays or
    tensors; returns (s1, s2, n_batches, ledger, stats) of the whole run as
    torch tensors on `device` (default: the device s1 lives on, or the CPU)."""
    import torch
    if device is None:
        device = s1.device if isinstance(s1, torch.Tensor) else "cpu"
    t1 = torch.as_tensor(s1, dtype=torch.float64, device=device).contiguous()
    t2 = torch.as_tensor(s2, dtype=torch.float64, device=device).contiguous()
    led = torch.tensor([float(ledger[k]) for k in LEDGER_KEYS], dtype=torch.float64, device=device)
    cnt = torch.tensor([int(n_batches)] + [int(stats.get(k, 0)) for k in STAT_KEYS], dtype=torch.int64, device=device)
    allreduce_sum([t1, t2, led, cnt], group)
    c = cnt.cpu().tolist()
    return (t1, t2, c[0], dict(zip(LEDGER_KEYS, led.cpu().tolist())), dict(zip(STAT_KEYS, c[1:])))


def reduce_tally(lsm, tally, group=None, stream=None):
    """Replace every rank's tally by the sum of all ranks' tallies (the run's
    one exchange step); afterwards lsm_dose / lsm_basis_matrix on any rank give
    the whole run's result."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    s1 = torch.empty(tally.ncell, dtype=torch.float64, device=dev)
    s2 = torch.empty_like(s1)
    _, _, nb = lsm.lsm_tally_read(tally, stream=stream, out=(s1, s2))
    led, st = lsm.lsm_tally_ledger(tally, stream=stream)
    r1, r2, nbt, ledt, stt = reduce_sums(s1, s2, nb, led, st, group=group, device=dev)
    lsm.lsm_tally_load(tally, r1, r2, nbt, ledt, stt, stream=stream)
    return nbt


def run_shard(lsm, psl, ph, tally, seed: int, opts, rank: int, world: int, group=None, stream=None):
    """Rank `rank`'s share of a run of opts.n_batches batches, then the sum
    over ranks. Returns the run status of this rank (OK or OVERFLOW)."""
    import dataclasses
    first, count = batch_shard(opts.n_batches, rank, world)
    o = dataclasses.replace(opts, n_batches=count, first_batch=opts.first_batch + first)
    rc = lsm.lsm_run(psl, ph, tally, seed, o, stream=stream)
    reduce_tally(lsm, tally, group=group, stream=stream)
    return rc
