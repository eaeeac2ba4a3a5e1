"""Oracle runs split over host processes -- TEST INFRASTRUCTURE ONLY.

A run of B batches of a plan equals runs of its disjoint batch ranges summed
(histories g = (first_batch + b) * plan + h), so the oracle's single-threaded
core can be spread over the host's cores: each spawn-started process builds
the seeded workload itself (paper_1503_01725_b300.workloads, no method
arithmetic), runs its batch range and returns its sums, restricted to a box of
voxels so that large phantoms do not move their whole tallies between
processes. Used by the GPU tests and by bench.py's CPU-baseline leg only.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

_W = {}


def _init(workload: str, n_hist_total: int, plan: int, box):
    from oracle import oracle as O
    from paper_1503_01725_b300 import workloads as W
    wl = getattr(W, workload)(n_hist_total)
    _W["wl"], _W["plan"], _W["box"] = wl, O.Plan(wl.model, wl.beams, plan), box


def _run(args):
    from oracle import oracle as O
    first, count, seed = args
    wl, plan, box = _W["wl"], _W["plan"], _W["box"]
    t0 = time.perf_counter()
    r = O.run(plan, wl.phantom, seed, n_batches=count, electron_mode=wl.electron_mode, first_batch=first)
    el = time.perf_counter() - t0
    (z0, z1), (y0, y1), (x0, x1) = box
    s1 = np.ascontiguousarray(r["s1"][z0:z1, y0:y1, x0:x1])
    s2 = np.ascontiguousarray(r["s2"][z0:z1, y0:y1, x0:x1])
    led = np.array([r["ledger"][k] for k in ("source", "rejected", "escaped", "deposited")])
    st = np.array([r["stats"][k] for k in ("histories", "photons", "electrons", "rejected", "missed",
                                           "flights", "real", "esteps")], dtype=np.int64)
    return s1, s2, led, st, r["max_balance"], el


def run_batches(workload: str, n_hist_total: int, plan: int, n_batches: int, seed: int, box,
                n_proc: int | None = None, first_batch: int = 0):
    """Batches [first_batch, first_batch + n_batches) of a `plan`-history plan
    of the named workload, in n_proc processes (default: the host's cores,
    at most n_batches). box = ((z0, z1), (y0, y1), (x0, x1)) voxel ranges.
    Returns s1, s2 over the box (sums over all batches), the ledger, the
    counters, the largest per-history energy imbalance, the process count and
    the wall time."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    n = max(1, min(n_proc or cores, n_batches))
    q, r = divmod(n_batches, n)
    spans, b = [], first_batch
    for i in range(n):
        c = q + (1 if i < r else 0)
        spans.append((b, c, seed))
        b += c
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(n, initializer=_init, initargs=(workload, n_hist_total, plan, box)) as pool:
        parts = pool.map(_run, spans, chunksize=1)
    wall = time.perf_counter() - t0
    s1 = sum(p[0] for p in parts)
    s2 = sum(p[1] for p in parts)
    led = sum(p[2] for p in parts)
    st = sum(p[3] for p in parts)
    bal = max(p[4] for p in parts)
    return {"s1": s1, "s2": s2, "ledger": led, "stats": st, "max_balance": bal, "processes": n,
            "wall_s": wall, "run_s": max(p[5] for p in parts)}
