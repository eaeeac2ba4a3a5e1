"""Launch-parameter autotuner for batched runs (lsm_run).

The transport of Sec. 2 is run as iterations of M histories (the paper's
particle batch, Sec. 2.1.3) by persistent kernels. Three launch parameters
change the speed and nothing else (the Philox streams are keyed by history,
so every choice gives the same histories):

- ``chunk``: histories per sample/transport iteration. Plans smaller than it
  run k whole batches per iteration (k = chunk // plan).
- ``ctas_per_sm``: CTAs per SM of the persistent transport kernels.
- ``use_graph``: capture the run's launch sequence once as a CUDA graph and
  replay it.

``tune`` times lsm_run on the caller's plan, phantom and tally for a small
grid of these, keeps the fastest, and caches the choice in a JSON file keyed
by device and workload signature. The tally is reset afterwards.
"""
from __future__ import annotations

import dataclasses
import json
import os
import statistics

from . import lsm

MAX_CHUNK = 1 << 24


def default_cache_path() -> str:
    return os.environ.get("LSM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lsm", "autotune.json"))


def signature(psl: lsm.PSL, ph: lsm.PhantomHandle, tally: lsm.Tally, base: lsm.RunOpts) -> str:
    """Device and workload key of a tuned choice."""
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    plan = int(psl.info["plan_size"])
    return (f"{p.name}|sm{p.multi_processor_count}|plan{plan}|ent{int(psl.info['n_ent'])}"
            f"|B{base.n_batches}|mode{tally.mode}|cells{tally.ncell}|vox{ph.desc.nvox}"
            f"|e{base.electron_mode}")


def candidates(plan: int, n_batches: int, ctas=(0, 2, 3), graphs=(False, True)):
    """Iteration sizes: whole-batch multiples of the plan (1, 2, 4, ... batches
    per iteration up to the run's batches) when the plan is small, fixed sizes
    2^21 .. 2^24 otherwise; crossed with CTAs per SM and graph replay."""
    chunks = set()
    if plan < MAX_CHUNK:
        k = 1
        while k <= n_batches and k * plan <= MAX_CHUNK:
            chunks.add(k * plan)
            k *= 2
        top = min(n_batches, MAX_CHUNK // plan)
        if top >= 1:
            chunks.add(top * plan)
    for s in (21, 22, 23, 24):
        if (1 << s) <= plan:
            chunks.add(1 << s)
    return [(c, a, g) for c in sorted(chunks) for a in ctas for g in graphs]


def _time_run(psl, ph, tally, opts, seed, reps):
    import torch
    stream = torch.cuda.current_stream()
    lsm.lsm_tally_reset(tally)
    lsm.lsm_run(psl, ph, tally, seed, opts)          # workspace, slots, graph capture
    ms = []
    for r in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lsm.lsm_tally_reset(tally)
        torch.cuda.synchronize()
        a.record(stream)
        lsm.lsm_run(psl, ph, tally, seed + 1 + r, opts)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def tune(psl: lsm.PSL, ph: lsm.PhantomHandle, tally: lsm.Tally, base: lsm.RunOpts | None = None,
         seed: int = 424242, reps: int = 3, cands=None, cache_path: str | None = "default",
         refresh: bool = False):
    """Fastest (chunk, ctas_per_sm, use_graph) for this plan/phantom/tally.

    Returns (RunOpts, report). The report lists every timed candidate in ms
    per run. With a cache path, a stored choice for the same signature is
    returned without timing unless ``refresh``.
    """
    base = base or lsm.RunOpts()
    if lsm.timing_enabled():
        raise RuntimeError("autotune: disable the library's kernel timers first (graphs bypass them)")
    key = signature(psl, ph, tally, base)
    path = default_cache_path() if cache_path == "default" else cache_path
    store = {}
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                store = json.load(f)
        except (OSError, ValueError):
            store = {}
    if path and not refresh and key in store:
        c = store[key]
        opts = dataclasses.replace(base, chunk=c["chunk"], ctas_per_sm=c["ctas_per_sm"],
                                   use_graph=bool(c["use_graph"]))
        return opts, {"signature": key, "cached": True, "choice": c}
    plan = int(psl.info["plan_size"])
    trials = []
    for chunk, ctas, graph in (cands or candidates(plan, base.n_batches)):
        o = dataclasses.replace(base, chunk=int(chunk), ctas_per_sm=int(ctas), use_graph=bool(graph))
        trials.append({"chunk": int(chunk), "ctas_per_sm": int(ctas), "use_graph": bool(graph),
                       "ms": _time_run(psl, ph, tally, o, seed, reps)})
    lsm.lsm_tally_reset(tally)
    best = min(trials, key=lambda t: t["ms"])
    if path:
        store[key] = best
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    opts = dataclasses.replace(base, chunk=best["chunk"], ctas_per_sm=best["ctas_per_sm"],
                               use_graph=best["use_graph"])
    return opts, {"signature": key, "cached": False, "choice": best, "trials": trials}
