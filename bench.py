#!/usr/bin/env python
"""Benchmark of the analytic-source-model dose calculation on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step is one pass of the whole hot path over one workload: PSR -> PSL
conversion with sampling areas and Eq. 3 counts (lsm_build_psl), then n_batches
passes of [sample M histories -> transport photons (and the annihilation
photons of their pair events) -> electrons -> tally flush] (lsm_run), then
dose and batch uncertainty
(lsm_dose). The workload is all three sub-sources, a 10x10 cm2 field, water
64^3 at 0.25 cm, 1e7 histories, CSDA electrons (synthetic inputs from
paper_1503_01725_b300.workloads). Prints one JSON line.

Metric: histories/s (source histories including jaw-rejected ones, per second
of device time) and seconds to 1% dose uncertainty, t_1% = T (u / 0.01)^2 with
u the mean batch relative standard deviation over voxels above 50% of Dmax.

--impl reference times the CPU oracle (plain single-threaded FP64 C, one
process per host core on disjoint seeds) on a bounded sample of the same
workload.
Under torchrun (N > 1) every rank runs the same workload on its own range of
batches of one seed (disjoint histories: weak scaling), and every step ends
with the one exchange step of the method, the sum of the ranks' tallies over
NCCL (paper_1503_01725_b300.dist); rank 0 prints the line with the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0

# Algorithmic bytes per unit of work:
#   sampling: per particle entering the phantom, its queue record (48 B); the plan
#     tables (entries and prefix, a few hundred KB) are read once per launch and
#     stay in cache for the lookups of every history;
#   photon transport: per Woodcock flight one density load (4 B), per photon the
#     queue read (48 B), per electron it queues (the run's `secondaries`) the
#     queue write (48 B), per other real interaction one tally update (8 B);
#   electron transport: per CSDA step one density load (4 B) + one tally update
#     (4 B read + 4 B write), per electron the queue read (48 B): source
#     electrons and the secondaries.
# DRAM bytes per unit measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# on a reduced case of this workload with the benchmark's 16 tally slices (4e6
# histories in one iteration: 227.0 MB over 3,101,770 photons and the
# annihilation photons they create; 112.2 MB over 9,896,378 electron steps;
# ncu replays start from flushed caches).
# Valid for the kernels as profiled; set to None when they change.
TRAFFIC_PER_UNIT = {"photon": ("photons", 73.2), "electron": ("esteps", 11.34)}
B_SAMPLE_PER_ENTERING = 48.0
B_FLIGHT = 4.0
B_QUEUE = 48.0
B_DEPOSIT = 8.0
B_ESTEP = 12.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-hist", type=int, default=10_000_000)
    p.add_argument("--n-batches", type=int, default=16)
    p.add_argument("--chunk", type=int, default=0, help="histories per iteration (0: autotuned)")
    p.add_argument("--no-autotune", action="store_true",
                   help="library defaults instead of the tuned iteration size, CTAs per SM and graph replay")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the commissioning (batched) block")
    p.add_argument("--no-denoised", action="store_true", help="skip the denoised-dose block")
    p.add_argument("--no-pslfile", action="store_true", help="skip the PSL-file comparator block")
    p.add_argument("--no-multibeam", action="store_true", help="skip the multi-beam plan block")
    p.add_argument("--no-validation", action="store_true", help="skip the commissioning validation loop")
    p.add_argument("--no-fields", action="store_true", help="skip the field-size sweep")
    p.add_argument("--no-precision", action="store_true", help="skip the 256x256x160 precision case")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


SEED = 1


def rank_first_batch(rank: int, n_batches: int) -> int:
    """Weak scaling: every rank runs n_batches batches of the same plan and
    seed, rank r the batches [r n_batches, (r + 1) n_batches) of one run of
    world x n_batches batches, so that the ranks draw disjoint histories; the
    step ends with the sum of the ranks' tallies (dist.reduce_tally)."""
    return rank * n_batches


def slowest_ms(total_ms: float, world: int) -> float:
    """Timing reduction over ranks: the job takes as long as its slowest rank."""
    if world <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def iteration_size(opts, plan: int) -> int:
    """Histories per sample/transport iteration of lsm_run (whole batches when
    the plan is smaller than the iteration size)."""
    chunk = opts.chunk if opts.chunk > 0 else 1 << 23
    if plan < chunk:
        return min(opts.n_batches, chunk // plan) * plan
    return chunk


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            P = json.load(f)
        return float(P["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples. Started before the
    warm-up (its start-up must not overlap the timed steps); only samples
    time-stamped inside the timed window are summarised."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.t0 = self.t1 = None

    def start(self):
        if os.environ.get("LSM_BENCH_NO_CLOCKS") == "1":
            return self
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            deadline = time.time() + 20
            while time.time() < deadline and os.path.getsize(self.f.name) == 0:
                time.sleep(0.05)
        except Exception:
            self.p = None
        return self

    def window(self, t0: float, t1: float):
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.p:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self) -> dict:
        import datetime
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if self.t0 is not None and not (self.t0 - 0.15 <= ts <= self.t1 + 0.15):
                    continue
                sm.append(float(r[2]))
                smax = float(r[3])
                for k, v in zip(names, r[6:10]):
                    if v.strip().lower() == "active":
                        reasons.add(k)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def u_mean_rel(dose: np.ndarray, sigma: np.ndarray, rho: np.ndarray | None = None) -> float:
    """Mean relative batch sigma over voxels above half the maximum dose; with
    rho, voxels below 0.1 g/cm^3 (air: dose per gram from a handful of
    deposits) are left out of the dose region."""
    d = dose if rho is None else np.where(np.reshape(rho, dose.shape) >= 0.1, dose, 0.0)
    sel = d > 0.5 * d.max()
    return float(np.mean(sigma[sel] / dose[sel]))


def cpu_oracle_rate(wl, seconds: float, per_step_hist: int = 100_000):
    """Oracle histories/s on a bounded sample: repeated 1e5-history plans of the
    same workload (same model, field, phantom) with fresh seeds."""
    from oracle import oracle as O
    plan = O.Plan(wl.model, wl.beams, per_step_hist)
    done, t0, seed = 0, time.perf_counter(), 1000
    while True:
        O.run(plan, wl.phantom, seed, n_batches=1, electron_mode=wl.electron_mode)
        done += per_step_hist
        seed += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done / el, done, el


_ORACLE = None


def _oracle_init(wl, per: int, electron_mode: int):
    """Pool initializer: each process loads the oracle and builds the plan once."""
    global _ORACLE
    from oracle import oracle as O
    _ORACLE = (O, O.Plan(wl.model, wl.beams, per), wl.phantom, electron_mode)


def _oracle_pass(seed: int) -> int:
    """One pass of the plan with the given seed (independent histories)."""
    O, plan, ph, em = _ORACLE
    O.run(plan, ph, seed, n_batches=1, electron_mode=em)
    return seed


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(wl, per: int, electron_mode: int):
    """Processes (started with spawn, so that none is forked from a process
    holding a CUDA context) that run the oracle on disjoint seeds, one per
    host core (at most 64)."""
    import multiprocessing as mp
    n = max(1, min(64, host_cores()))
    pool = mp.get_context("spawn").Pool(n, initializer=_oracle_init, initargs=(wl, per, electron_mode))
    pool.map(_oracle_pass, range(900, 900 + n), chunksize=1)     # every process has loaded the oracle
    return pool, n


def cpu_oracle_rate_all_cores(wl, seconds: float, per: int = 100_000):
    """Oracle histories/s on all host cores: rounds of one 1e5-history pass
    per process with fresh seeds until `seconds` have passed."""
    pool, n = oracle_pool(wl, per, wl.electron_mode)
    try:
        done, seed, t0 = 0, 2000, time.perf_counter()
        while True:
            pool.map(_oracle_pass, range(seed, seed + n), chunksize=1)
            done += n * per
            seed += n
            el = time.perf_counter() - t0
            if el >= seconds:
                break
    finally:
        pool.terminate()
        pool.join()
    return done / el, done, el, n


def _u_A(s1, s2, nb, ref):
    """Mean relative batch sigma of the basis-matrix entries above half their
    column's maximum (the commissioning analogue of u for D > 50 % Dmax). The
    entries are chosen on `ref`, the basis matrix of an independent run, so
    that a run does not choose the entries where it fluctuated high."""
    var_b = np.clip(s2 - s1 * s1 / nb, 0, None) / max(nb - 1, 1)
    sig = np.sqrt(nb * var_b).reshape(ref.shape)
    S1 = s1.reshape(ref.shape)
    sel = (ref > 0.5 * ref.max(axis=0, keepdims=True)) & (ref > 0) & (S1 > 0)
    return float(np.mean(sig[sel] / S1[sel]))


def commissioning_block(lsm, W, reps: int = 3, n_batches: int = 16):
    """Basis-dose runs of commissioning (Sec. 2.2.2: 300 PSRs x 3 fields,
    per-PSR history counts proportional to weight, clamped to 1e4-1e6) two
    ways, with the same histories per PSR and batch:

    - batched: every PSR's runs in one plan and one run, launch parameters
      picked by the autotuner and the run replayed as one CUDA graph;
    - plain: one plan and one run per PSR (300 dose calculations).

    Each arm's device time, the measured uncertainty u_A of the basis entries
    and the time to u_A = 1 % by the 1/N law (confirmed by a batched run of 4x
    the histories); then the FP64 NNLS fit of Eq. 8 over the photon PSRs and
    the electron units (Sec. 2.2.3), by active set and by gradient projection."""
    import torch
    from paper_1503_01725_b300 import autotune
    wl = W.workload_commissioning()
    n_k = np.asarray(wl.extra["n_k"], dtype=np.int64)
    ph = lsm.lsm_phantom_create(wl.phantom)
    ph.desc = wl.phantom
    idx, n_rows = W.commissioning_index(wl.phantom)
    m = wl.model
    mh = lsm.lsm_model_create(m)
    nb_beams = wl.beams.n_beams
    tally = lsm.lsm_tally_create(ph, mode=1, idx3d=idx, n_rows=n_rows, n_psr=m.n_psr, n_beams=nb_beams)
    stream = torch.cuda.current_stream()
    base = lsm.RunOpts(electron_mode=1, n_batches=n_batches)

    def timed(fn, k):
        ms = []
        for r in range(k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            out = fn(r)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms)), out

    # batched arm: launch parameters tuned on this plan (graph replay among them)
    psl = lsm.lsm_build_psl(mh, wl.beams, per_psr_hist=n_k)
    plan = int(psl.info["plan_size"])
    opts, tune_rep = autotune.tune(psl, ph, tally, base, cache_path=None,
                                   cands=autotune.candidates(plan, n_batches, ctas=(0,)))

    def batched(r):
        lsm.lsm_tally_reset(tally)
        g = lsm.lsm_build_psl(mh, wl.beams, per_psr_hist=n_k)      # the plan build is part of the arm
        lsm.lsm_run(g, ph, tally, 10 + r, dataclasses.replace(opts, use_graph=False))
        return g

    # (a new plan object per run would defeat the graph cache: replay the tuned plan's graph)
    def batched_replay(r):
        lsm.lsm_tally_reset(tally)
        lsm.lsm_run(psl, ph, tally, 10 + r, opts)
        return psl

    batched_replay(0)
    ms_b, _ = timed(batched_replay, reps)
    ms_b_build, _ = timed(batched, 1)
    s1, s2, nb = lsm.lsm_tally_read(tally)
    hist = plan * n_batches
    # columns of Eq. 8: photon PSRs, then one effective electron unit per energy bin
    Ag = lsm.lsm_basis_matrix(tally, psl, ph, units=True)
    # synthetic measurement: an independent basis run, known weights, 0.5 % noise;
    # its per-PSR matrix also chooses the entries u_A is taken over
    batched_replay(989)
    A2g = lsm.lsm_basis_matrix(tally, psl, ph, units=True)
    ref = lsm.lsm_basis_matrix(tally, psl, ph)
    u_b = _u_A(s1, s2, nb, ref)
    # 4x the histories (64 batches): u_A should halve
    o4 = dataclasses.replace(opts, n_batches=4 * n_batches, use_graph=False)
    lsm.lsm_tally_reset(tally)
    ms_4x, _ = timed(lambda r: lsm.lsm_run(psl, ph, tally, 77, o4), 1)
    s1_4, s2_4, nb_4 = lsm.lsm_tally_read(tally)
    u_4x = _u_A(s1_4, s2_4, nb_4, ref)

    # plain arm: one plan and one run per PSR, the same histories per PSR and batch
    lsm.lsm_tally_reset(tally)
    plain_opts = dataclasses.replace(base)

    def plain(r):
        for k in range(m.n_psr):
            nk = np.zeros_like(n_k)
            nk[k] = n_k[k]
            g = lsm.lsm_build_psl(mh, wl.beams, per_psr_hist=nk)
            lsm.lsm_run(g, ph, tally, 20 + k, plain_opts)
        return None

    ms_p, _ = timed(plain, 1)
    s1p, s2p, _ = lsm.lsm_tally_read(tally)
    u_p = _u_A(s1p, s2p, n_batches, ref)         # every cell holds its own PSR's n_batches batches
    t_b, t_p = ms_b / 1e3, ms_p / 1e3
    x_true = W.commissioning_truth(Ag.shape[1])
    rng = np.random.default_rng(3)
    bvec = A2g @ x_true * (1 + 0.005 * rng.standard_normal(Ag.shape[0]))
    scale = 1.0 / np.abs(bvec).max()
    out = {}
    f_opt = None
    for method, name, it, delta in ((0, "active_set", 0, 1e-12), (1, "projected_gradient", 20000, 1e-12),
                                    (2, "projected_gradient_bb", 20000, 1e-12)):
        lsm.lsm_commission(Ag * scale, bvec * scale, method=method, max_iter=it, delta=delta)      # warm-up
        t0 = time.perf_counter()
        x, rep = lsm.lsm_commission(Ag * scale, bvec * scale, method=method, max_iter=it, delta=delta)
        out[name] = {"ms": (time.perf_counter() - t0) * 1e3, "iterations": rep["iterations"],
                     "converged": rep["converged"], "delta": delta,
                     # fit residual and error of the dose the fitted weights predict
                     "fit_residual": float(np.linalg.norm(Ag @ x - bvec) / np.linalg.norm(bvec)),
                     "dose_rel_err": float(np.linalg.norm(A2g @ (x - x_true)) / np.linalg.norm(A2g @ x_true)),
                     "objective": rep["objective"], "kkt": rep["kkt"]}
        if method == 0:
            f_opt = rep["objective"]
        else:
            # the paper's iteration (Sec. 2.2.4), and the same projection with
            # Barzilai-Borwein steps, with a bounded budget: the objective
            # against the active-set minimum of the same problem
            out[name]["objective_gap_rel"] = (rep["objective"] - f_opt) / f_opt
    return {"workload": wl.name, "histories": hist, "A_shape": list(Ag.shape),
            "batched": {"ms": ms_b, "ms_with_plan_build": ms_b_build, "histories_per_s": hist / t_b,
                        "u_A_rel": u_b, "s_to_1pct_A": t_b * (u_b / 0.01) ** 2,
                        "launch": {"chunk": opts.chunk, "ctas_per_sm": opts.ctas_per_sm,
                                   "cuda_graph": bool(opts.use_graph), "autotune_candidates": len(tune_rep["trials"]),
                                   "autotune_trials_ms": [[t["chunk"], int(t["use_graph"]), round(t["ms"], 2)]
                                                          for t in tune_rep["trials"]]}},
            "plain": {"ms": ms_p, "runs": m.n_psr, "histories_per_s": hist / t_p, "u_A_rel": u_p,
                      "s_to_1pct_A": t_p * (u_p / 0.01) ** 2,
                      "how": "one per-PSR plan build and one lsm_run per PSR (300), library defaults"},
            "speedup_batched_over_plain": t_p / t_b,
            "scaling_check": {"histories": 4 * hist, "ms": ms_4x, "u_A_rel": u_4x,
                              "u_ratio_vs_1x": u_4x / u_b, "expected_ratio": 0.5},
            "nnls": out}


def conv_gflop(d: int, h: int, w: int) -> float:
    """Algorithmic FLOPs of the network's 14 3x3x3 convolutions (2 per MAC)."""
    from paper_1503_01725_b300 import denoiser as DZ
    lv = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
    return sum(2.0 * 27 * ci * co * (d >> l) * (h >> l) * (w >> l) for (ci, co), l in zip(DZ.LAYERS, lv)) / 1e9


def denoised_block(lsm, reps: int = 5, case: int = 192):
    """Denoised dose on a held-out 128^3 case (Sec. 3 run-time comparison at
    equal error): MC at 1e6 histories plus the network, against plain MC,
    both judged by a 1e9-history run of the same case."""
    import torch
    from paper_1503_01725_b300 import denoiser as DZ
    from paper_1503_01725_b300 import workloads as W
    net = DZ.load()
    p = DZ.generate([case], n_lo=1_000_000, n_hi=1_000_000, n_ref=1_000_000_000)[0]
    wl = W.workload_denoise(case)
    ph = lsm.lsm_phantom_create(wl.phantom)
    keep = (p["rho"] >= DZ.RHO_MIN).float()
    t_mc, t_net, t_conv, u_lo, u_den, g_den = [], [], [], [], [], []
    for r in range(reps + 1):
        lsm.lsm_timing_enable(False)                   # the MC run and the network untimed by kernel timers
        lo, _, ms = DZ.mc_dose(wl, 1_000_000, 777 + r, ph=ph)
        lo = (lo * keep).contiguous()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        den = lsm.lsm_unet_forward(net, lo, p["rho"])
        b.record()
        torch.cuda.synchronize()
        # a second forward with the per-kernel timers on gives the convolutions' share
        lsm.lsm_timing_enable(True)
        lsm.lsm_timing_read(reset=True)
        lsm.lsm_unet_forward(net, lo, p["rho"])
        torch.cuda.synchronize()
        tm = lsm.lsm_timing_read(reset=True)
        lsm.lsm_timing_enable(False)
        if r == 0:
            continue                                   # warm-up (buffers, graph of the MC run)
        t_mc.append(ms)
        t_net.append(a.elapsed_time(b))
        t_conv.append(tm["conv3d"][0])
        u_lo.append(lsm.lsm_dose_error(lo, p["ref"], p["s_ref"], level=0.5))
        u_den.append(lsm.lsm_dose_error(den, p["ref"], p["s_ref"], level=0.5))
        g_den.append(lsm.lsm_gamma(den, p["ref"], (2.5, 2.5, 2.5), 0.02, 2.0, 0.1)[0])
    T_mc, T_net, T_conv = (float(np.median(x)) / 1e3 for x in (t_mc, t_net, t_conv))
    ulo, uden = float(np.mean(u_lo)), float(np.mean(u_den))
    t_den = T_mc + T_net
    t_plain_same_err = T_mc * (ulo / uden) ** 2
    gf = conv_gflop(128, 128, 128)
    hbm, kind = peaks()
    try:
        with open(PEAKS_PATH) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
            bkind = "measured bf16_tflops (burst: the network is timed alone)"
    except Exception:
        bf16, bkind = 1800.0, "fallback"
    ach = gf / T_conv / 1e3
    # every held-out case (20, fields 4-20 cm), each judged by its own 1e9-history run
    rows = []
    for c in W.DENOISE_TEST:
        q = DZ.generate([c], n_lo=1_000_000, n_hi=1_000_000, n_ref=1_000_000_000)[0]
        dq = lsm.lsm_unet_forward(net, q["lo"], q["rho"])
        rows.append({"case": c, "field_cm": round(float(q["field_cm"]), 2),
                     "gamma": lsm.lsm_gamma(dq, q["ref"], (2.5, 2.5, 2.5), 0.02, 2.0, 0.1)[0],
                     "u_rms": lsm.lsm_dose_error(dq, q["ref"], q["s_ref"], level=0.5),
                     "gamma_mc_1e6": lsm.lsm_gamma(q["lo"], q["ref"], (2.5, 2.5, 2.5), 0.02, 2.0, 0.1)[0]})
    held_out = {"cases": len(rows), "gamma_mean": float(np.mean([r["gamma"] for r in rows])),
                "gamma_min": float(min(r["gamma"] for r in rows)),
                "cases_gamma_ge_99": int(sum(r["gamma"] >= 0.99 for r in rows)),
                "u_rms_mean": float(np.mean([r["u_rms"] for r in rows])),
                "u_rms_max": float(max(r["u_rms"] for r in rows)), "per_case": rows}
    return {"workload": f"denoise-{case} 128^3 (field {wl.extra['field_cm']:.1f} cm), weights unet128.npz",
            "held_out_20": held_out,
            "judge": "1e9-history MC of the same case", "s_mc_1e6": T_mc, "s_network": T_net,
            "s_denoised": t_den, "u_rms_mc_1e6": ulo, "u_rms_denoised": uden,
            "gamma_2pct_2mm_denoised": float(np.mean(g_den)),
            "s_to_1pct_plain": T_mc * (ulo / 0.01) ** 2,
            "s_plain_to_denoised_error": t_plain_same_err, "speedup_at_equal_error": t_plain_same_err / t_den,
            "roofline": {"bound": "tensor", "kernel": "k_conv3d (14 layers)", "achieved": ach, "peak": bf16,
                         "unit": "TFLOP/s", "frac": ach / bf16, "peak_source": bkind,
                         "algorithmic_gflop": gf, "s_conv": T_conv}}


def commission_validation_block(lsm):
    """The commissioning validation loop of Sec. 3.2 (Tables 2-3): PSR doses
    of the 40x40 and 5x5 fields, Eq. 8 by gradient projection, doses of five
    fields for the commissioned and the uncommissioned model against the
    synthetic linac's, timed end to end."""
    import torch
    from paper_1503_01725_b300 import commission as CM
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = CM.run()
    torch.cuda.synchronize()
    return {"case": "water 52x52x30 cm (0.5 cm), 360 PSRs; fields 40/20/10/5/2 cm, commissioned on 40 and 5",
            "s_total": time.perf_counter() - t0, "seconds": rep["seconds"], "histories": rep["histories"],
            "nnls_iterations": rep["nnls"]["iterations"], "factor_rel_err": rep["factor_rel_err"],
            "table": CM.summary(rep),
            "output_factor_max_rel_diff": {"commissioned": rep["output_factors"]["max_rel_diff_commissioned"],
                                           "reference": rep["output_factors"]["max_rel_diff_reference"]}}


def multibeam_block(lsm, W, opts, n_hist: int = 10_000_000, n_batches: int = 16, reps: int = 5):
    """Multi-beam plans of Table 1 (7-beam prostate, 6-beam head and neck) on
    CT-like phantoms: the whole plan (PSL build + run over all beams) per
    step, event-timed, as histories/s and the projected time for 1e9 source
    particles (the paper's T_total column for its analytic source)."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for wl in (W.workload_prostate_7beam(n_hist), W.workload_hn_6beam(n_hist)):
        ph = lsm.lsm_phantom_create(wl.phantom)
        tally = lsm.lsm_tally_create(ph)
        n_plan = n_hist // n_batches
        o = lsm.RunOpts(electron_mode=1, n_batches=n_batches, chunk=opts.chunk, ctas_per_sm=opts.ctas_per_sm,
                        no_sync=True)

        def step(seed):
            lsm.lsm_tally_reset(tally)
            psl = lsm.lsm_build_psl(wl.model, wl.beams, n_plan, async_=True)
            lsm.lsm_run(psl, ph, tally, seed, o)
            return psl

        for r in range(3):
            step(100 + r)
        lsm.lsm_timing_read(reset=True)
        evs, plans = [], []
        torch.cuda.synchronize()
        for r in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plans.append(step(200 + r))
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        psl = plans[-1]
        tm = lsm.lsm_timing_read(reset=True)
        led, st = lsm.lsm_tally_ledger(tally)
        d, sg = lsm.lsm_dose(tally, ph, psl.denom / n_plan)
        t = float(np.median(ms)) / 1e3
        out[wl.name] = {
            "beams": wl.beams.n_beams, "field_cm": float(wl.beams.jaws[0, 1] - wl.beams.jaws[0, 0]),
            "histories": n_plan * n_batches, "ms": t * 1e3, "histories_per_s": n_plan * n_batches / t,
            "s_per_1e9": t * 1e9 / (n_plan * n_batches), "u_mean_rel_D50": u_mean_rel(d, sg),
            "entering_fraction": (st["photons"] + st["electrons"]) / max(st["histories"], 1),
            "kernels_ms": {k: round(v[0] / reps, 4) for k, v in tm.items() if v[0] > 0}}
    return out


def _timed_steps(lsm, wl, opts, n_plan: int, reps: int, seed0: int, model_h=None):
    """Event-timed whole dose calculations (plan build + run) of a workload:
    median ms, the kernel split per step, the last step's dose and sigma, the
    tally and its counters."""
    import torch
    stream = torch.cuda.current_stream()
    ph = lsm.lsm_phantom_create(wl.phantom)
    tally = lsm.lsm_tally_create(ph)
    mh = model_h if model_h is not None else lsm.lsm_model_create(wl.model)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def step(seed):
        lsm.lsm_tally_reset(tally)
        psl = lsm.lsm_build_psl(mh, wl.beams, n_plan, async_=True)
        lsm.lsm_run(psl, ph, tally, seed, opts)
        return psl

    for r in range(2):
        step(seed0 + r)
    torch.cuda.synchronize()
    lsm.lsm_timing_read(reset=True)
    # steps queued back to back, each timed by its own events (L2 flush between
    # them, outside the events), as in the headline loop
    evs, plans = [], []
    torch.cuda.synchronize()
    for r in range(reps):
        flush.fill_(r & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plans.append(step(seed0 + 10 + r))
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    psl = plans[-1]
    tm = lsm.lsm_timing_read(reset=True)
    led, st = lsm.lsm_tally_ledger(tally)
    d, sg = lsm.lsm_dose(tally, ph, psl.denom / n_plan)
    return {"ms": float(np.median(ms)), "kernels_ms": {k: round(v[0] / reps, 4) for k, v in tm.items() if v[0] > 0},
            "dose": d, "sigma": sg, "ledger": led, "stats": st, "tally": tally, "phantom": ph}


def fields_block(lsm, W, opts, n_hist: int = 10_000_000, n_batches: int = 16, reps: int = 5):
    """Open fields of 4, 10 and 20 cm on water and 10 cm on the heterogeneous
    phantom (64^3 voxels of 0.5 cm): the field-size sweep of Table 1 (Sec. 3.1)
    on this engine, histories/s and seconds to 1 % per field."""
    out = {}
    o = dataclasses.replace(opts, n_batches=n_batches, no_sync=True, use_graph=False, first_batch=0)
    n_plan = n_hist // n_batches
    lsm.lsm_timing_enable(True)
    for field, hetero in ((4.0, False), (10.0, False), (20.0, False), (10.0, True)):
        wl = W.workload_field(field, n_hist, hetero)
        r = _timed_steps(lsm, wl, o, n_plan, reps, 300)
        t = r["ms"] / 1e3
        u = u_mean_rel(r["dose"], r["sigma"], wl.phantom.rho)
        st = r["stats"]
        out[wl.name] = {"field_cm": field, "phantom": "heterogeneous" if hetero else "water",
                        "histories": n_plan * n_batches, "ms": r["ms"], "histories_per_s": n_plan * n_batches / t,
                        "u_mean_rel_D50": u, "s_to_1pct": t * (u / 0.01) ** 2,
                        "entering_fraction": (st["photons"] + st["electrons"]) / max(st["histories"], 1),
                        "kernels_ms": r["kernels_ms"]}
    lsm.lsm_timing_enable(False)
    return out


def precision_block(lsm, W, opts, n_hist: int = 100_000_000, n_batches: int = 16, reps: int = 3):
    """The precision case: 256x256x160 heterogeneous phantom at 0.25 cm, 1e8
    histories, FP32 transport with FP32 partial slices folded into the FP64
    tally. Its error against the FP64 oracle is measured in the CPU-baseline
    leg on the dose kept here."""
    wl = W.workload_hetero(n_hist)
    n_plan = n_hist // n_batches
    o = dataclasses.replace(opts, n_batches=n_batches, no_sync=True, use_graph=False, first_batch=0,
                            chunk=1 << 24)
    lsm.lsm_timing_enable(True)
    r = _timed_steps(lsm, wl, o, n_plan, reps, 500)
    lsm.lsm_timing_enable(False)
    s1, s2, nb = lsm.lsm_tally_read(r["tally"])
    t = r["ms"] / 1e3
    u = u_mean_rel(r["dose"], r["sigma"], wl.phantom.rho)
    led = r["ledger"]
    # an independent run (another seed) chooses the voxels the oracle
    # comparison uses, so that neither compared estimate selects itself
    mh = lsm.lsm_model_create(wl.model)
    lsm.lsm_tally_reset(r["tally"])
    lsm.lsm_run(lsm.lsm_build_psl(mh, wl.beams, n_plan), r["phantom"], r["tally"], 9999,
                dataclasses.replace(o, no_sync=False))
    sel_s1, _, _ = lsm.lsm_tally_read(r["tally"])
    out = {"workload": wl.name, "histories": n_plan * n_batches, "ms": r["ms"],
           "histories_per_s": n_plan * n_batches / t, "u_mean_rel_D50": u, "s_to_1pct": t * (u / 0.01) ** 2,
           "kernels_ms": r["kernels_ms"],
           # FP32 transport and FP32 partial tallies against FP64 bookkeeping of the same run:
           # the energy ledger (FP64 sums of FP32 values) against the source energy, and the
           # folded FP64 tally against the ledger's deposited energy
           "energy_balance_rel": abs(led["source"] - led["rejected"] - led["escaped"] - led["deposited"])
           / led["source"],
           "tally_vs_ledger_rel": float(s1.sum() / led["deposited"] - 1)}
    return out, {"s1": s1, "s2": s2, "n_batches": nb, "n_hist": n_plan * n_batches, "shape": wl.phantom.rho.shape,
                 "select": sel_s1}


def precision_vs_oracle(keep, n_o: int = 6_000_000, plan_o: int = 375_000):
    """CPU-baseline leg of the precision case: an independent FP64 oracle run
    of n_o histories (disjoint batches over the host's cores) timed and
    compared voxel by voxel with the GPU's 1e8-history dose: fraction of |z| < 3
    over voxels above 10 % of the maximum, and the mean dose ratio with its
    statistical sigma."""
    from oracle import oracle as O
    from oracle import pool
    nz, ny, nx = keep["shape"]
    c = nx // 2
    box = ((0, nz), (c - 32, c + 32), (c - 32, c + 32))
    b_o = n_o // plan_o
    r = pool.run_batches("workload_hetero", n_o, plan_o, b_o, seed=17, box=box)
    dg, sg = O.dose_and_sigma(keep["s1"], keep["s2"], keep["n_batches"])
    dg = dg.reshape(nz, ny, nx)[:, c - 32:c + 32, c - 32:c + 32] / keep["n_hist"]
    sg = sg.reshape(nz, ny, nx)[:, c - 32:c + 32, c - 32:c + 32] / keep["n_hist"]
    do, so = O.dose_and_sigma(r["s1"], r["s2"], b_o)
    do, so = do / n_o, so / n_o
    # voxels above 10 % of the maximum of an independent GPU run (no selection bias)
    ref = keep["select"].reshape(nz, ny, nx)[:, c - 32:c + 32, c - 32:c + 32]
    sel = ref > 0.1 * ref.max()
    z = (dg - do)[sel] / np.sqrt(sg[sel] ** 2 + so[sel] ** 2 + 1e-300)
    ratio = float(dg[sel].sum() / do[sel].sum())
    sig_ratio = float(np.sqrt((sg[sel] ** 2).sum()) / dg[sel].sum() + np.sqrt((so[sel] ** 2).sum()) / do[sel].sum())
    return {"kind": "oracle", "value": n_o / r["run_s"], "unit": "histories/s", "cores": r["processes"],
            "sample": f"{n_o} histories of the precision case as {b_o} batches of {plan_o} over "
                      f"{r['processes']} processes, {r['wall_s']:.1f} s with set-up",
            "voxels_compared": int(sel.sum()), "z_pass_frac": float(np.mean(np.abs(z) < 3)),
            "mean_dose_ratio_gpu_over_oracle": ratio, "mean_dose_ratio_sigma": sig_ratio,
            "oracle_max_history_imbalance": float(r["max_balance"])}


def headline_vs_oracle(keep, seed: int = 23):
    """CPU-baseline leg of the headline workload: the FP64 oracle runs the
    same plan (the step's 16 batches of its batch-size plan, one seed of its
    own) on the host's cores, and its dose per history is compared voxel by
    voxel with the GPU's FP32 step: fraction of |z| < 3 over voxels above 10 %
    of the maximum (chosen on another GPU step), and the mean dose ratio with
    its statistical sigma."""
    from oracle import oracle as O
    from oracle import pool
    nz, ny, nx = keep["shape"]
    box = ((0, nz), (0, ny), (0, nx))
    nb = keep["n_batches"]
    r = pool.run_batches("workload_full_10x10", keep["n_hist"], keep["n_plan"], nb, seed=seed, box=box)
    dg, sg = O.dose_and_sigma(keep["s1"], keep["s2"], nb)
    dg, sg = dg.reshape(nz, ny, nx) / keep["n_hist"], sg.reshape(nz, ny, nx) / keep["n_hist"]
    n_o = keep["n_plan"] * nb
    do, so = O.dose_and_sigma(r["s1"], r["s2"], nb)
    do, so = do / n_o, so / n_o
    ref = keep["select"].reshape(nz, ny, nx)
    sel = ref > 0.1 * ref.max()
    z = (dg - do)[sel] / np.sqrt(sg[sel] ** 2 + so[sel] ** 2 + 1e-300)
    ratio = float(dg[sel].sum() / do[sel].sum())
    sig_ratio = float(np.sqrt((sg[sel] ** 2).sum()) / dg[sel].sum() + np.sqrt((so[sel] ** 2).sum()) / do[sel].sum())
    return {"kind": "oracle", "value": n_o / r["run_s"], "unit": "histories/s", "cores": r["processes"],
            "sample": f"{n_o} histories of the headline workload as {nb} batches of {keep['n_plan']} over "
                      f"{r['processes']} processes, {r['wall_s']:.1f} s with set-up",
            "voxels_compared": int(sel.sum()), "z_pass_frac": float(np.mean(np.abs(z) < 3)),
            "mean_dose_ratio_gpu_over_oracle": ratio, "mean_dose_ratio_sigma": sig_ratio,
            "oracle_max_history_imbalance": float(r["max_balance"])}


def _fs_type(path: str) -> str:
    """File-system type of the mount holding `path` (from /proc/mounts)."""
    best, kind = "", "unknown"
    try:
        with open("/proc/mounts") as f:
            for ln in f:
                parts = ln.split()
                if len(parts) >= 3 and path.startswith(parts[1]) and len(parts[1]) > len(best):
                    best, kind = parts[1], parts[2]
    except OSError:
        pass
    return kind


def pslfile_block(lsm, W, n_file: int = 1 << 24, n_batches: int = 10):
    """The comparator of Table 1: dose from PSL files on disk (read, copy to
    the GPU, translate there, transport) against particles sampled on the fly
    from the analytic model, at equal histories, for a 10x10 and a 2x2 cm2
    field. The file holds every history of a 40x40 cm2 plan of the same
    model; each field reads the records of the PSL cells it includes."""
    import torch
    wl = W.workload_full_10x10()
    ph = lsm.lsm_phantom_create(wl.phantom)
    d = tempfile.mkdtemp(prefix="lsm_pslfile_")
    path = os.path.join(d, "open40.psl")
    try:
        open_plan = lsm.lsm_build_psl(wl.model, W.beams(W.square_field(40.0)), n_file)
        t0 = time.perf_counter()
        lsm.lsm_pslfile_write(open_plan, 4242, path)
        t_write = time.perf_counter() - t0
        del open_plan
        fields = {}
        stream = torch.cuda.current_stream()
        for size in (10.0, 2.0):
            beams = W.beams(W.square_field(size))
            field = lsm.lsm_build_psl(wl.model, beams, 1000)
            t = lsm.lsm_tally_create(ph)
            opts = lsm.RunOpts(n_batches=n_batches)
            lsm.lsm_pslfile_run(path, field, ph, t, 1, n_batches=n_batches, opts=opts)     # warm-up
            runs = {}
            for cold in (True, False):
                lsm.lsm_tally_reset(t)
                lsm.lsm_timing_read(reset=True)
                st = lsm.lsm_pslfile_run(path, field, ph, t, 2, n_batches=n_batches, cold=cold, opts=opts)
                tm = lsm.lsm_timing_read(reset=True)
                runs["cold" if cold else "page_cache"] = {
                    "s_total": st["t_total_s"], "s_read": st["t_read_s"], "s_copy": st["t_copy_s"],
                    "s_translate": tm["sample"][0] / 1e3,
                    "s_transport": (tm["photon"][0] + tm["annihilation_photon"][0] + tm["electron"][0]) / 1e3,
                    "GB_read": st["bytes"] / 1e9, "cache_dropped": bool(st["cold"])}
            n = int(st["records"])
            # the analytic source at the same histories (n_batches passes over
            # a plan of n / n_batches): plan build + sampled run
            lsm.lsm_tally_reset(t)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = lsm.lsm_build_psl(wl.model, beams, -(-n // n_batches))
            torch.cuda.synchronize()
            t_init = time.perf_counter() - t0
            lsm.lsm_run(g, ph, t, 3, opts)                                               # warm-up
            lsm.lsm_tally_reset(t)
            lsm.lsm_timing_read(reset=True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a.record(stream)
            lsm.lsm_run(g, ph, t, 4, opts)
            b.record(stream)
            torch.cuda.synchronize()
            t_run = time.perf_counter() - t0
            tm = lsm.lsm_timing_read(reset=True)
            cold = runs["cold"]
            fields[f"{size:g}x{size:g}"] = {
                "histories": n, "histories_analytic": -(-n // n_batches) * n_batches, "psl_files": runs,
                "analytic": {"s_total": t_init + t_run, "s_src_init": t_init, "s_run_events": a.elapsed_time(b) / 1e3,
                             "s_gen_translate": tm["sample"][0] / 1e3,
                             "s_transport": (tm["photon"][0] + tm["annihilation_photon"][0] + tm["electron"][0]) / 1e3},
                "speedup_analytic_vs_cold_files": cold["s_total"] / (t_init + t_run),
                "read_share_cold": cold["s_read"] / cold["s_total"]}
        return {"file": {"records": n_file, "GB": os.path.getsize(path) / 1e9, "s_write": t_write,
                         "fs": _fs_type(d), "plan": "40x40 cm2, all PSLs"},
                "n_batches": n_batches, "fields": fields}
    finally:
        try:
            os.remove(path)
        except OSError:
            pass
        os.rmdir(d)


def run_reference(args, rank, world):
    """The CPU oracle, as it stands, timed on this host (reference arm)."""
    from paper_1503_01725_b300 import workloads as W
    if rank != 0:
        return
    wl = W.workload_full_10x10(args.n_hist)
    per = 50_000
    pool, n = oracle_pool(wl, per, wl.electron_mode)
    try:
        for i in range(args.warmup):
            pool.map(_oracle_pass, range(10 + i * n, 10 + (i + 1) * n), chunksize=1)
        t0 = time.perf_counter()
        for i in range(args.steps):
            pool.map(_oracle_pass, range(100_000 + i * n, 100_000 + (i + 1) * n), chunksize=1)
        el = time.perf_counter() - t0
    finally:
        pool.terminate()
        pool.join()
    rate = n * per * args.steps / el
    line = {
        "impl": "reference", "metric": "histories/s", "value": rate, "unit": "histories/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n_hist_workload": args.n_hist,
                   "sample": f"{n} x {per} histories per step (one pass of a {per}-history plan of the same "
                             f"workload in each of {n} processes, disjoint seeds)"},
        "cpu_baseline": {"value": rate, "unit": "histories/s", "cores": n, "kind": "oracle",
                         "sample": f"{args.steps} x {n} x {per} histories"},
        "e2e": {"value": rate, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        # tally sums over NCCL, host scalars (timing) over gloo
        dist.init_process_group("cpu:gloo,cuda:nccl", device_id=torch.device("cuda", local))
    from paper_1503_01725_b300 import lsm
    from paper_1503_01725_b300 import workloads as W

    lsm.load_library()
    wl = W.workload_full_10x10(args.n_hist)
    n_plan = args.n_hist // args.n_batches
    opts = lsm.RunOpts(electron_mode=1, n_batches=args.n_batches, chunk=args.chunk,
                       first_batch=rank_first_batch(rank, args.n_batches))
    seed0 = SEED
    stream = torch.cuda.current_stream()

    # device-resident inputs: phantom and tally created once
    ph = lsm.lsm_phantom_create(W.Phantom(**{**wl.phantom.__dict__,
                                            "rho": torch.tensor(wl.phantom.rho, device="cuda"),
                                            "mat": torch.tensor(wl.phantom.mat, device="cuda")}))
    ph.desc = wl.phantom
    tally = lsm.lsm_tally_create(ph)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    tuned = None
    if not args.no_autotune and args.chunk == 0:
        # launch parameters picked on this device before the warm-up (untimed)
        from paper_1503_01725_b300 import autotune
        psl_t = lsm.lsm_build_psl(wl.model, wl.beams, n_plan)
        # the step rebuilds its plan, so a run graph (captured per plan) would be
        # re-captured every step: tune without graph replay
        cands = autotune.candidates(n_plan, args.n_batches, graphs=(False,))
        opts, rep = autotune.tune(psl_t, ph, tally, opts, cache_path=None, cands=cands)
        tuned = {"chunk": opts.chunk, "ctas_per_sm": opts.ctas_per_sm, "use_graph": opts.use_graph,
                 "candidates": len(rep["trials"])}
        del psl_t

    # the step is queued without host synchronisation: the plan build does
    # not wait for its results (read when the dose scale is needed, by then
    # long done) and the run does not wait for its overflow counter
    # (checked from the run statistics after the timed steps)
    step_opts = dataclasses.replace(opts, no_sync=True)

    # the linac's PSR model is loaded once, like the phantom (lsm_model_create)
    model_h = lsm.lsm_model_create(wl.model)
    from paper_1503_01725_b300 import dist as DP

    def step(i):
        psl = lsm.lsm_build_psl(model_h, wl.beams, n_plan, async_=True)
        lsm.lsm_tally_reset(tally)
        lsm.lsm_run(psl, ph, tally, seed0 + i, step_opts)
        if world > 1:
            DP.reduce_tally(lsm, tally)            # the one exchange step: sum of the ranks' tallies
        d, s = lsm.lsm_dose(tally, ph, psl.denom / n_plan, device=True)
        return psl, d, s

    # End-to-end figures first: an nvidia-smi sampler that has run in this
    # process's lifetime was measured to slow the host-side calls of later
    # end-to-end steps by about a quarter (1.9 -> 2.4 ms per step; the
    # device-timed steps are unaffected), and clocks are sampled for the
    # device-timed steps only.
    # end-to-end through the public API with host buffers: every step creates
    # the phantom from pinned host arrays, builds the plan from the host model,
    # runs, and reads the dose and its sigma back into pinned host memory
    e2e_s, h2d, d2h = [], 0, 0
    e2e_opts = dataclasses.replace(opts, use_graph=False, no_sync=True)   # one-shot runs: nothing to replay
    host_ph = W.Phantom(**{**wl.phantom.__dict__, "rho": torch.from_numpy(wl.phantom.rho).pin_memory(),
                           "mat": torch.from_numpy(wl.phantom.mat).pin_memory()})
    out_d = torch.empty(wl.phantom.nvox, dtype=torch.float64).pin_memory()
    out_s = torch.empty(wl.phantom.nvox, dtype=torch.float64).pin_memory()
    # every call only queues its work on the step's stream (the phantom's
    # input check is left to the device and reported by lsm_dose); the host
    # waits once, for the dose
    def e2e_enqueue(i, stream):
        phh = lsm.lsm_phantom_create(host_ph, stream=stream, async_=True)   # host rho/mat -> device
        phh.desc = wl.phantom
        psl = lsm.lsm_build_psl(wl.model, wl.beams, n_plan, async_=True, stream=stream)   # host model -> handle -> device
        tt = lsm.lsm_tally_create(phh, stream=stream)
        lsm.lsm_run(psl, phh, tt, 5000 + i, e2e_opts, stream=stream)
        return phh, psl, tt, stream

    def e2e_read(job, out):
        phh, psl, tt, stream = job
        if world > 1:
            DP.reduce_tally(lsm, tt, stream=stream)
        return lsm.lsm_dose(tt, phh, psl.denom / n_plan, out=out, stream=stream)   # device -> host, waits

    # one step at a time: each call sequence completes before the next starts;
    # two untimed steps first (the memory pool grows to hold a second tally's
    # workspace, as the device-timed loop has its own warm-up)
    for i in range(2 + max(4, min(6, args.steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dose, sig = e2e_read(e2e_enqueue(i, torch.cuda.current_stream()), (out_d, out_s))
        if i >= 2:
            e2e_s.append(time.perf_counter() - t0)
    h2d = wl.phantom.rho.nbytes + wl.phantom.mat.nbytes + sum(
        np.asarray(getattr(wl.model, k)).nbytes for k in ("w", "mix_c", "mix_mu", "mix_sa", "mix_sb", "e_sa", "e_sb")) \
        + wl.beams.jaws.nbytes
    d2h = dose.nbytes + sig.nbytes
    print("e2e per-step ms: " + " ".join(f"{v * 1e3:.3f}" for v in e2e_s), file=sys.stderr)
    e2e_serial_rate = world * args.n_hist / statistics.median(e2e_s)
    # a stream of dose calculations on two CUDA streams: step i's upload and run
    # are queued before step i-1's dose is read back, so that the read-back and
    # the host's calls overlap device work; every step still uploads its own
    # inputs from pinned memory and reads its dose and sigma into pinned memory
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [(out_d, out_s), (torch.empty_like(out_d).pin_memory(), torch.empty_like(out_s).pin_memory())]
    n_pipe = 12
    reps = []
    for rep in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = None
        for i in range(n_pipe):
            job = e2e_enqueue(100 * rep + i, streams[i % 2])
            if prev is not None:
                e2e_read(prev, outs[(i - 1) % 2])
            prev = job
        e2e_read(prev, outs[(n_pipe - 1) % 2])
        reps.append(time.perf_counter() - t0)
        del prev, job
    e2e_rate = world * args.n_hist * n_pipe / statistics.median(reps)
    # leave nothing of the end-to-end steps behind: their handles freed, and
    # the memory pool (grown by two concurrent workspaces) trimmed back, so
    # that the device-timed steps start from the state they run in
    del host_ph, outs, streams
    import gc
    gc.collect()
    torch.cuda.synchronize()
    try:
        from cuda.bindings import runtime as _rt
        _err, _pool = _rt.cudaDeviceGetDefaultMemPool(local)
        _rt.cudaMemPoolTrimTo(_pool, 0)
        torch.cuda.synchronize()
    except Exception:
        pass

    clk = ClockSampler(local).start()
    # The headline steps run without the library's kernel-group event timers
    # (their events between kernels cost about 0.01 ms per step); the kernel
    # split comes from as many further steps with the timers on. A captured
    # graph holds its timers, so a graph-replayed step keeps them on throughout.
    split_timers_apart = not step_opts.use_graph
    lsm.lsm_timing_enable(not split_timers_apart)
    for i in range(args.warmup):
        step(1000 + i)
    torch.cuda.synchronize()
    # the plan build's launches follow the host: while nvidia-smi settles into
    # its sampling (it takes driver locks) the first steps after its start were
    # measured up to 0.3 ms slower; a second of untimed steps lets it settle
    t_settle = time.time() + 1.0
    while time.time() < t_settle:
        step(2000)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    lsm.lsm_timing_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = lsm.lsm_launch_count()
    # The steps are queued back to back, as a stream of dose calculations
    # runs: the host does not wait for one step before queueing the next, so
    # its calls overlap the previous step's device work instead of delaying
    # the step's first kernels. Each step's device time is taken by its own
    # pair of events; the L2 flush between steps lies outside them. Plans and
    # doses are kept until the last step has run.
    keep = []
    torch.cuda.synchronize()
    tw0 = time.time()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                      # L2 flush outside the timed events
        ev[i][0].record(stream)
        keep.append(step(i))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk.window(tw0, time.time())
    clk.stop()
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    u_vals = [u_mean_rel(d.cpu().numpy(), s.cpu().numpy()) for _, d, s in keep]
    del keep
    print("per-step ms: " + " ".join(f"{v:.3f}" for v in ms_steps), file=sys.stderr)
    launches = lsm.lsm_launch_count() - launches0
    if split_timers_apart:
        lsm.lsm_timing_enable(True)
        lsm.lsm_timing_read(reset=True)
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            step(3000 + i)
        torch.cuda.synchronize()
    timers = lsm.lsm_timing_read(reset=True)
    lsm.lsm_timing_enable(False)
    led, st = lsm.lsm_tally_ledger(tally)      # counters of the last step (reset each step)
    if world > 1:                              # summed over the ranks: per-rank work below
        st = {k: v // world for k, v in st.items()}
    total_ms = float(sum(ms_steps))
    total_ms = slowest_ms(total_ms, world)
    if world > 1:
        dist.barrier()


    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    hist_total = world * args.n_hist * args.steps
    value = hist_total / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps
    u = float(np.mean(u_vals))
    t1 = ms_per_step / 1e3 * (u / 0.01) ** 2

    # roofline of the dominant kernel group, algorithmic bytes / event-timed duration
    hbm, hbm_kind = peaks()
    n_st = args.steps
    per_step = {k: v[0] / n_st for k, v in timers.items()}
    units = {
        "sample": (st["photons"] + st["electrons"]) * B_SAMPLE_PER_ENTERING,
        "photon": st["flights"] * B_FLIGHT + st["photons"] * B_QUEUE + st["secondaries"] * B_QUEUE
        + max(st["real"] - st["secondaries"], 0) * B_DEPOSIT,
        "electron": st["esteps"] * B_ESTEP + (st["electrons"] + st["secondaries"]) * B_QUEUE,
    }
    dom = max(("sample", "photon", "electron"), key=lambda k: per_step[k])
    achieved = units[dom] / (per_step[dom] / 1e3) / 1e9
    traffic = None
    if dom in TRAFFIC_PER_UNIT and TRAFFIC_PER_UNIT[dom] is not None:
        unit_key, per = TRAFFIC_PER_UNIT[dom]
        traffic = per * st[unit_key]                       # bytes per step, like achieved
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "traffic_unit": "bytes per step",
                "peak_source": f"{hbm_kind} hbm_gbs",
                "algorithmic_bytes_per_step": units[dom],
                # every kernel group of the step on the same terms (algorithmic
                # bytes per step over its event-timed time per step)
                "by_kernel": {k: {"ms_per_step": per_step[k], "algorithmic_bytes_per_step": units[k],
                                  "achieved": units[k] / (per_step[k] / 1e3) / 1e9,
                                  "frac": units[k] / (per_step[k] / 1e3) / 1e9 / hbm}
                              for k in ("sample", "photon", "electron") if per_step.get(k, 0) > 0}}

    # the tally-update ceiling: FP32 atomics to scattered cells of a tally the
    # size of this run's batch slots, against the transport's step rates
    # (each Woodcock flight or CSDA step makes at most one tally update)
    n_cells = wl.phantom.nvox * args.n_batches
    peak_at = lsm.lsm_l2_atomic_peak(n_cells)
    l2_atomics = {"peak_atomics_per_s": peak_at, "cells": n_cells,
                  "source": "lsm_l2_atomic_peak (FP32 atomicAdd, result unused, LCG-scattered cells)"}
    for k, units_k in (("photon", st["flights"]), ("electron", st["esteps"])):
        if per_step.get(k, 0) > 0:
            r = units_k / (per_step[k] / 1e3)
            l2_atomics[f"{k}_steps_per_s"] = r
            l2_atomics[f"{k}_frac"] = r / peak_at if peak_at > 0 else None

    # two more (untimed) steps of the headline workload for its comparison with
    # the FP64 oracle in the CPU leg: the first chooses the voxels, the second
    # is compared (no selection bias)
    keep_h = None
    if not args.no_cpu_baseline and world == 1:
        step(7001)
        sel_h, _, _ = lsm.lsm_tally_read(tally)
        step(7002)
        s1_h, s2_h, nb_h = lsm.lsm_tally_read(tally)
        keep_h = {"s1": s1_h, "s2": s2_h, "n_batches": nb_h, "n_hist": args.n_hist, "select": sel_h,
                  "n_plan": n_plan, "shape": wl.phantom.rho.shape}

    # the other blocks run after the timed steps: run before them, the PSL-file
    # block (file writes and reads of 0.5 GB, a memory pool grown to 5.6 GB)
    # was measured to slow the plan build's kernel launches in later steps
    # (1.66 -> 2.0 ms per step; 1.73 ms after trimming the pool)
    batched = None
    if not args.no_batched:
        batched = commissioning_block(lsm, W)
    denoised = None
    if not args.no_denoised:
        lsm.lsm_timing_enable(True)
        denoised = denoised_block(lsm)
        lsm.lsm_timing_enable(False)
    validation = None
    if not args.no_validation:
        validation = commission_validation_block(lsm)
    multibeam = None
    if not args.no_multibeam:
        lsm.lsm_timing_enable(True)
        multibeam = multibeam_block(lsm, W, opts)
        lsm.lsm_timing_enable(False)
    fields = None
    if not args.no_fields:
        fields = fields_block(lsm, W, opts)
    precision, keep = None, None
    if not args.no_precision:
        precision, keep = precision_block(lsm, W, opts)
    pslfile = None
    if not args.no_pslfile:
        lsm.lsm_timing_enable(True)
        pslfile = pslfile_block(lsm, W)
        lsm.lsm_timing_enable(False)
    cpu = None
    if not args.no_cpu_baseline:
        rate, n_done, el, n_proc = cpu_oracle_rate_all_cores(wl, args.cpu_seconds)
        rate1, n_done1, el1 = cpu_oracle_rate(wl, args.cpu_seconds / 3)
        cpu = {"value": rate, "unit": "histories/s", "cores": n_proc, "kind": "oracle",
               "sample": f"{n_done} histories as 1e5-history plans of the same workload in {n_proc} processes "
                         f"(disjoint seeds), {el:.1f} s",
               "one_core": {"value": rate1, "cores": 1,
                            "sample": f"{n_done1} histories as 1e5-history plans, {el1:.1f} s"}}
        if keep_h is not None:
            # the headline dose's error against the FP64 oracle, same workload and size
            cpu["headline_vs_oracle"] = headline_vs_oracle(keep_h)
        if keep is not None:
            # the precision case's error against the FP64 oracle (FP32 transport, FP32 partials)
            cpu["precision_case"] = precision_vs_oracle(keep)
    line = {
        "metric": "histories/s", "value": value, "unit": "histories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "n_hist": args.n_hist, "n_batches": args.n_batches,
                   "histories_per_iteration": iteration_size(opts, n_plan),
                   "ctas_per_sm": opts.ctas_per_sm, "cuda_graph": bool(opts.use_graph), "autotuned": tuned,
                   "phantom": "water 64^3 x 0.25 cm", "field_cm": 10,
                   "sub_sources": 3, "electrons": "CSDA",
                   "parallelism": (f"data-parallel x{world}: disjoint batch ranges of one seed, "
                                   "tally summed over ranks (NCCL) in every step") if world > 1 else "1 GPU",
                   "l2": "flushed by a 512 MiB write before each step, outside the timed events"},
        "s_to_1pct": t1, "u_mean_rel_D50": u,
        "kernels_ms_per_step": {k: round(v, 4) for k, v in per_step.items() if v > 0},
        "work_per_step": {"photons": st["photons"], "electrons": st["electrons"], "flights": st["flights"],
                          "real": st["real"], "secondaries": st["secondaries"], "esteps": st["esteps"],
                          "rejected": st["rejected"], "queue_overflows": st["overflows"]},
        "roofline": roofline,
        "l2_atomics": l2_atomics,
        "batched": batched,
        "denoised": denoised,
        "commissioning_validation": validation,
        "multibeam": multibeam,
        "fields": fields,
        "precision": precision,
        "pslfile": pslfile,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_serial_rate, "unit": "histories/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "how": "one step at a time, each completed (dose and sigma in pinned host memory) before "
                       "the next starts; median of 4-6 steps after 2 untimed ones",
                "pipelined": {"value": e2e_rate,
                              "how": "12 steps on two CUDA streams, each step's read-back and host calls "
                                     "overlapping the next step's upload and run; median of 3 repetitions"}},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
