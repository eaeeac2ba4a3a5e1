"""Dose denoiser driver: training pairs from the engine, training, evaluation.

    python -m paper_1503_01725_b300.denoiser [--cases 200] [--epochs 12] [--out FILE] [--report FILE]

Pairs: for every seeded 128^3 workload (workloads.workload_denoise) the engine
computes the dose per source particle at 1e6 histories (network input) and at
1e8 histories (training target), with 16 batches for the uncertainty. Dose in
voxels below 0.1 g/cm^3 (air) is left out: dose per gram there rests on a
handful of deposits. Cases 0-179 train the network (lsm_unet_train_step,
Adam); cases 180-199 are judged against a 1e9-history run of the same case:
RMS relative error over D > 50 % Dmax (the judge's own variance removed) and
the global gamma pass rate at 2 %/2 mm (10 % threshold), for the raw 1e6 dose,
the denoised dose and the 1e8 dose. Every step runs in the library's kernels;
PyTorch holds the device arrays.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import lsm
from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "unet128.npz")


def mc_dose(wl: W.Workload, n_hist: int, seed: int, n_batches: int = 16, ph=None):
    """Dose per source particle and its batch sigma (device FP32 [d, h, w]) and
    the device time of the run in ms."""
    import torch
    ph = ph or lsm.lsm_phantom_create(wl.phantom)
    n_plan = n_hist // n_batches
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    # queued without host waits: the plan's results are read when the dose
    # scale needs them, the run leaves its overflow count in the statistics
    psl = lsm.lsm_build_psl(wl.model, wl.beams, n_plan, async_=True)
    tally = lsm.lsm_tally_create(ph)
    lsm.lsm_run(psl, ph, tally, seed, lsm.RunOpts(electron_mode=wl.electron_mode, n_batches=n_batches, no_sync=True))
    d, s = lsm.lsm_dose(tally, ph, psl.denom / n_plan, device=True)
    b.record()
    torch.cuda.synchronize()
    shp = (wl.phantom.nz, wl.phantom.ny, wl.phantom.nx)
    return d.float().reshape(shp).contiguous(), s.float().reshape(shp).contiguous(), a.elapsed_time(b)


RHO_MIN = 0.1        # voxels below this density (air) are outside the dose region


def generate(cases, n_lo: int = 1_000_000, n_hi: int = 100_000_000, n_ref: int = 0):
    """Per case, device tensors: lo (input dose), hi (training target), s_hi,
    rho, and with n_ref > 0 a lower-noise judge (ref, s_ref); doses are set to
    zero in voxels below RHO_MIN. Also the device time of the input run (ms)."""
    import torch
    out = []
    for c in cases:
        wl = W.workload_denoise(c)
        ph = lsm.lsm_phantom_create(wl.phantom)
        rho = torch.tensor(wl.phantom.rho, device="cuda").contiguous()
        keep = (rho >= RHO_MIN).float()
        lo, _, t_lo = mc_dose(wl, n_lo, wl.seed, ph=ph)
        hi, s_hi, _ = mc_dose(wl, n_hi, wl.seed + 100000, ph=ph)
        rec = {"lo": lo * keep, "hi": hi * keep, "s_hi": s_hi * keep, "rho": rho, "field_cm": wl.extra["field_cm"],
               "ms_lo": t_lo, "case": c}
        if n_ref:
            ref, s_ref, _ = mc_dose(wl, n_ref, wl.seed + 200000, ph=ph)
            rec["ref"], rec["s_ref"] = ref * keep, s_ref * keep
        out.append(rec)
    return out


# (c_in, c_out) of the 14 conv layers, then a 16 -> 1 head (include/lsm.h)
LAYERS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 64), (128, 64), (64, 32),
          (64, 32), (32, 16), (32, 16), (16, 16)]


def init_params(seed: int = 0, head_scale: float = 0.0) -> np.ndarray:
    """He-normal conv weights (fan-in of the real input channels), zero biases;
    head weights scaled by head_scale (0: the untrained network returns its
    input dose)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co) in enumerate(LAYERS):
        fan = 27 * (2 if i == 0 else ci)
        w = rng.standard_normal((co, 3, 3, 3, ci)) * np.sqrt(2.0 / fan)
        if i == 0:
            w[..., 2:] = 0.0
        parts += [w.ravel(), np.zeros(co)]
    parts += [rng.standard_normal(16) * head_scale, np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == lsm.lsm_unet_param_count()
    return p


def train(pairs, epochs: int = 12, lr: float = 1e-3, seed: int = 0, log=print, transpose: bool = False,
          small_field_power: float = 0.0):
    """Adam over the training pairs: one volume per step, shuffled each epoch,
    random x/y mirroring of input and target together (and, with transpose,
    random exchange of x and y: the square fields and the ring-symmetric source
    make the transposed case a valid case up to the X/Y jaw heights),
    cosine-decayed learning rate. With small_field_power p > 0 an epoch draws
    its cases with replacement, with probability proportional to field_cm^-p
    (small fields, whose penumbrae are a larger part of the dose, come up more
    often). Returns (network, mean loss per epoch, seconds)."""
    import torch
    net = lsm.lsm_unet_create(init_params(seed, head_scale=0.01))
    rng = np.random.default_rng(seed)
    steps, k, hist = epochs * len(pairs), 0, []
    t0 = time.time()
    prob = None
    if small_field_power > 0:
        f = np.array([p["field_cm"] for p in pairs], dtype=np.float64) ** -small_field_power
        prob = f / f.sum()
    for ep in range(epochs):
        losses = []
        order = rng.permutation(len(pairs)) if prob is None else rng.choice(len(pairs), len(pairs), p=prob)
        for i in order:
            lo, hi, rho = pairs[i]["lo"], pairs[i]["hi"], pairs[i]["rho"]
            dims = [d for d, f in ((1, rng.random() < 0.5), (2, rng.random() < 0.5)) if f]
            if dims:
                lo, hi, rho = (torch.flip(t, dims).contiguous() for t in (lo, hi, rho))
            if transpose and rng.random() < 0.5:
                lo, hi, rho = (t.transpose(1, 2).contiguous() for t in (lo, hi, rho))
            lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * k / steps))
            losses.append(lsm.lsm_unet_train_step(net, lo, rho, hi, lr=lr_k))
            k += 1
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.4e} ({time.time() - t0:.0f} s)")
    return net, hist, time.time() - t0


def evaluate(net, pairs, voxel_mm=(2.5, 2.5, 2.5)):
    """Per test case: RMS relative error over D > 50 % Dmax (judge's variance
    removed) and global gamma 2 %/2 mm (10 % threshold) of the input dose and
    of the denoised dose against the judge (ref if generated, else hi), plus
    the device time of the network (ms)."""
    import torch
    rows = []
    for p in pairs:
        ref, s_ref = (p["ref"], p["s_ref"]) if "ref" in p else (p["hi"], p["s_hi"])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        den = lsm.lsm_unet_forward(net, p["lo"], p["rho"])
        b.record()
        torch.cuda.synchronize()
        r = {"case": p["case"], "field_cm": p["field_cm"], "ms_mc_lo": p["ms_lo"], "ms_denoise": a.elapsed_time(b)}
        for name, est in (("mc_lo", p["lo"]), ("denoised", den), ("target_hi", p["hi"])):
            r[f"{name}_rms"] = lsm.lsm_dose_error(est, ref, s_ref, level=0.5)
            r[f"{name}_gamma"] = lsm.lsm_gamma(est, ref, voxel_mm, 0.02, 2.0, 0.1)[0]
        rows.append(r)
    return rows


def load(path: str = WEIGHTS):
    """Network with the stored parameters."""
    z = np.load(path)
    return lsm.lsm_unet_create(z["params"].astype(np.float32))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cases", type=int, default=W.DENOISE_CASES)
    ap.add_argument("--epochs", type=int, default=240)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--n-lo", type=int, default=1_000_000)
    ap.add_argument("--n-hi", type=int, default=100_000_000)
    ap.add_argument("--n-ref", type=int, default=1_000_000_000, help="judge histories for the test cases")
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--report", default=None)
    ap.add_argument("--transpose", action="store_true", help="also exchange x and y at random in training")
    ap.add_argument("--small-field-power", type=float, default=0.0,
                    help="draw training cases with probability proportional to field_cm^-p")
    a = ap.parse_args()
    lsm.load_library()
    n_test = max(1, a.cases // 10)
    train_ids = list(range(0, a.cases - n_test))
    test_ids = list(range(a.cases - n_test, a.cases)) if a.cases < W.DENOISE_CASES else list(W.DENOISE_TEST)
    t0 = time.time()
    tr = generate(train_ids, a.n_lo, a.n_hi)
    te = generate(test_ids, a.n_lo, a.n_hi, a.n_ref)
    t_gen = time.time() - t0
    print(f"generated {len(tr) + len(te)} pairs in {t_gen:.0f} s", flush=True)
    net, hist, t_train = train(tr, a.epochs, a.lr, transpose=a.transpose, small_field_power=a.small_field_power)
    rows = evaluate(net, te)
    params = lsm.lsm_unet_params(net)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.savez(a.out, params=params, epochs=a.epochs, lr=a.lr, n_lo=a.n_lo, n_hi=a.n_hi, transpose=a.transpose,
             small_field_power=a.small_field_power,
             train_cases=np.array(train_ids), test_cases=np.array(test_ids), loss=np.array(hist))
    summary = {k: float(np.mean([r[k] for r in rows])) for k in rows[0] if k not in ("field_cm", "case")}
    summary["gamma_min_denoised"] = float(min(r["denoised_gamma"] for r in rows))
    rep = {"train_cases": len(train_ids), "test_cases": len(test_ids), "epochs": a.epochs, "lr": a.lr,
           "seconds_generate": t_gen, "seconds_train": t_train, "loss_per_epoch": hist, "test_mean": summary,
           "per_case": rows}
    print(json.dumps(summary))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
