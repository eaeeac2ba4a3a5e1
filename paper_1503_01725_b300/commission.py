"""Commissioning validation loop (Sec. 2.2 and Sec. 3.2) above the C ABI.

1. PSR doses (Sec. 2.2.2): one batched basis run per commissioning field
   (40x40 and 5x5 cm2 open fields, SSD 100 cm) filling the PSR-indexed tally
   at the measurement points: the central-axis depth dose and the inline and
   crossline profiles at 1.5, 10 and 20 cm depth. Electron PSRs are grouped
   per energy bin (Sec. 2.2.3) by lsm_basis_matrix_units.
2. "Measurements": the doses of a linac whose PSR weights differ from the
   model's by known correction factors (a synthetic stand-in: no measured data
   exist here), computed by the same engine at high statistics.
3. The correction factors from Eq. 8 (NNLS on the GPU), the commissioned
   model W' = x W (lsm_model_commission), and the doses of five open fields (40, 20, 10, 5, 2 cm)
   for the commissioned and the uncommissioned ("reference") model.
4. The comparison of Sec. 3.2: depth doses (build-up: distance to agreement;
   beyond: RMS and maximum difference, Eq. 10-11) and profiles (inner and
   outer beam: RMS and maximum; penumbra: distance to agreement), and output
   factors (axis dose at 9-11 cm depth relative to the 10x10 field's).

Every dose, fit and comparison runs in liblsm's kernels; this module only
orders the calls and gathers the measurement points out of the dose arrays.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import lsm
from . import workloads as W

FIELDS = (40.0, 20.0, 10.0, 5.0, 2.0)
COMMISSION_FIELDS = (40.0, 5.0)
DEPTHS = (1.5, 10.0, 20.0)


@dataclass
class Case:
    model: W.PSRModel
    phantom: W.Phantom
    idx: np.ndarray        # uint16 (nz, ny, nx): 0 or measurement row + 1
    n_rows: int
    curves: dict           # name -> (positions cm, row indices)


def validation_case(nx: int = 104, nz: int = 60, voxel: float = 0.5, n_r: int = 12, dr: float = 0.35,
                    seed: int = 3, model: W.PSRModel | None = None) -> Case:
    """Water 52 x 52 x 30 cm (0.5 cm voxels) at SSD 100 cm and a 360-PSR model
    (3 sub-sources x 10 energy bins x 12 rings of 0.35 cm: the plane out to
    4.2 cm, 21 cm at the isocentre), or the given model."""
    model = model if model is not None else W.psr_model(10, n_r, dr, seed=seed)
    ph = W.water_phantom(nx, nx, nz, voxel)
    idx, n_rows = W.commissioning_index(ph, DEPTHS)
    cy = cx = nx // 2
    curves = {"pdd": ((np.arange(nz) + 0.5) * ph.dz, idx[:, cy, cx].astype(np.int64) - 1)}
    lat = ph.x0 + (np.arange(nx) + 0.5) * voxel
    for d in DEPTHS:
        k = min(nz - 1, int(d / ph.dz))
        curves[f"crossline@{d:g}"] = (lat, idx[k, cy, :].astype(np.int64) - 1)
        curves[f"inline@{d:g}"] = (lat, idx[k, :, cx].astype(np.int64) - 1)
    return Case(model, ph, idx, n_rows, curves)


def truth_factors(model: W.PSRModel, seed: int = 3) -> np.ndarray:
    """Known per-unit correction factors of the synthetic linac (photon PSRs,
    then one per electron energy bin)."""
    return W.commissioning_truth(2 * model.n_e * model.n_r + model.n_e, seed=seed)


def field_histories(field_cm: float, n_large: float) -> int:
    """Histories for a field: proportional to its area (equal statistics per
    voxel inside the field), at least 5 % of the 40x40 field's."""
    return int(max(n_large * (field_cm / 40.0) ** 2, 0.05 * n_large))


def field_rows(ph_handle, case: Case, model: W.PSRModel, field_cm: float, n_hist: int, seed: int,
               n_batches: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """Dose per source weight (and its batch sigma) at the measurement rows
    for one open field."""
    beams = W.beams(W.square_field(field_cm))
    n_plan = max(n_hist // n_batches, 1)
    psl = lsm.lsm_build_psl(model, beams, n_plan)
    t = lsm.lsm_tally_create(ph_handle)
    lsm.lsm_run(psl, ph_handle, t, seed, lsm.RunOpts(electron_mode=1, n_batches=n_batches))
    d, s = lsm.lsm_dose(t, ph_handle, psl.denom / n_plan)
    sel = case.idx.reshape(-1) > 0
    rows = case.idx.reshape(-1)[sel].astype(np.int64) - 1
    out = np.zeros(case.n_rows)
    sig = np.zeros(case.n_rows)
    out[rows] = d.reshape(-1)[sel]
    sig[rows] = s.reshape(-1)[sel]
    return out, sig


def curve(case: Case, rows: np.ndarray, name: str):
    pos, r = case.curves[name]
    return pos.astype(np.float32), rows[r].astype(np.float32)


def compare_field(case: Case, field_cm: float, calc: np.ndarray, meas: np.ndarray, calc_sig=None,
                  meas_sig=None) -> dict:
    """Sec. 3.2 metrics of one field (fractions of the measured maximum; cm).
    With the batch sigmas of both doses, the depth dose also gets its noise
    floor: the RMS difference that two exact models would show through the
    statistical noise of the two Monte Carlo curves alone."""
    pos, c = curve(case, calc, "pdd")
    _, m = curve(case, meas, "pdd")
    dmax = float(m.max())
    d_max = float(pos[int(np.argmax(m >= 0.99 * dmax))])   # end of the build-up
    bu = lsm.lsm_curve_compare(pos, c, m, -np.inf, d_max, dmax)
    after = lsm.lsm_curve_compare(pos, c, m, d_max, np.inf, dmax)
    out = {"pdd": {"buildup_dta_mean": bu["dta_mean"], "buildup_dta_max": bu["dta_max"],
                   "rms": after["rms"], "max": after["max"]}}
    if calc_sig is not None and meas_sig is not None:
        _, sc = curve(case, calc_sig, "pdd")
        _, sm = curve(case, meas_sig, "pdd")
        k = pos >= d_max
        out["pdd"]["noise_rms"] = float(np.sqrt(np.mean(sc[k].astype(np.float64) ** 2 + sm[k] ** 2)) / dmax)
    for d in DEPTHS:
        w = 0.5 * field_cm * (W.SSD + d) / W.SAD
        for kind in ("inline", "crossline"):
            pos, c = curve(case, calc, f"{kind}@{d:g}")
            _, m = curve(case, meas, f"{kind}@{d:g}")
            inner = lsm.lsm_curve_compare(pos, c, m, 0.0, 0.8 * w, dmax, use_abs=True)
            pen = lsm.lsm_curve_compare(pos, c, m, 0.8 * w, 1.2 * w, dmax, use_abs=True)
            outer = lsm.lsm_curve_compare(pos, c, m, 1.2 * w, np.inf, dmax, use_abs=True)
            out[f"{kind}@{d:g}"] = {"inner_rms": inner["rms"], "inner_max": inner["max"],
                                    "penumbra_dta_mean": pen["dta_mean"], "penumbra_dta_max": pen["dta_max"],
                                    "outer_rms": outer["rms"] if outer["points"] else None,
                                    "outer_max": outer["max"] if outer["points"] else None}
    return out


def run(case: Case | None = None, *, n_large: float = 2e9, hist_lo: int = 20_000, hist_hi: int = 4_000_000,
        basis_batches: int = 4, seed: int = 11, method: int = 1, max_iter: int = 3000, delta: float = 1e-9) -> dict:
    """The whole loop; returns the factors, the per-field metrics for the
    commissioned and the reference model, output factors and timings."""
    import torch
    case = case or validation_case()
    m = case.model
    ph = lsm.lsm_phantom_create(case.phantom)
    t0 = time.perf_counter()
    # 1. PSR doses of the two commissioning fields (one plan, two beams)
    w = m.w.reshape(-1)
    n_k = np.clip(np.round(w / w.max() * hist_hi), hist_lo, hist_hi).astype(np.int64)
    beams = W.beams(*[W.square_field(f) for f in COMMISSION_FIELDS])
    mh = lsm.lsm_model_create(m)
    psl = lsm.lsm_build_psl(mh, beams, per_psr_hist=n_k)
    tb = lsm.lsm_tally_create(ph, mode=1, idx3d=case.idx, n_rows=case.n_rows, n_psr=m.n_psr,
                              n_beams=beams.n_beams)
    lsm.lsm_run(psl, ph, tb, seed, lsm.RunOpts(electron_mode=1, n_batches=basis_batches))
    # columns: photon PSRs, then one effective electron unit per energy bin (Sec. 2.2.3)
    A = lsm.lsm_basis_matrix(tb, psl, ph, units=True)
    torch.cuda.synchronize()
    t_basis = time.perf_counter() - t0
    # 2. measurements of the synthetic linac
    x_true = truth_factors(m)
    m_true = lsm.lsm_model_commission(mh, x_true)
    meas_rs = {f: field_rows(ph, case, m_true, f, field_histories(f, n_large), seed + 100 + k)
               for k, f in enumerate(FIELDS)}
    meas = {f: v[0] for f, v in meas_rs.items()}
    # 3. Eq. 8 on the two commissioning fields (rows beam-major, as A)
    b = np.concatenate([meas[f] for f in COMMISSION_FIELDS])
    scale = 1.0 / np.abs(b).max()
    t1 = time.perf_counter()
    # gradient projection from the uncommissioned weights (x = 1), Sec. 2.2.4
    x, rep = lsm.lsm_commission(A * scale, b * scale, method=method, max_iter=max_iter, delta=delta)
    t_fit = time.perf_counter() - t1
    m_com = lsm.lsm_model_commission(mh, x)
    t2 = time.perf_counter()
    calc_rs = {f: field_rows(ph, case, m_com, f, field_histories(f, n_large), seed + 200 + k)
               for k, f in enumerate(FIELDS)}
    torch.cuda.synchronize()
    t_val = time.perf_counter() - t2
    ref_rs = {f: field_rows(ph, case, mh, f, field_histories(f, n_large), seed + 300 + k)
              for k, f in enumerate(FIELDS)}
    calc = {f: v[0] for f, v in calc_rs.items()}
    ref = {f: v[0] for f, v in ref_rs.items()}
    # 4. comparison
    # output factor: axis dose over 9-11 cm depth relative to the 10x10 field's
    r10 = case.curves["pdd"][1][np.abs(case.curves["pdd"][0] - 10.0) <= 1.0]

    def of(rows):
        return {f"{f:g}": float(rows[f][r10].mean() / rows[10.0][r10].mean()) for f in FIELDS}

    of_meas, of_com, of_ref = of(meas), of(calc), of(ref)
    fields = {}
    for f in FIELDS:
        fields[f"{f:g}x{f:g}"] = {
            "commissioned": compare_field(case, f, calc[f], meas[f], calc_rs[f][1], meas_rs[f][1]),
            "reference": compare_field(case, f, ref[f], meas[f], ref_rs[f][1], meas_rs[f][1])}
    return {
        "x": x, "x_true": x_true, "nnls": rep, "model_handle": m_com,
        "model": m.with_weights(lsm.lsm_model_weights(m_com)),
        "factor_rel_err": float(np.linalg.norm(x - x_true) / np.linalg.norm(x_true)),
        "fields": fields,
        "output_factors": {"measured": of_meas, "commissioned": of_com, "reference": of_ref,
                           "max_rel_diff_commissioned": max(abs(of_com[k] / of_meas[k] - 1) for k in of_meas),
                           "max_rel_diff_reference": max(abs(of_ref[k] / of_meas[k] - 1) for k in of_meas)},
        "histories": {"basis": int(2 * n_k.sum() * basis_batches),
                      "per_model": int(sum(field_histories(f, n_large) // 8 * 8 for f in FIELDS))},
        "seconds": {"basis": t_basis, "fit": t_fit, "validation_doses": t_val},
    }


def write_phase_space(model: W.PSRModel, path: str, n_records: int, seed: int = 1, open_field_cm: float = 40.0):
    """A phase-space file of the (commissioned) model for other Monte Carlo
    codes (Sec. 4): every history of a wide-open plan sampled on the
    phase-space plane and written grouped by PSL cell (lsm_pslfile_write).
    Returns the record count."""
    plan = lsm.lsm_build_psl(model, W.beams(W.square_field(open_field_cm)), n_records)
    return lsm.lsm_pslfile_write(plan, seed, path)


def summary(rep: dict) -> dict:
    """Table 2-3 style ranges over the fields: RMS and Max in percent of the
    measured maximum, distances to agreement in cm."""
    def rng(curve_name, key, which):
        v = [rep["fields"][f][which][curve_name][key] for f in rep["fields"]]
        v = [a for a in v if a is not None]
        if "dta" in key:
            return [round(min(v), 4), round(max(v), 4)]
        return [round(100 * min(v), 3), round(100 * max(v), 3)]
    out = {}
    for which in ("reference", "commissioned"):
        out[which] = {"pdd_buildup_dta_mean_cm": rng("pdd", "buildup_dta_mean", which),
                      "pdd_buildup_dta_max_cm": rng("pdd", "buildup_dta_max", which),
                      "pdd_rms_pct": rng("pdd", "rms", which), "pdd_max_pct": rng("pdd", "max", which),
                      "inline10_inner_rms_pct": rng("inline@10", "inner_rms", which),
                      "inline10_inner_max_pct": rng("inline@10", "inner_max", which),
                      "inline10_penumbra_dta_mean_cm": rng("inline@10", "penumbra_dta_mean", which),
                      "inline10_outer_rms_pct": rng("inline@10", "outer_rms", which)}
        if all("noise_rms" in rep["fields"][f][which]["pdd"] for f in rep["fields"]):
            out[which]["pdd_noise_floor_pct"] = rng("pdd", "noise_rms", which)
    return out


def main():
    rep = run()
    import json
    print(json.dumps({"factor_rel_err": rep["factor_rel_err"], "summary": summary(rep),
                      "output_factors": rep["output_factors"], "seconds": rep["seconds"],
                      "histories": rep["histories"]}, indent=1))


if __name__ == "__main__":
    lsm.load_library()
    main()
