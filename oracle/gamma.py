"""Global gamma index (Low, Harms, Mutic & Purdy, Med. Phys. 25, 656 (1998))
and error statistics used to judge a dose estimate against a reference dose
(test and measurement infrastructure; not part of the product path).

For every reference voxel above a threshold, gamma is the minimum over points
r of sqrt(|r - r_ref|^2 / DTA^2 + (D_eval(r) - D_ref)^2 / (c Dmax_ref)^2),
with D_eval interpolated trilinearly. A point can only reach gamma <= 1 within
distance DTA, so the search covers the DTA sphere on a grid of step `step_mm`.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def gamma_pass_rate(d_eval, d_ref, voxel_mm, dose_crit: float = 0.02, dta_mm: float = 2.0,
                    threshold: float = 0.1, step_mm: float = 0.5):
    """(fraction of reference voxels above threshold * max(d_ref) with gamma
    <= 1, number of such voxels). voxel_mm: (z, y, x) voxel size."""
    d_eval = np.asarray(d_eval, dtype=np.float64)
    d_ref = np.asarray(d_ref, dtype=np.float64)
    vz, vy, vx = voxel_mm
    dmax = d_ref.max()
    roi = np.argwhere(d_ref > threshold * dmax)
    if len(roi) == 0:
        return 1.0, 0
    dref = d_ref[tuple(roi.T)]
    crit = dose_crit * dmax
    # offsets within the DTA sphere, nearest first
    k = int(np.floor(dta_mm / step_mm))
    g = np.arange(-k, k + 1) * step_mm
    oz, oy, ox = np.meshgrid(g, g, g, indexing="ij")
    r2 = oz ** 2 + oy ** 2 + ox ** 2
    keep = r2 <= dta_mm ** 2 + 1e-12
    order = np.argsort(r2[keep], kind="stable")
    offs = np.stack([oz[keep], oy[keep], ox[keep]], axis=1)[order]
    dist2 = r2[keep][order] / dta_mm ** 2
    passed = np.zeros(len(roi), bool)
    todo = np.arange(len(roi))
    for (a, b, c), s2 in zip(offs, dist2):
        if todo.size == 0:
            break
        coords = roi[todo].T.astype(np.float64) + np.array([[a / vz], [b / vy], [c / vx]])
        de = ndimage.map_coordinates(d_eval, coords, order=1, mode="nearest")
        ok = s2 + ((de - dref[todo]) / crit) ** 2 <= 1.0
        passed[todo[ok]] = True
        todo = todo[~ok]
    return float(passed.mean()), int(len(roi))


def rms_relative_error(d_est, d_ref, sigma_ref=None, level: float = 0.5):
    """RMS of (d_est - d_ref) / d_ref over voxels with d_ref > level * max(d_ref);
    with sigma_ref (the reference's own standard deviation) its variance is
    subtracted: sqrt(max(mean(e^2) - mean((sigma_ref / d_ref)^2), 0))."""
    d_est = np.asarray(d_est, dtype=np.float64)
    d_ref = np.asarray(d_ref, dtype=np.float64)
    sel = d_ref > level * d_ref.max()
    e2 = np.mean(((d_est[sel] - d_ref[sel]) / d_ref[sel]) ** 2)
    if sigma_ref is not None:
        e2 -= np.mean((np.asarray(sigma_ref, dtype=np.float64)[sel] / d_ref[sel]) ** 2)
    return float(np.sqrt(max(e2, 0.0)))
