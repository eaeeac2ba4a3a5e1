"""Dose comparison metrics of the commissioning validation (Sec. 3.2) -- TEST
INFRASTRUCTURE ONLY; nothing in the product path imports this module.

Low-gradient regions (depth dose beyond the build-up, the inner and outer
parts of a lateral profile) are judged by the RMS and the maximum of the dose
difference normalised by the measured dose maximum (Eq. 10-11); high-gradient
regions (build-up, penumbra) by the distance to agreement: at a measured
point x, the smallest |x - y| over positions y where the calculated curve
takes the measured value D_m(x). The calculated curve between its sample
points is the straight-line interpolation, continued along its end segments
beyond the first and last points. The split into regions follows
AAPM TG-53 as the paper does: build-up = depths shallower than the first
depth where the measured dose reaches 99 % of its maximum; penumbra = 80-120 % of the geometric field half-width at that
depth, inner and outer beam inside and outside it.
"""
from __future__ import annotations

import math

import numpy as np


def rms_max(calc, meas, dmax_m: float):
    """Eq. 10 and Eq. 11 over the given points (fractions, not percent)."""
    d = np.asarray(calc, np.float64) - np.asarray(meas, np.float64)
    return float(np.sqrt(np.mean(d * d)) / dmax_m), float(np.max(np.abs(d)) / dmax_m)


def dta_point(x: float, m: float, pos, calc) -> float:
    """Distance to agreement at position x for measured value m: minimum of
    |x - y| over y with C(y) = m, C the calculated curve, straight between its
    sample points and continued along its first and last segments beyond the
    end points (a depth-dose curve starts at the surface, half a voxel above
    its first sample); inf when C never takes the value m."""
    best = math.inf
    last = len(pos) - 2
    for j in range(len(pos) - 1):
        c0, c1 = float(calc[j]), float(calc[j + 1])
        y0, y1 = float(pos[j]), float(pos[j + 1])
        if c0 == c1:                       # a flat segment at the value m: nearest point of it
            if c0 != m:
                continue
            dist = 0.0 if y0 <= x <= y1 else min(abs(x - y0), abs(x - y1))
        else:
            t = (m - c0) / (c1 - c0)
            if not ((0.0 <= t <= 1.0) or (j == 0 and t < 0.0) or (j == last and t > 1.0)):
                continue
            dist = abs(x - (y0 + t * (y1 - y0)))
        best = min(best, dist)
    return best


def compare(pos, calc, meas, lo: float, hi: float, dmax_m: float, use_abs: bool = False):
    """(RMS, Max, mean DTA, max DTA, points, points without a crossing) over
    the points with lo <= pos < hi (lo <= |pos| < hi with use_abs), as the
    GPU call returns them; the DTA search runs over the whole curve."""
    pos = np.asarray(pos, np.float64)
    calc = np.asarray(calc, np.float64)
    meas = np.asarray(meas, np.float64)
    key = np.abs(pos) if use_abs else pos
    sel = (key >= lo) & (key < hi)
    if not sel.any():
        return 0.0, 0.0, 0.0, 0.0, 0, 0
    rms, mx = rms_max(calc[sel], meas[sel], dmax_m)
    d = np.array([dta_point(x, m, pos, calc) for x, m in zip(pos[sel], meas[sel])])
    fin = np.isfinite(d)
    return (rms, mx, float(d[fin].mean()) if fin.any() else 0.0, float(d[fin].max()) if fin.any() else 0.0,
            int(sel.sum()), int((~fin).sum()))


def depth_regions(depth, pdd_meas):
    """(build-up limits, beyond-build-up limits) in depth: the build-up ends
    at the first depth where the measured dose reaches 99 % of its maximum
    (the maximum of a noisy, flat-topped curve can sit centimetres deeper)."""
    m = np.asarray(pdd_meas, np.float64)
    d_max = float(np.asarray(depth)[int(np.argmax(m >= 0.99 * m.max()))])
    return (-math.inf, d_max), (d_max, math.inf)


def profile_regions(field_cm: float, depth_cm: float, ssd: float = 100.0, sad: float = 100.0):
    """Inner beam, penumbra and outer beam limits in |x| for a square field of
    side field_cm defined at the isocentre, at the given depth: the geometric
    half-width w = field/2 * (ssd + depth) / sad; inner |x| < 0.8 w, penumbra
    0.8-1.2 w, outer > 1.2 w."""
    w = 0.5 * field_cm * (ssd + depth_cm) / sad
    return (0.0, 0.8 * w), (0.8 * w, 1.2 * w), (1.2 * w, math.inf)
