"""Pins of the commissioning-validation metrics (Eq. 10-11, distance to
agreement, TG-53 regions) against closed forms."""
import math

import numpy as np

from oracle import commission_eval as E


def test_rms_and_max_of_a_constant_offset():
    m = np.linspace(0.2, 1.0, 50)
    rms, mx = E.rms_max(m + 0.01, m, 2.0)
    assert math.isclose(rms, 0.005, rel_tol=1e-12)
    assert math.isclose(mx, 0.005, rel_tol=1e-12)
    # Eq. 10 is the root of the mean square, Eq. 11 the largest magnitude
    d = np.array([0.0, 0.03, -0.04, 0.0])
    rms, mx = E.rms_max(d, np.zeros(4), 1.0)
    assert math.isclose(rms, math.sqrt((0.03 ** 2 + 0.04 ** 2) / 4), rel_tol=1e-12)
    assert math.isclose(mx, 0.04, rel_tol=1e-12)


def test_dta_of_a_shifted_ramp_is_the_shift():
    x = np.linspace(0.0, 10.0, 101)
    meas = 0.3 * x + 1.0
    calc = 0.3 * (x - 0.37) + 1.0            # the same line moved by +0.37
    r = E.compare(x, calc, meas, 1.0, 9.0, 4.0)
    assert math.isclose(r[2], 0.37, rel_tol=1e-9) and math.isclose(r[3], 0.37, rel_tol=1e-9)
    assert r[5] == 0
    # near the end the crossing lies on the continuation of the last segment
    r = E.compare(x, calc, meas, 9.45, 11.0, 4.0)
    assert r[4] == 6 and r[5] == 0
    assert math.isclose(r[2], 0.37, rel_tol=1e-9)
    # a curve that never takes a value: a flat calculated curve above it
    r = E.compare(x, np.full_like(x, 9.0), meas, 0.0, 11.0, 4.0)
    assert r[5] == len(x)


def test_dta_of_a_shifted_penumbra():
    x = np.linspace(-10, 10, 401)
    edge = lambda x, w: 1.0 / (1.0 + np.exp((np.abs(x) - w) / 0.3))
    meas, calc = edge(x, 5.0), edge(x, 5.2)
    r = E.compare(x, calc, meas, 4.5, 5.5, 1.0, use_abs=True)
    assert abs(r[2] - 0.2) < 2e-3 and abs(r[3] - 0.2) < 5e-3
    assert r[4] == 2 * np.sum((np.abs(x) >= 4.5) & (np.abs(x) < 5.5)) // 2


def test_dta_special_cases():
    pos = np.array([0.0, 1.0, 2.0, 3.0])
    calc = np.array([1.0, 2.0, 2.0, 3.0])
    assert E.dta_point(1.0, 2.0, pos, calc) == 0.0          # equal at the point
    # continued below the first point along the first segment: C(-0.5) = 0.5
    assert math.isclose(E.dta_point(0.0, 0.5, pos, calc), 0.5)
    # but not along an interior segment: the value 2.5 is met only inside [2, 3]
    assert math.isclose(E.dta_point(1.0, 2.5, pos, calc), 1.5)
    assert E.dta_point(1.5, 2.0, pos, calc) == 0.0          # inside a flat segment at the value
    assert E.dta_point(0.0, 2.0, pos, calc) == 1.0          # nearest point of the flat segment
    assert math.isclose(E.dta_point(0.0, 5.0, pos, calc), 5.0)   # on the last segment's continuation
    flat = np.array([2.0, 2.0, 2.0, 2.0])
    assert math.isinf(E.dta_point(0.0, 5.0, pos, flat))     # never reached
    assert math.isclose(E.dta_point(3.0, 1.5, pos, calc), 2.5)


def test_regions():
    depth = np.arange(0.25, 30, 0.5)
    pdd = np.exp(-0.05 * depth) * (1 - np.exp(-2.0 * depth))
    bu, after = E.depth_regions(depth, pdd)
    assert bu[1] == depth[np.argmax(pdd >= 0.99 * pdd.max())] and after[0] == bu[1]
    assert bu[1] <= depth[np.argmax(pdd)]
    inner, pen, outer = E.profile_regions(10.0, 10.0)
    assert math.isclose(inner[1], 4.4) and math.isclose(pen[1], 6.6) and math.isinf(outer[1])
