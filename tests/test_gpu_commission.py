"""Commissioning validation loop (Sec. 2.2 and 3.2) through the C ABI.

Bars: the curve comparison (Eq. 10-11, distance to agreement) equals the
oracle's to FP64 rounding with identical counts, from host and device arrays;
the whole loop (PSR doses of two fields, NNLS, doses of five fields) brings the
commissioned model closer to the synthetic measurements than the
uncommissioned one in the depth-dose and inner-profile RMS of every field."""
import math

import numpy as np
import pytest

from oracle import commission_eval as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    return lsm


def _curves(seed):
    rng = np.random.default_rng(seed)
    z = (np.arange(60) + 0.5) * 0.5
    pdd = (1 - np.exp(-1.8 * z)) * np.exp(-0.045 * z)
    x = np.linspace(-20, 20, 81)
    prof = 1.0 / (1.0 + np.exp((np.abs(x) - 8.0) / 0.4)) + 0.02
    noisy = lambda a, s: (a * (1 + s * rng.standard_normal(a.shape))).astype(np.float32)
    return [(z.astype(np.float32), noisy(pdd, 0.01), noisy(pdd, 0.01)),
            (x.astype(np.float32), noisy(prof, 0.02), noisy(np.roll(prof, 1), 0.01))]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_curve_compare_matches_oracle(L, seed):
    import torch
    (z, pc, pm), (x, xc, xm) = _curves(seed)
    cases = [(z, pc, pm, -math.inf, 1.5, False), (z, pc, pm, 1.5, math.inf, False), (z, pc, pm, 0.0, 100.0, False),
             (x, xc, xm, 0.0, 6.4, True), (x, xc, xm, 6.4, 9.6, True), (x, xc, xm, 9.6, math.inf, True),
             (x, xc, xm, -3.0, 3.0, False)]
    for pos, c, m, lo, hi, ab in cases:
        dmax = float(m.max())
        want = E.compare(pos, c, m, lo, hi, dmax, use_abs=ab)
        for dev in (False, True):
            args = [torch.tensor(a, device="cuda") for a in (pos, c, m)] if dev else [pos, c, m]
            got = L.lsm_curve_compare(*args, lo=lo, hi=hi, dmax_m=dmax, use_abs=ab)
            assert got["points"] == want[4] and got["no_crossing"] == want[5]
            for k, v in zip(("rms", "max", "dta_mean", "dta_max"), want[:4]):
                assert got[k] == pytest.approx(v, rel=1e-9, abs=1e-12), (k, lo, hi, ab)


def test_curve_compare_errors(L):
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_curve_compare(np.zeros(1), np.zeros(1), np.zeros(1), dmax_m=1.0)
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_curve_compare(np.arange(4.0), np.ones(4), np.ones(4), dmax_m=0.0)


def test_validation_loop_improves_on_the_reference_model(L):
    from paper_1503_01725_b300 import commission as CM
    rep = CM.run(n_large=2e9, hist_hi=4_000_000)
    assert rep["nnls"]["status"] in (L.LSM_OK, L.LSM_ERR_NOT_CONVERGED)
    assert rep["factor_rel_err"] < 0.5
    for f, v in rep["fields"].items():
        c, r = v["commissioned"], v["reference"]
        assert c["pdd"]["rms"] < r["pdd"]["rms"], f
        assert c["inline@10"]["inner_rms"] < r["inline@10"]["inner_rms"], f
        assert c["crossline@10"]["inner_rms"] < 1.2 * r["crossline@10"]["inner_rms"], f
    s = CM.summary(rep)
    assert s["commissioned"]["pdd_rms_pct"][1] < s["reference"]["pdd_rms_pct"][1]
