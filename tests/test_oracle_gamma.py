"""Pins of the gamma evaluation (oracle/gamma.py) against closed forms."""
import numpy as np

from oracle import gamma as G


def _field(shape=(12, 12, 40)):
    z, y, x = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")
    return z, y, x


def test_identical_and_small_scaling_pass():
    rng = np.random.default_rng(0)
    d = rng.random((10, 11, 12)) + 0.5
    assert G.gamma_pass_rate(d, d, (2.5, 2.5, 2.5))[0] == 1.0
    # global 2 % criterion: a 1 % scaling passes everywhere
    assert G.gamma_pass_rate(1.01 * d, d, (2.5, 2.5, 2.5))[0] == 1.0


def test_flat_region_fails_beyond_dose_criterion():
    d = np.ones((8, 8, 8))
    assert G.gamma_pass_rate(1.03 * d, d, (2.5, 2.5, 2.5))[0] == 0.0
    assert G.gamma_pass_rate(1.019 * d, d, (2.5, 2.5, 2.5))[0] == 1.0


def test_shifted_linear_ramp_matches_closed_form():
    """D = g x (x in mm); evaluating D(x - s): on a linear ramp the minimum over
    points is gamma = |s| g / sqrt(crit^2 + g^2 DTA^2) (continuous search)."""
    _, _, x = _field()
    vox = 1.0
    g = 0.05                                   # dose per mm, Dmax = 0.05 * 39 = 1.95
    ref = 0.5 + g * x * vox
    crit = 0.02 * ref.max()
    dta = 2.0
    for s_mm, expect_pass in ((1.0, True), (3.0, False)):
        ev = 0.5 + g * (x * vox - s_mm)
        gam = abs(s_mm) * g / np.sqrt(crit ** 2 + g ** 2 * dta ** 2)
        assert (gam <= 1.0) == expect_pass
        rate, n = G.gamma_pass_rate(ev, ref, (vox, vox, vox), threshold=0.0, step_mm=0.25)
        inner = rate                               # edge voxels see the clamped boundary
        assert (inner > 0.9) == expect_pass, (s_mm, rate)


def test_dta_rescues_a_shifted_step_only_within_reach():
    _, _, x = _field((6, 6, 40))
    ref = np.where(x >= 20, 1.0, 0.2)
    ev = np.where(x >= 21, 1.0, 0.2)           # edge moved by one 1 mm voxel
    r_ok, _ = G.gamma_pass_rate(ev, ref, (1.0, 1.0, 1.0), dta_mm=2.0, threshold=0.0)
    r_bad, _ = G.gamma_pass_rate(ev, ref, (1.0, 1.0, 1.0), dta_mm=0.5, threshold=0.0)
    assert r_ok == 1.0 and r_bad < 1.0


def test_rms_relative_error_subtracts_reference_noise():
    rng = np.random.default_rng(1)
    truth = np.full(100000, 2.0)
    ref = truth * (1 + 0.01 * rng.standard_normal(truth.size))
    est = truth * (1 + 0.03 * rng.standard_normal(truth.size))
    e = G.rms_relative_error(est, ref, sigma_ref=0.01 * ref)
    assert abs(e - 0.03) < 0.002
