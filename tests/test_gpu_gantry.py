"""Multi-beam plans with gantry rotation through the C ABI, against the oracle.

Bars: the sampled particles are the same histories on both sides, so the
counts of photons and electrons entering the phantom agree to within the
histories whose entry decision lies at a box edge (1e-3 relative); doses pass
the z-test of the parity suite (|z| < 3 on >= 99% of voxels above 10% of the
maximum, mean within 1%)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1503_01725_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    return lsm


def _zcheck(dg, sg, do, so, frac=0.99, thr=0.1, mean_tol=0.01):
    sel = do > thr * do.max()
    z = (dg - do)[sel] / np.sqrt(sg[sel] ** 2 + so[sel] ** 2 + 1e-300)
    assert np.mean(np.abs(z) < 3) >= frac, np.mean(np.abs(z) < 3)
    assert abs(dg[sel].mean() / do[sel].mean() - 1) < mean_tol


def _gpu_run(L, model, beams, ph, n, seed, nb, electron_mode=1):
    g = L.lsm_build_psl(model, beams, n)
    phh = L.lsm_phantom_create(ph)
    t = L.lsm_tally_create(phh)
    L.lsm_run(g, phh, t, seed, L.RunOpts(electron_mode=electron_mode, n_batches=nb))
    s1, s2, b = L.lsm_tally_read(t)
    led, st = L.lsm_tally_ledger(t)
    return s1, s2, b, led, st


@pytest.mark.parametrize("angles", [(0.0, 90.0, 225.0), (30.0, 180.0)])
def test_rotated_beams_match_oracle(L, angles):
    model = W.psr_model(6, 10, 0.25, seed=2)
    beams = W.gantry_beams(angles, 5.0)
    ph = W.pelvis_phantom(40, 24, 32, 1.0)
    n, nb = 60_000, 8
    s1, s2, b, led, st = _gpu_run(L, model, beams, ph, n, 11, nb)
    r = O.run(O.Plan(model, beams, n), ph, 11, n_batches=nb, electron_mode=1)
    for k in ("histories", "rejected"):
        assert st[k] == r["stats"][k], k
    for k in ("photons", "electrons", "missed"):
        assert abs(st[k] - r["stats"][k]) <= 1e-3 * st["histories"] + 2, k
    dg, sg = O.dose_and_sigma(s1, s2, nb)
    do, so = O.dose_and_sigma(r["s1"].ravel(), r["s2"].ravel(), nb)
    _zcheck(dg, sg, do, so)
    np.testing.assert_allclose(led["source"], r["ledger"]["source"], rtol=1e-6)
    np.testing.assert_allclose(led["deposited"], r["ledger"]["deposited"], rtol=0.02)


def test_gantry_zero_is_the_unrotated_beam(L):
    model = W.psr_model(6, 10, 0.25, seed=2)
    ph = W.water_phantom(32, 32, 32, 0.5)
    a = _gpu_run(L, model, W.beams(W.square_field(6.0)), ph, 200_000, 3, 1)
    b = _gpu_run(L, model, W.gantry_beams([0.0], 6.0), ph, 200_000, 3, 1)
    assert a[4]["rejected"] == b[4]["rejected"]
    assert abs(a[4]["photons"] - b[4]["photons"]) <= 5
    # same histories and streams; the rotated path starts 1e-4 cm inside
    assert np.abs(a[0] - b[0]).sum() / a[0].sum() < 0.02


def test_prostate_and_hn_layouts_run(L):
    for wl in (W.workload_prostate_7beam(700_000), W.workload_hn_6beam(600_000)):
        s1, s2, b, led, st = _gpu_run(L, wl.model, wl.beams, wl.phantom, wl.n_hist, wl.seed, 4)
        # energy balance: source = rejected + escaped + deposited
        tot = led["rejected"] + led["escaped"] + led["deposited"]
        assert abs(tot / led["source"] - 1) < 1e-6
        d = s1.reshape(wl.phantom.nz, wl.phantom.ny, wl.phantom.nx) / np.maximum(wl.phantom.rho, 1e-3)
        nz, ny, nx = d.shape
        c = d[nz // 2 - 2: nz // 2 + 2, ny // 2 - 2: ny // 2 + 2, nx // 2 - 2: nx // 2 + 2].mean()
        # the beams converge at the isocentre: its dose exceeds the body's mean dose
        body = wl.phantom.rho > 0.5
        assert c > 1.5 * d[body].mean(), wl.name


def test_sixteen_beams_the_maximum(L):
    # sixteen rotated beams (the limit): the plan's counts bit-exact against the
    # oracle's Eq. 3 over all beams, the run's counters as the oracle's
    model = W.psr_model(6, 10, 0.25, seed=2)
    beams = W.gantry_beams([k * 22.5 for k in range(16)], 4.0)
    ph = W.pelvis_phantom(40, 24, 32, 1.0)
    n = 32_000
    g = L.lsm_build_psl(model, beams, n)
    plan = O.Plan(model, beams, n)
    np.testing.assert_array_equal(L.lsm_psl_copy(g, 3), plan.count)
    s1, s2, b, led, st = _gpu_run(L, model, beams, ph, n, 13, 4)
    r = O.run(plan, ph, 13, n_batches=4, electron_mode=1)
    for k in ("histories", "rejected"):
        assert st[k] == r["stats"][k], k
    for k in ("photons", "electrons", "missed"):
        assert abs(st[k] - r["stats"][k]) <= 1e-3 * st["histories"] + 2, k
    np.testing.assert_allclose(led["source"], r["ledger"]["source"], rtol=1e-6)
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_build_psl(model, W.gantry_beams([k * 20.0 for k in range(17)], 4.0), n)
