"""Failure paths of the device code, forced from the host without faulting a GPU.

Each bounded resource is made to run out on purpose -- a tiny secondary-electron
queue, a per-particle step cap of a few steps, a table-staging wait of zero
polls, a convolution pipeline wait of zero nanoseconds -- and the test checks
what the library promises for it: the event is counted and reported, energy
stays balanced, the results are otherwise unchanged, and the library stays
usable afterwards. Every wait in these paths is bounded and every kernel
drains its own copies and tensor-core operations before it exits.
"""
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


def _case(n_hist=20_000):
    wl = W.workload_full_10x10(n_hist)
    wl.phantom = W.water_phantom(32, 32, 32, 0.5)
    return wl


def _run(L, wl, n_batches=4, **kw):
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    rc = L.lsm_run(g, ph, t, wl.seed, L.RunOpts(electron_mode=1, n_batches=n_batches, **kw))
    s1, s2, nb = L.lsm_tally_read(t)
    led, st = L.lsm_tally_ledger(t)
    return rc, s1, s2, led, st


def _balanced(led, rel=1e-6):
    return abs(led["source"] - (led["rejected"] + led["escaped"] + led["deposited"])) <= rel * led["source"]


def test_full_electron_queue_is_counted_reported_and_balanced(L):
    """A 64-slot secondary-electron queue overflows: lsm_run returns
    LSM_ERR_OVERFLOW, the excess electrons (source electrons included) are
    counted in stats[9] and deposited where they were created, the energy
    balance holds, and the photon transport is the unconstrained run's."""
    wl = _case()
    rc0, s10, _, led0, st0 = _run(L, wl)
    rc, s1, _, led, st = _run(L, wl, e_queue_cap=64)
    assert rc0 == L.LSM_OK and st0["overflows"] == 0
    assert rc == L.LSM_ERR_OVERFLOW and st["overflows"] > 0
    assert _balanced(led) and _balanced(led0)
    for k in ("histories", "photons", "electrons", "rejected", "missed", "flights", "real"):
        assert st[k] == st0[k], k
    # the electrons that fit were transported: fewer steps than unconstrained
    assert 0 < st["esteps"] < st0["esteps"]
    assert led["source"] == pytest.approx(led0["source"], rel=1e-12)
    # no-sync runs leave the overflow in the statistics instead of the status
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    assert L.lsm_run(g, ph, t, wl.seed, L.RunOpts(n_batches=4, e_queue_cap=64, no_sync=True)) == L.LSM_OK
    assert L.lsm_tally_ledger(t)[1]["overflows"] == st["overflows"]
    # the same tally runs normally afterwards
    L.lsm_tally_reset(t)
    assert L.lsm_run(g, ph, t, wl.seed, L.RunOpts(n_batches=4)) == L.LSM_OK
    assert L.lsm_tally_ledger(t)[1]["overflows"] == 0


@pytest.mark.parametrize("max_steps", [1, 3])
def test_step_cap_matches_the_oracle_and_balances(L, max_steps):
    """With a per-particle cap of a few steps, particles that reach it deposit
    their energy where they stand and are counted (stats[8]); the capped dose
    and the counts of capped particles match the oracle's capped run."""
    wl = _case(40_000)
    rc, s1, s2, led, st = _run(L, wl, n_batches=8, max_steps=max_steps)
    assert rc == L.LSM_OK
    assert st["cap_hits"] > 0 and _balanced(led)
    o = O.Plan(wl.model, wl.beams, wl.n_hist)
    r = O.run(o, wl.phantom, wl.seed, n_batches=8, electron_mode=1, max_steps=max_steps)
    assert r["max_balance"] < 1e-12
    assert st["cap_hits"] == pytest.approx(r["cap_hits"], rel=0.02)
    for k in ("flights", "real", "esteps"):
        assert st[k] == pytest.approx(r["stats"][k], rel=0.02), k
    dg, sg = O.dose_and_sigma(s1, s2, 8)
    do, so = O.dose_and_sigma(r["s1"].ravel(), r["s2"].ravel(), 8)
    sel = do > 0.1 * do.max()
    z = (dg - do)[sel] / np.sqrt(sg[sel] ** 2 + so[sel] ** 2 + 1e-300)
    assert np.mean(np.abs(z) < 3) >= 0.99
    assert abs(dg[sel].mean() / do[sel].mean() - 1) < 0.005


def test_table_staging_fallback_gives_the_same_run(L):
    """With zero polls every transport CTA gives up waiting for its tables in
    shared memory, counts a fallback and reads them from global memory: the
    same values, so the integer counters are identical and the dose equal up
    to the order of the FP32 tally additions."""
    wl = _case()
    L.lsm_run_fallbacks(reset=True)
    rc0, s10, _, led0, st0 = _run(L, wl)
    assert L.lsm_run_fallbacks(reset=True) == 0
    try:
        L.lsm_set_wait_limits(stage_polls=0)
        rc, s1, _, led, st = _run(L, wl)
        n_fb = L.lsm_run_fallbacks(reset=True)
    finally:
        L.lsm_set_wait_limits(stage_polls=1 << 22)
    assert rc == rc0 == L.LSM_OK
    assert n_fb > 0
    for k in ("histories", "photons", "electrons", "rejected", "missed", "flights", "real", "esteps",
              "cap_hits", "overflows"):
        assert st[k] == st0[k], k
    np.testing.assert_allclose(s1, s10, rtol=1e-4, atol=1e-6 * s10.max())
    assert led["deposited"] == pytest.approx(led0["deposited"], rel=1e-6)
    # staging works again once the limit is restored
    _run(L, wl)
    assert L.lsm_run_fallbacks(reset=True) == 0


def test_conv_wait_timeout_is_reported_and_recovers(L):
    """A zero-nanosecond pipeline wait makes the convolution kernels give up:
    they drain their own copies and MMAs, release tensor memory, and the
    forward returns LSM_ERR_TIMEOUT. With the default limit restored the same
    network gives the result it gave before, bit for bit."""
    from paper_1503_01725_b300 import denoiser as DZ
    rng = np.random.default_rng(5)
    u = L.lsm_unet_create(DZ.init_params(seed=3, head_scale=0.5))
    n = 32
    dose = rng.random((n, n, n), dtype=np.float32)
    rho = np.ones((n, n, n), dtype=np.float32)
    ref = L.lsm_unet_forward(u, dose, rho)
    L.lsm_timing_enable(True)          # direct launches (no replayed graph): the new limit applies
    try:
        L.lsm_set_wait_limits(conv_wait_ns=0)
        with pytest.raises(L.LSMError) as e:
            L.lsm_unet_forward(u, dose, rho)
        assert e.value.status == L.LSM_ERR_TIMEOUT
    finally:
        L.lsm_set_wait_limits(conv_wait_ns=2_000_000_000)
        L.lsm_timing_enable(False)
    again = L.lsm_unet_forward(u, dose, rho)
    assert np.array_equal(again, ref)


def test_async_phantom_equals_checked_one_and_reports_bad_input_later(L):
    """lsm_phantom_create_async leaves the input check to the device: a valid
    phantom gives the dose of the checked creation (same seed and histories);
    an invalid one (a density above 25 g/cm^3) is created, transports nothing,
    and lsm_dose into host memory and lsm_phantom_check report LSM_ERR_ARG."""
    wl = _case(20_000)
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    scale = g.denom / wl.n_hist
    doses = []
    for async_ in (False, True):
        ph = L.lsm_phantom_create(wl.phantom, async_=async_)
        t = L.lsm_tally_create(ph)
        assert L.lsm_run(g, ph, t, wl.seed, L.RunOpts(electron_mode=1, n_batches=4)) == L.LSM_OK
        doses.append(L.lsm_dose(t, ph, scale)[0])
        L.lsm_phantom_check(ph)
    np.testing.assert_allclose(doses[1], doses[0], rtol=1e-5, atol=1e-9 * doses[0].max())
    bad = W.Phantom(**{**wl.phantom.__dict__, "rho": wl.phantom.rho.copy()})
    bad.rho.flat[bad.rho.size // 2] = 30.0
    with pytest.raises(L.LSMError):
        L.lsm_phantom_create(bad)
    ph = L.lsm_phantom_create(bad, async_=True)
    t = L.lsm_tally_create(ph)
    rc = L.lsm_run(g, ph, t, wl.seed, L.RunOpts(electron_mode=1, n_batches=2, no_sync=True, max_steps=50))
    assert rc == L.LSM_OK
    with pytest.raises(L.LSMError) as e:
        L.lsm_dose(t, ph, scale)
    assert e.value.status == L.LSM_ERR_ARG
    with pytest.raises(L.LSMError):
        L.lsm_phantom_check(ph)
    s1, _, _ = L.lsm_tally_read(t)
    assert not np.any(s1)
    # the library stays usable
    ph2 = L.lsm_phantom_create(wl.phantom, async_=True)
    t2 = L.lsm_tally_create(ph2)
    assert L.lsm_run(g, ph2, t2, wl.seed, L.RunOpts(electron_mode=1, n_batches=2)) == L.LSM_OK
    L.lsm_phantom_check(ph2)
