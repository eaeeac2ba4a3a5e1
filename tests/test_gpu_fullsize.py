"""Parity at the benchmark's full sizes and launch configuration.

The oracle cannot redo 1e7-1e8 histories in test time, so these tests use
what it can compute one by one (sampled particles of scattered history ids),
subsets it can run exactly (the first batches of the same plan), and
properties that hold at any size (energy balance, bit-exact plans, two GPU
estimators of the same basis matrix).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1503_01725_b300 import workloads as W

pytestmark = pytest.mark.gpu

N_FULL = 10_000_000
B_FULL = 16


@pytest.fixture(scope="module")
def L():
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    return lsm


@pytest.fixture(scope="module")
def full_run(L):
    """The benchmark's workload and launch configuration: 1e7 histories as 16
    batches of a 625k-history plan, default iteration size."""
    wl = W.workload_full_10x10(N_FULL)
    n_plan = N_FULL // B_FULL
    g = L.lsm_build_psl(wl.model, wl.beams, n_plan)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    rc = L.lsm_run(g, ph, t, wl.seed, L.RunOpts(electron_mode=1, n_batches=B_FULL))
    s1, s2, nb = L.lsm_tally_read(t)
    led, st = L.lsm_tally_ledger(t)
    return wl, n_plan, g, (s1, s2, nb, led, st, rc)


def test_full_plan_bit_exact(L, full_run):
    wl, n_plan, g, _ = full_run
    o = O.Plan(wl.model, wl.beams, n_plan)
    assert np.array_equal(L.lsm_psl_copy(g, 3), o.count)
    assert np.array_equal(L.lsm_psl_copy(g, 4), o.ent_start)


def test_full_sampling_on_scattered_histories(L, full_run):
    import torch
    wl, n_plan, g, _ = full_run
    o = O.Plan(wl.model, wl.beams, n_plan)
    for g0 in (0, 3_141_592, N_FULL - 20_000):
        out = L.lsm_sample(g, wl.seed, g0, 20_000, W.SSD)
        torch.cuda.synchronize()
        gs = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
        os_ = O.sample(o, wl.seed, g0, 20_000, W.SSD)
        assert np.array_equal(gs["info"][:, 3], os_["entry"])
        assert np.array_equal(gs["info"][:, 1], os_["ring"])
        assert np.array_equal(gs["info"][:, 2], os_["comp"])
        assert np.array_equal(gs["psr"].astype(np.int64) & 0xFFFF, os_["psr"])
        far = os_["edge"] > 1e-4
        assert np.array_equal(gs["status"][far], os_["status"][far])
        ok = far & (os_["status"] == 0)
        for k in ("u", "v", "w"):
            np.testing.assert_allclose(gs[k][ok], os_[k][ok], rtol=1e-5, atol=2e-6, err_msg=k)
        np.testing.assert_allclose(gs["E"][ok], os_["E"][ok], rtol=1e-6, err_msg="E")
        # surface positions follow an 80 cm straight flight: they inherit the
        # direction tolerance times the flight length
        for k in ("x", "y"):
            np.testing.assert_allclose(gs[k][ok], os_[k][ok], rtol=1e-5, atol=2e-6 * (W.SSD - W.Z_PHSP),
                                       err_msg=k)


def test_full_sampling_geometry_over_every_history(L, full_run):
    """Every one of the 1e7 sampled histories of the benchmark plan, on the
    GPU: the straight line through the particle's surface position and
    direction crosses the phase-space plane inside its plan entry's PSL
    square; accepted particles (also those that miss the phantom) pass both
    jaw openings (given at the isocentre, scaled to each plane); rejected ones
    do not pass both. Tolerance 1e-3 cm (FP32 positions after an 80 cm flight)."""
    import torch
    wl, n_plan, g, _ = full_run
    m, b = wl.model, wl.beams
    ent = torch.tensor(L.lsm_psl_copy(g, 5), device="cuda", dtype=torch.int64)   # beam stype ebin ix iy ring
    x1, x2, y1, y2 = (float(v) for v in b.jaws[0])
    tol, pitch, n_r = 1e-3, float(m.dr), int(m.n_r)
    chunk = 2_500_000
    n_acc = n_rej = 0
    for g0 in range(0, N_FULL, chunk):
        out = L.lsm_sample(g, wl.seed, g0, chunk, W.SSD)
        x, y, u, v, w = (out[k].double() for k in ("x", "y", "u", "v", "w"))
        e = ent[out["info"][:, 3].long()]

        def at(z):
            t = (z - W.SSD) / w
            return x + t * u, y + t * v

        xp, yp = at(W.Z_PHSP)
        lox, loy = (e[:, 3] - n_r).double() * pitch, (e[:, 4] - n_r).double() * pitch
        assert bool(((xp >= lox - tol) & (xp <= lox + pitch + tol)).all())
        assert bool(((yp >= loy - tol) & (yp <= loy + pitch + tol)).all())
        xj, _ = at(b.z_jaw_x)
        _, yj = at(b.z_jaw_y)
        sx, sy = b.z_jaw_x / b.sad, b.z_jaw_y / b.sad
        inside = (xj >= x1 * sx - tol) & (xj <= x2 * sx + tol) & (yj >= y1 * sy - tol) & (yj <= y2 * sy + tol)
        deep = (xj > x1 * sx + tol) & (xj < x2 * sx - tol) & (yj > y1 * sy + tol) & (yj < y2 * sy - tol)
        acc = out["status"] != 1
        assert bool(inside[acc].all())
        assert not bool(deep[~acc].any())
        n_acc += int(acc.sum())
        n_rej += int((~acc).sum())
    assert n_acc + n_rej == N_FULL and n_rej > 0 and n_acc > 0


def test_full_energy_ledger(full_run):
    _, _, _, (s1, s2, nb, led, st, rc) = full_run
    assert rc == 0 and nb == B_FULL
    assert st["histories"] == N_FULL
    assert st["overflows"] == 0 and st["cap_hits"] == 0
    assert led["source"] == pytest.approx(led["rejected"] + led["escaped"] + led["deposited"], rel=1e-6)
    assert s1.sum() == pytest.approx(led["deposited"], rel=1e-5)


def test_full_dose_against_oracle_batches(full_run):
    """The oracle runs batches 0-1 of the same plan (histories 0 .. 1.25e6);
    per-batch dose from the full GPU run must agree with them."""
    wl, n_plan, _, (s1, s2, nb, led, st, rc) = full_run
    o = O.Plan(wl.model, wl.beams, n_plan)
    r = O.run(o, wl.phantom, wl.seed, n_batches=2, electron_mode=1)
    dg, sg = O.dose_and_sigma(s1, s2, nb)
    do, so = O.dose_and_sigma(r["s1"].ravel(), r["s2"].ravel(), 2)
    dg, sg = dg / nb, sg / nb
    do, so = do / 2, so / 2
    # two oracle batches give a poor batch sigma: use the GPU's per-batch spread for both.
    # Voxels are selected on a smoothed GPU dose, not on the 16x noisier oracle
    # dose (selecting on noisy values biases the selected mean upwards).
    from scipy import ndimage
    sm = ndimage.uniform_filter(dg.reshape(wl.phantom.rho.shape), size=3).ravel()
    sel = sm > 0.1 * sm.max()
    sb = np.sqrt(np.clip(s2 / nb - (s1 / nb) ** 2, 0, None))          # per-batch sd of the GPU run
    z = (dg - do)[sel] / np.sqrt(sg[sel] ** 2 + (sb[sel] / np.sqrt(2)) ** 2 + 1e-300)
    assert np.mean(np.abs(z) < 3) >= 0.99
    assert abs(dg[sel].mean() / do[sel].mean() - 1) < 0.005


def test_precision_case_voxel_parity(L):
    """The precision case: 256x256x160 heterogeneous phantom at 0.25 cm, 1e8
    histories in the benchmark's launch configuration (one run of 16 batches:
    FP32 transport, FP32 partial slices folded into FP64 sums). Energy balances
    at full size, and the dose matches an independent FP64 oracle run of 1.2e7
    histories (32 batches spread over the host's cores) voxel by voxel: |z| < 3
    on at least 99 % of the voxels above 10 % of the maximum and the mean dose
    within 0.5 %."""
    from oracle import pool
    wl = W.workload_hetero(100_000_000)
    n_plan = wl.n_hist // 16
    g = L.lsm_build_psl(wl.model, wl.beams, n_plan)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    rc = L.lsm_run(g, ph, t, wl.seed, L.RunOpts(electron_mode=1, n_batches=16))
    s1, s2, nb = L.lsm_tally_read(t)
    led, st = L.lsm_tally_ledger(t)
    assert rc == 0 and st["histories"] == wl.n_hist and st["overflows"] == 0
    assert led["source"] == pytest.approx(led["rejected"] + led["escaped"] + led["deposited"], rel=1e-6)
    P = wl.phantom
    c = P.nx // 2
    box = ((0, P.nz), (c - 32, c + 32), (c - 32, c + 32))       # +-8 cm around the 10x10 field
    # 1.2e7 oracle histories in 32 batches: voxels near 10 % of the maximum
    # then collect enough deposits per batch for their batch sigma to hold
    n_o, plan_o, b_o = 12_000_000, 375_000, 32
    r = pool.run_batches("workload_hetero", n_o, plan_o, b_o, seed=17, box=box)
    assert r["max_balance"] < 1e-12 and int(r["stats"][0]) == n_o
    # energy per history in each voxel and its batch sigma, both sides
    dg_full, sg_full = O.dose_and_sigma(s1, s2, nb)
    dg_full = dg_full.reshape(P.nz, P.ny, P.nx) / wl.n_hist
    sg_full = sg_full.reshape(P.nz, P.ny, P.nx) / wl.n_hist
    do, so = O.dose_and_sigma(r["s1"], r["s2"], b_o)
    do, so = do / n_o, so / n_o
    (z0, z1), (y0, y1), (x0, x1) = box
    dg, sg = dg_full[z0:z1, y0:y1, x0:x1], sg_full[z0:z1, y0:y1, x0:x1]
    # the box holds every voxel above 10 % of the maximum
    outside = dg_full.copy()
    outside[z0:z1, y0:y1, x0:x1] = 0
    assert outside.max() < 0.1 * dg_full.max()
    # voxels chosen on an independent GPU run (another seed): choosing them on
    # either compared estimate favours voxels where it fluctuated high and
    # biases the mean ratio (by a few percent when chosen on the oracle)
    L.lsm_tally_reset(t)
    L.lsm_run(g, ph, t, wl.seed + 1000, L.RunOpts(electron_mode=1, n_batches=16))
    ref = L.lsm_tally_read(t)[0].reshape(P.nz, P.ny, P.nx)[z0:z1, y0:y1, x0:x1]
    sel = ref > 0.1 * ref.max()
    assert sel.sum() > 50_000
    z = (dg - do)[sel] / np.sqrt(sg[sel] ** 2 + so[sel] ** 2 + 1e-300)
    frac = float(np.mean(np.abs(z) < 3))
    mean_rel = float(dg[sel].sum() / do[sel].sum() - 1)
    hi = (dg > 0.5 * dg.max())[sel]
    assert frac >= 0.99, (frac, float(np.mean(np.abs(z[hi]) < 3)), float(np.mean(np.abs(z[~hi]) < 3)), mean_rel)
    assert abs(mean_rel) < 0.005, mean_rel


def test_batched_basis_equals_single_run_decomposition(L):
    """Two estimators of the commissioning basis matrix: per-PSR batched runs
    (lsm_build_psl with per-PSR counts) and one whole-source run tallied by the
    PSR index each particle carries (Sec. 2.2.2). Both estimate the dose per
    source particle of every PSR at the measurement points."""
    wl = W.workload_commissioning(hist_lo=2000, hist_hi=100_000)
    m = wl.model
    ph = W.water_phantom(64, 64, 128, 0.25)
    idx, n_rows = W.commissioning_index(ph)
    phh = L.lsm_phantom_create(ph)
    # batched per-PSR runs
    gk = L.lsm_build_psl(m, wl.beams, per_psr_hist=wl.extra["n_k"])
    tk = L.lsm_tally_create(phh, mode=1, idx3d=idx, n_rows=n_rows, n_psr=m.n_psr, n_beams=wl.beams.n_beams)
    L.lsm_run(gk, phh, tk, 5, L.RunOpts(n_batches=8))
    Ak = L.lsm_basis_matrix(tk, gk, phh)
    s1k, s2k, nbk = L.lsm_tally_read(tk)
    # one whole-source run, PSR-indexed tally; dose per source particle = S1 / (B N) * D / mass
    N = 4_000_000
    gw = L.lsm_build_psl(m, wl.beams, N)
    tw = L.lsm_tally_create(phh, mode=1, idx3d=idx, n_rows=n_rows, n_psr=m.n_psr, n_beams=wl.beams.n_beams)
    L.lsm_run(gw, phh, tw, 6, L.RunOpts(n_batches=8))
    s1w, s2w, nbw = L.lsm_tally_read(tw)
    mass = np.zeros(n_rows)
    flat = idx.ravel()
    mass[flat[flat > 0] - 1] = ph.rho.ravel()[flat > 0] * ph.dx * ph.dy * ph.dz
    mass_r = np.tile(mass, wl.beams.n_beams)[:, None]
    Aw = s1w.reshape(Ak.shape) / (nbw * N) * gw.denom / mass_r
    # per-cell z-scores with each estimator's batch standard deviation (8
    # batches: chi-square tails, hence the 4-sigma band), over cells carrying signal
    def sd(s1_, s2_, nb_, scale):
        v = np.clip(s2_ - s1_ * s1_ / nb_, 0, None) / (nb_ - 1)
        return np.sqrt(nb_ * v).reshape(Ak.shape) * scale
    scale_k = np.divide(Ak, s1k.reshape(Ak.shape), out=np.zeros_like(Ak), where=s1k.reshape(Ak.shape) > 0)
    sk = sd(s1k, s2k, nbk, scale_k)
    sw = sd(s1w, s2w, nbw, 1.0 / (nbw * N) * gw.denom / mass_r)
    # cells are selected on the mean of the two estimates, so that neither
    # estimate's own fluctuations decide which cells are compared
    Am = 0.5 * (Ak + Aw)
    sel = (Am > 0.1 * Am.max(axis=0, keepdims=True)) & (sk > 0) & (sw > 0)
    z = (Ak - Aw)[sel] / np.sqrt(sk[sel] ** 2 + sw[sel] ** 2)
    assert sel.sum() > 1000
    assert np.mean(np.abs(z) < 4) >= 0.99
    # unselected totals per field
    tk_ = Ak.reshape(wl.beams.n_beams, -1).sum(axis=1)
    tw_ = Aw.reshape(wl.beams.n_beams, -1).sum(axis=1)
    np.testing.assert_allclose(tk_, tw_, rtol=0.03)


def test_commissioning_system_active_set_against_the_oracle(L):
    """Eq. 8 at the commissioning size: A from the batched basis runs of 300
    PSRs x 3 fields (electron PSRs grouped per energy bin: 1518 x 210), b from
    an independent run times known weights with 0.5 % noise. The GPU's active
    set equals the oracle's Lawson-Hanson solution to 1e-9 with the same
    iteration count, and its KKT residual is below 1e-10 |A^T b|."""
    from oracle import nnls as N
    wl = W.workload_commissioning()
    m = wl.model
    ph = L.lsm_phantom_create(wl.phantom)
    idx, n_rows = W.commissioning_index(wl.phantom)
    t = L.lsm_tally_create(ph, mode=1, idx3d=idx, n_rows=n_rows, n_psr=m.n_psr, n_beams=wl.beams.n_beams)
    n_ph = 2 * m.n_e * m.n_r

    def grouped(seed):
        g = L.lsm_build_psl(m, wl.beams, per_psr_hist=wl.extra["n_k"])
        L.lsm_tally_reset(t)
        L.lsm_run(g, ph, t, seed, L.RunOpts(electron_mode=1, n_batches=4))
        A = L.lsm_basis_matrix(t, g, ph)
        Au = L.lsm_basis_matrix(t, g, ph, units=True)
        # the library's electron units equal the column sums of the per-PSR matrix
        Ah = np.concatenate([A[:, :n_ph], A[:, n_ph:].reshape(A.shape[0], m.n_e, m.n_r).sum(axis=2)], axis=1)
        np.testing.assert_allclose(Au, Ah, rtol=1e-13, atol=1e-300)
        return Au

    A, A2 = grouped(1), grouped(999)
    x_true = W.commissioning_truth(A.shape[1])
    b = A2 @ x_true * (1 + 0.005 * np.random.default_rng(3).standard_normal(A.shape[0]))
    sc = 1.0 / np.abs(b).max()
    A, b = A * sc, b * sc
    x, rep = L.lsm_commission(A, b, method=0)
    xo, it_o = N.lawson_hanson(A, b)
    assert rep["converged"] and rep["iterations"] == it_o
    np.testing.assert_allclose(x, xo, atol=1e-9 * np.abs(xo).max())
    assert rep["kkt"] < 1e-10 * np.linalg.norm(A.T @ b)
