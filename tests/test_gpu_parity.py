"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars:
* integer work is bit-exact: PSL inclusion, Eq. 3 counts, plan entries and
  prefixes, and per history the plan entry, sub-source, energy bin, ring,
  mixture component, PSR index, beam and particle type;
* the FP64 PSL weights, sampling areas and per-PSR scales are bit-identical
  (same IEEE operations in the same order, no FMA on either side);
* jaw rejection agrees except within 1e-4 cm of a jaw edge (the decision
  follows a chain of transcendentals evaluated in FP32 on the GPU and FP64 in
  the oracle); such histories must be fewer than 1e-3 of the total;
* sampled attributes within 1e-5 relative (positions also 1e-5 cm absolute,
  direction components 2e-6 absolute);
* dose: |z| < 3 on >= 99% of voxels above 10% of the maximum and mean dose
  within 0.5%, z = (D_gpu - D_oracle) / sqrt(s_gpu^2 + s_oracle^2).
"""
import math

import numpy as np
import pytest

from oracle import nnls as N
from oracle import oracle as O
from paper_1503_01725_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    return lsm


def _models():
    m1 = W.primary_only_model()
    m2 = W.psr_model(6, 10, 0.25, seed=2)
    m3 = W.psr_model(5, 12, 0.3, seed=31)
    return [
        (m1, W.beams(W.square_field(5.0)), 100_000),
        (m2, W.beams(W.square_field(10.0)), 1_000_003),
        (m3, W.beams(W.square_field(4.0, cx=1.5, cy=-2.0), W.square_field(20.0),
                     np.array([-7.0, 2.0, -1.0, 9.0])), 777_777),
        # 3.1e6 cells in four beams: the largest-remainder selection over a
        # million included cells, 1136 of their remainders within 2^-11 of
        # the threshold
        (W.psr_model(64, 32, 0.1, seed=7),
         W.beams(*[W.square_field(40.0, cx=0.3 * k, cy=-0.2 * k) for k in range(4)]), 10_000_019),
    ]


@pytest.mark.parametrize("case", range(4))
def test_psl_build_bit_exact(L, case):
    m, b, n = _models()[case]
    g = L.lsm_build_psl(m, b, n)
    o = O.Plan(m, b, n)
    assert g.info["n_xy"] == o.n_xy and g.info["n_ent"] == o.n_ent and g.info["plan_size"] == n
    assert g.denom == o.denom
    assert np.array_equal(L.lsm_psl_copy(g, 0), o.wpsl)          # FP64 bit-identical
    assert np.array_equal(L.lsm_psl_copy(g, 1), o.incl)
    assert np.array_equal(L.lsm_psl_copy(g, 2), o.area)
    assert np.array_equal(L.lsm_psl_copy(g, 3), o.count)
    assert np.array_equal(L.lsm_psl_copy(g, 4), o.ent_start)
    assert np.array_equal(L.lsm_psl_copy(g, 5), o.entries)


def test_per_psr_plan_bit_exact(L):
    wl = W.workload_commissioning(hist_lo=200, hist_hi=5000)
    n_k = wl.extra["n_k"]
    g = L.lsm_build_psl(wl.model, wl.beams, per_psr_hist=n_k)
    o = O.Plan(wl.model, wl.beams, per_psr_n=n_k)
    assert g.info["plan_size"] == o.n_hist and g.info["n_ent"] == o.n_ent
    assert np.array_equal(L.lsm_psl_copy(g, 3), o.count)
    assert np.array_equal(L.lsm_psl_copy(g, 4), o.ent_start)
    assert np.array_equal(L.lsm_psl_copy(g, 5), o.entries)
    assert np.array_equal(L.lsm_psl_copy(g, 6), o.ent_scale)


@pytest.mark.parametrize("graph", [False, True])
def test_two_stream_iterations_equal_one_stream(L, graph):
    """streams = 2 splits an iteration's batches into two halves on two CUDA
    streams: the same histories, so every integer counter equals the
    one-stream run and the dose agrees up to the order of the FP32 tally
    additions; with graph replay too (the capture forks and joins the second
    stream), and an odd batch count (halves of 3 and 2)."""
    wl = W.workload_full_10x10(400_000)
    wl.phantom = W.water_phantom(32, 32, 32, 0.5)
    g = L.lsm_build_psl(wl.model, wl.beams, 40_000)
    ph = L.lsm_phantom_create(wl.phantom)
    out = []
    for streams in (1, 2):
        t = L.lsm_tally_create(ph)
        o = L.RunOpts(electron_mode=1, n_batches=5, chunk=200_000, streams=streams, use_graph=graph)
        for rep in range(2 if graph else 1):          # second run replays the graph
            L.lsm_tally_reset(t)
            assert L.lsm_run(g, ph, t, 77, o) == L.LSM_OK
        s1, s2, nb = L.lsm_tally_read(t)
        out.append((s1, s2, nb, L.lsm_tally_ledger(t)[1]))
    (a1, a2, an, ast), (b1, b2, bn, bst) = out
    assert an == bn == 5 and ast == bst
    np.testing.assert_allclose(b1, a1, rtol=2e-5, atol=1e-6 * a1.max())
    np.testing.assert_allclose(b2, a2, rtol=5e-5, atol=1e-6 * a2.max())


def test_model_handle_plans_equal_the_oracle(L):
    """A plan built from a model handle equals the oracle's plan of the same
    model; the commissioned handle (lsm_model_commission with per-unit
    factors: photon PSRs, then one factor per electron energy bin) builds the
    oracle's plan of the model whose weights are W_R x_R, bit for bit."""
    m, b, n = _models()[1]
    mh = L.lsm_model_create(m)
    g = L.lsm_build_psl(mh, b, n)
    o = O.Plan(m, b, n)
    assert g.denom == o.denom and np.array_equal(L.lsm_psl_copy(g, 3), o.count)
    n_ph = 2 * m.n_e * m.n_r
    x = np.random.default_rng(8).uniform(0.7, 1.3, n_ph + m.n_e)
    x[5] = 0.0
    mc = L.lsm_model_commission(mh, x)
    wc = m.w.reshape(-1) * np.concatenate([x[:n_ph], np.repeat(x[n_ph:], m.n_r)])
    assert np.array_equal(L.lsm_model_weights(mc).ravel(), wc)
    del mh                                  # a handle's plans do not need the handle that built them
    gc = L.lsm_build_psl(mc, b, n)
    oc = O.Plan(m.with_weights(wc.reshape(m.w.shape)), b, n)
    assert gc.denom == oc.denom
    assert np.array_equal(L.lsm_psl_copy(gc, 0), oc.wpsl)
    assert np.array_equal(L.lsm_psl_copy(gc, 3), oc.count)
    assert np.array_equal(L.lsm_psl_copy(gc, 5), oc.entries)


def test_empty_sampling_area_is_an_argument_error(L):
    m = W.psr_model(3, 4, 0.25, seed=1)
    with pytest.raises(L.LSMError) as e:
        L.lsm_build_psl(m, W.beams(np.array([60.0, 70.0, 60.0, 70.0])), 1000)
    assert e.value.status == L.LSM_ERR_ARG


def _sample_both(L, m, b, n_plan, seed, g0, n):
    import torch
    g = L.lsm_build_psl(m, b, n_plan)
    o = O.Plan(m, b, n_plan)
    out = L.lsm_sample(g, seed, g0, n, W.SSD)
    torch.cuda.synchronize()
    gs = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    os_ = O.sample(o, seed, g0, n, W.SSD)
    return gs, os_


@pytest.mark.parametrize("case,seed,g0", [(0, 1, 0), (1, 7, 3_000_000), (2, 99, 2 ** 33 + 5)])
def test_sampling_parity(L, case, seed, g0):
    m, b, n_plan = _models()[case]
    n = 200_000
    gs, os_ = _sample_both(L, m, b, n_plan, seed, g0, n)
    info = gs["info"]
    assert np.array_equal(info[:, 3], os_["entry"])
    assert np.array_equal(info[:, 0] & 0xFF, os_["stype"])
    assert np.array_equal(info[:, 0] >> 8, os_["ebin"])
    assert np.array_equal(info[:, 1], os_["ring"])
    assert np.array_equal(info[:, 2], os_["comp"])
    assert np.array_equal(gs["psr"].astype(np.int64) & 0xFFFF, os_["psr"])
    assert np.array_equal(gs["beam"], os_["beam"])
    assert np.array_equal(gs["type"], os_["type"])
    assert np.array_equal(gs["hist"], g0 + np.arange(n))
    # jaw rejection: equal away from the jaw edges
    far = os_["edge"] > 1e-4
    assert np.mean(~far) < 1e-3
    assert np.array_equal(gs["status"][far], os_["status"][far])
    ok = far & (os_["status"] == 0)
    for k, atol in (("x", 1e-5), ("y", 1e-5), ("u", 2e-6), ("v", 2e-6), ("w", 2e-6), ("E", 0.0)):
        np.testing.assert_allclose(gs[k][ok], os_[k][ok], rtol=1e-5, atol=atol, err_msg=k)
    assert np.all(gs["z"] == np.float32(W.SSD))


def test_sampling_edge_cases(L):
    import torch
    m, b, n_plan = _models()[0]
    g = L.lsm_build_psl(m, b, n_plan)
    L.lsm_sample(g, 1, 0, 0, W.SSD, out=L.alloc_particles(1))   # n = 0 is a no-op
    # the plan is periodic: history g and g + plan size share the PSL
    a = L.lsm_sample(g, 5, 10, 1000, W.SSD)
    c = L.lsm_sample(g, 5, 10 + n_plan, 1000, W.SSD)
    torch.cuda.synchronize()
    assert torch.equal(a["info"][:, 3], c["info"][:, 3])
    assert not torch.equal(a["x"], c["x"])
    with pytest.raises(L.LSMError):
        L.lsm_sample(g, 1, 0, -1, W.SSD, out=L.alloc_particles(1))


def test_interaction_tables_match_closed_forms(L):
    ph = L.lsm_phantom_create(W.heterogeneous_phantom(16, 16, 16, 0.5, seed=3))
    xs, mm, kn, grid = L.lsm_phantom_tables(ph)
    E = np.exp(grid[0] + grid[1] * np.arange(1024))
    sel = (E > 0.01) & (E < 7.0)
    for m in (0, 1):
        for comp in range(3):
            want = np.array([O.mu_mass(e, m, comp) for e in E[sel]])
            np.testing.assert_allclose(xs[m, sel, comp], want, rtol=2e-6, atol=1e-30)
        want = np.array([O.scol_mass(e, m) for e in E[sel]])
        np.testing.assert_allclose(xs[m, sel, 3], want, rtol=2e-6)
    rho = ph.desc.rho
    rmax = [rho[ph.desc.mat == k].max() if (ph.desc.mat == k).any() else 0.0 for k in (0, 1)]
    want = np.maximum(rmax[0] * np.array([O.mu_mass(e, 0, 3) for e in E[sel]]),
                      rmax[1] * np.array([O.mu_mass(e, 1, 3) for e in E[sel]]))
    assert np.all(mm[sel] >= want * (1 - 1e-6))
    np.testing.assert_allclose(mm[sel], want, rtol=5e-5)


def test_inverse_kn_table_matches_exact_inversion(L):
    """GPU Compton table against the closed-form CDF inverted in FP64."""
    from scipy import optimize
    ph = L.lsm_phantom_create(W.water_phantom(8, 8, 8, 0.5))
    _, _, kn, _ = L.lsm_phantom_tables(ph)
    lnE = np.linspace(np.log(0.05), np.log(7.0), 32)
    for i in range(0, 32, 3):
        k = np.exp(lnE[i]) / 0.51099895
        emax = 1 + 2 * k
        tot = O.kn_cdf(emax, k)
        for j in range(1, 128, 7):
            u = j / 128
            eta = optimize.brentq(lambda t: O.kn_cdf(t, k) - u * tot, 1.0, emax, xtol=1e-14)
            assert kn[i, j] == pytest.approx((eta - 1) / (2 * k), rel=2e-6, abs=1e-7)
    assert np.all(kn[:, 0] == 0) and np.all(kn[:, -1] == 1)
    assert np.all(np.diff(kn, axis=1) >= 0)


def _dose_zcheck(dg, sg, do, so, frac=0.99, thr=0.1, mean_tol=0.005):
    sel = do > thr * do.max()
    z = (dg - do)[sel] / np.sqrt(sg[sel] ** 2 + so[sel] ** 2 + 1e-300)
    assert np.mean(np.abs(z) < 3) >= frac, np.mean(np.abs(z) < 3)
    assert abs(dg[sel].mean() / do[sel].mean() - 1) < mean_tol


def _run_both(L, wl, n_batches, **kw):
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    opts = L.RunOpts(electron_mode=wl.electron_mode, n_batches=n_batches, **kw)
    rc = L.lsm_run(g, ph, t, wl.seed, opts)
    assert rc == L.LSM_OK
    s1, s2, nb = L.lsm_tally_read(t)
    led, st = L.lsm_tally_ledger(t)
    o = O.Plan(wl.model, wl.beams, wl.n_hist)
    r = O.run(o, wl.phantom, wl.seed, n_batches=n_batches, electron_mode=wl.electron_mode)
    return (s1, s2, nb, led, st), r, (g, ph, t)


def test_dose_parity_primary_local_deposition(L):
    wl = W.workload_primary_5x5(100_000)
    (s1, s2, nb, led, st), r, _ = _run_both(L, wl, 8)
    assert nb == 8
    dg, sg = O.dose_and_sigma(s1, s2, nb)
    do, so = O.dose_and_sigma(r["s1"].ravel(), r["s2"].ravel(), 8)
    _dose_zcheck(dg, sg, do, so)
    # histories and the integer outcome of sampling agree exactly
    assert st["histories"] == r["stats"]["histories"]
    assert abs(st["rejected"] - r["stats"]["rejected"]) <= 1e-3 * st["histories"]
    assert led["source"] == pytest.approx(r["ledger"]["source"], rel=1e-6)
    assert led["source"] == pytest.approx(led["rejected"] + led["escaped"] + led["deposited"], rel=1e-6)
    assert s1.sum() == pytest.approx(led["deposited"], rel=1e-5)


def test_dose_parity_three_sources_csda(L):
    wl = W.workload_full_10x10(400_000)
    (s1, s2, nb, led, st), r, _ = _run_both(L, wl, 8)
    dg, sg = O.dose_and_sigma(s1, s2, nb)
    do, so = O.dose_and_sigma(r["s1"].ravel(), r["s2"].ravel(), 8)
    _dose_zcheck(dg, sg, do, so)
    assert st["overflows"] == 0 and st["cap_hits"] == 0
    assert led["source"] == pytest.approx(led["rejected"] + led["escaped"] + led["deposited"], rel=1e-6)
    # algorithmic work within statistics of the oracle's counts
    for k in ("flights", "real", "esteps", "secondaries"):
        assert st[k] == pytest.approx(r["stats"][k], rel=0.01), k
    assert st["electrons"] == r["stats"]["electrons"]


def test_dose_parity_heterogeneous(L):
    wl = W.workload_full_10x10(200_000)
    wl.phantom = W.heterogeneous_phantom(48, 48, 40, 0.4, seed=4, n_slabs=3, n_spheres=6)
    (s1, s2, nb, led, st), r, _ = _run_both(L, wl, 8)
    dg, sg = O.dose_and_sigma(s1, s2, nb)
    do, so = O.dose_and_sigma(r["s1"].ravel(), r["s2"].ravel(), 8)
    _dose_zcheck(dg, sg, do, so)


def test_ragged_chunks_and_reuse(L):
    """Plan size not a multiple of the iteration size; a second run on the same
    tally continues the batch count."""
    wl = W.workload_full_10x10(50_021)
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    L.lsm_run(g, ph, t, 3, L.RunOpts(n_batches=2, chunk=4096))
    a1, _, nb = L.lsm_tally_read(t)
    assert nb == 2
    t2 = L.lsm_tally_create(ph)
    L.lsm_run(g, ph, t2, 3, L.RunOpts(n_batches=2, chunk=50_021))
    b1, _, _ = L.lsm_tally_read(t2)
    # same histories, different iteration split: identical up to FP32 atomics order
    np.testing.assert_allclose(a1, b1, rtol=1e-4, atol=1e-6 * a1.max())
    L.lsm_run(g, ph, t2, 4, L.RunOpts(n_batches=1))
    _, _, nb2 = L.lsm_tally_read(t2)
    assert nb2 == 3


def test_graph_replay_matches_direct_runs(L):
    """A run captured in a CUDA graph and replayed with other seeds gives the
    same tallies as direct runs with those seeds (up to FP32 atomic order)."""
    wl = W.workload_full_10x10(200_000)
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    ph = L.lsm_phantom_create(wl.phantom)
    res = {}
    for graph in (False, True):
        t = L.lsm_tally_create(ph)
        for seed in (11, 12, 13):
            L.lsm_tally_reset(t)
            n0 = L.lsm_launch_count()
            L.lsm_run(g, ph, t, seed, L.RunOpts(n_batches=4, use_graph=graph))
            s1, _, nb = L.lsm_tally_read(t)
            assert nb == 4
            assert L.lsm_launch_count() > n0
            res[(graph, seed)] = s1
    for seed in (11, 12, 13):
        a, b = res[(False, seed)], res[(True, seed)]
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * a.max())
    assert not np.allclose(res[(True, 11)], res[(True, 12)])


def test_graph_cache_tells_plans_apart(L):
    """A plan built after another was freed may reuse its addresses; the graph
    of the first must not be replayed for the second."""
    wl = W.workload_full_10x10(100_000)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    g1 = L.lsm_build_psl(wl.model, wl.beams, 25_000)
    L.lsm_run(g1, ph, t, 5, L.RunOpts(n_batches=4, use_graph=True))
    del g1
    g2 = L.lsm_build_psl(wl.model, W.beams(W.square_field(5.0)), 20_000)
    L.lsm_tally_reset(t)
    L.lsm_run(g2, ph, t, 5, L.RunOpts(n_batches=4, use_graph=True))
    a, _, _ = L.lsm_tally_read(t)
    led, st = L.lsm_tally_ledger(t)
    assert st["histories"] == 4 * 20_000
    L.lsm_tally_reset(t)
    L.lsm_run(g2, ph, t, 5, L.RunOpts(n_batches=4, use_graph=False))
    b, _, _ = L.lsm_tally_read(t)
    np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * b.max())


def test_graph_replay_keeps_kernel_timers(L):
    """Timers captured into the graph are read after every replay: same kernel
    groups and launch counts as a direct run."""
    wl = W.workload_full_10x10(100_000)
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    got = {}
    L.lsm_timing_enable(True)
    try:
        for graph in (False, False, True, True):       # the first run also sizes the tally slices
            L.lsm_timing_read(reset=True)
            L.lsm_tally_reset(t)
            L.lsm_run(g, ph, t, 3, L.RunOpts(n_batches=4, use_graph=graph))
            got.setdefault(graph, []).append(L.lsm_timing_read(reset=True))
    finally:
        L.lsm_timing_enable(False)
    direct, replays = got[False][1], got[True]
    for rep in replays:
        for k in ("sample", "photon", "electron", "tally"):
            assert rep[k][1] == direct[k][1] > 0, k
            assert rep[k][0] > 0, k


def test_autotune_choice_and_cache(L, tmp_path):
    from paper_1503_01725_b300 import autotune as A
    wl = W.workload_full_10x10(400_000)
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist // 8)
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    base = L.RunOpts(n_batches=8)
    cache = str(tmp_path / "tune.json")
    cands = A.candidates(wl.n_hist // 8, 8, ctas=(0, 2))
    o, rep = A.tune(g, ph, t, base, reps=1, cands=cands, cache_path=cache)
    assert not rep["cached"] and len(rep["trials"]) == len(cands)
    assert (o.chunk, o.ctas_per_sm, o.use_graph) in cands
    o2, rep2 = A.tune(g, ph, t, base, cache_path=cache)
    assert rep2["cached"] and o2 == o
    # the tuned options change the speed, not the histories
    L.lsm_tally_reset(t)
    L.lsm_run(g, ph, t, 9, base)
    a = L.lsm_tally_read(t)[0]
    L.lsm_tally_reset(t)
    L.lsm_run(g, ph, t, 9, o)
    b = L.lsm_tally_read(t)[0]
    np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * a.max())


def test_sample_then_transport_equals_run(L):
    import torch
    wl = W.workload_full_10x10(30_000)
    g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist)
    ph = L.lsm_phantom_create(wl.phantom)
    t1 = L.lsm_tally_create(ph)
    L.lsm_run(g, ph, t1, 9, L.RunOpts(n_batches=1))
    a, _, _ = L.lsm_tally_read(t1)
    t2 = L.lsm_tally_create(ph)
    parts = L.lsm_sample(g, 9, 0, wl.n_hist, ph.desc.z0)
    L.lsm_transport(ph, parts, wl.n_hist, 9, t2, L.RunOpts(n_batches=1))
    L.lsm_tally_end_batch(t2)
    torch.cuda.synchronize()
    b, _, _ = L.lsm_tally_read(t2)
    np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * a.max())


def test_basis_tally_parity(L):
    wl = W.workload_commissioning(hist_lo=100, hist_hi=2000)
    ph = W.water_phantom(32, 32, 48, 0.5)
    idx, n_rows = W.commissioning_index(ph, depths_cm=(1.5, 10.0))
    n_k = wl.extra["n_k"]
    g = L.lsm_build_psl(wl.model, wl.beams, per_psr_hist=n_k)
    phh = L.lsm_phantom_create(ph)
    t = L.lsm_tally_create(phh, mode=1, idx3d=idx, n_rows=n_rows, n_psr=wl.model.n_psr,
                           n_beams=wl.beams.n_beams)
    L.lsm_run(g, phh, t, 3, L.RunOpts(n_batches=4))
    s1, s2, nb = L.lsm_tally_read(t)
    o = O.Plan(wl.model, wl.beams, per_psr_n=n_k)
    r = O.run(o, ph, 3, n_batches=4, tally_mode=1, idx3d=idx, n_rows=n_rows)
    dg, sg = O.dose_and_sigma(s1, s2, 4)
    do, so = O.dose_and_sigma(r["s1"].ravel(), r["s2"].ravel(), 4)
    _dose_zcheck(dg, sg, do, so, thr=0.1)
    # basis matrix normalisation: S1 / B * (in-area PSR weight / n_k) / voxel mass
    A = L.lsm_basis_matrix(t, g, phh)
    scale = np.zeros((wl.model.n_psr, wl.beams.n_beams))
    for (b_, s, e, ix, iy, k), sc in zip(o.entries, o.ent_scale):
        scale[k, b_] = sc
    mass = np.zeros(n_rows)
    flat = idx.ravel()
    mass[flat[flat > 0] - 1] = ph.rho.ravel()[flat > 0] * ph.dx * ph.dy * ph.dz
    S = s1.reshape(wl.beams.n_beams, n_rows, -1)
    want = S / 4 * scale.T[:, None, :] / mass[None, :, None]
    np.testing.assert_allclose(A.reshape(S.shape), want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("seed", range(3))
def test_commission_active_set_parity(L, seed):
    rng = np.random.default_rng(seed)
    m, n = 400, 60
    A = np.abs(rng.standard_normal((m, n))) + 0.1 * rng.standard_normal((m, n))
    xt = rng.uniform(0.8, 1.2, n)
    xt[rng.random(n) < 0.1] = 0
    b = A @ xt * (1 + 0.005 * rng.standard_normal(m))
    x, rep = L.lsm_commission(A, b, method=0)
    xo, _ = N.lawson_hanson(A, b)
    np.testing.assert_allclose(x, xo, atol=1e-9 * max(1.0, np.abs(xo).max()))
    assert rep["kkt"] < 1e-10 * np.linalg.norm(2 * A.T @ b)
    assert rep["objective"] == pytest.approx(N.objective(A, b, xo), rel=1e-9)


@pytest.mark.parametrize("seed", [0, 2, 3, 6])
def test_commission_active_set_drops_variables(L, seed):
    """Correlated columns (rank-3 structure plus noise): variables enter the
    passive set and later leave it (one or two removals for these seeds), so
    the passive-set factor has rows and columns deleted as well as added."""
    rng = np.random.default_rng(1000 + seed)
    m, n = 40, 20
    base = rng.standard_normal((m, 3))
    A = base @ rng.standard_normal((3, n)) + 0.2 * rng.standard_normal((m, n))
    b = A @ rng.standard_normal(n) + rng.standard_normal(m)
    x, rep = L.lsm_commission(A, b, method=0)
    xo, it_o = N.lawson_hanson(A, b)
    np.testing.assert_allclose(x, xo, atol=1e-8 * max(1.0, np.abs(xo).max()))
    assert rep["iterations"] == it_o
    assert rep["objective"] == pytest.approx(N.objective(A, b, xo), rel=1e-9)


def test_commission_projected_gradient(L):
    """Sec. 2.2.4 on an inconsistent problem (F* > 0, so the relative change of
    F goes to zero and the stopping rule fires); the limit is the NNLS minimiser."""
    rng = np.random.default_rng(5)
    A = np.abs(rng.standard_normal((300, 40)))
    xt = rng.uniform(0.8, 1.2, 40)
    xt[[4, 9]] = 0.0
    b = A @ xt * (1 + 0.005 * rng.standard_normal(300))
    x, rep = L.lsm_commission(A, b, method=1, delta=1e-13, max_iter=200000)
    assert rep["converged"]
    xo, _ = N.lawson_hanson(A, b)
    xp, _, ok = N.gradient_projection(A, b, delta=1e-13)
    assert ok
    fo = N.objective(A, b, xo)
    assert N.objective(A, b, x) == pytest.approx(fo, rel=1e-7)
    np.testing.assert_allclose(x, xo, atol=2e-3)
    np.testing.assert_allclose(x, xp, atol=2e-3)


def test_commission_spectral_projected_gradient(L):
    """Method 2 (Barzilai-Borwein steps, nonmonotone line search) on the
    problem above: the NNLS minimiser, in far fewer iterations than the Armijo
    projection, and the oracle's version of the method lands on the same x."""
    rng = np.random.default_rng(5)
    A = np.abs(rng.standard_normal((300, 40)))
    xt = rng.uniform(0.8, 1.2, 40)
    xt[[4, 9]] = 0.0
    b = A @ xt * (1 + 0.005 * rng.standard_normal(300))
    x, rep = L.lsm_commission(A, b, method=2, delta=1e-13, max_iter=200000)
    assert rep["converged"]
    _, rep1 = L.lsm_commission(A, b, method=1, delta=1e-13, max_iter=200000)
    assert rep["iterations"] < rep1["iterations"]
    xo, _ = N.lawson_hanson(A, b)
    xb, it_b, ok = N.gradient_projection_bb(A, b, delta=1e-13)
    assert ok
    fo = N.objective(A, b, xo)
    assert N.objective(A, b, x) == pytest.approx(fo, rel=1e-7)
    np.testing.assert_allclose(x, xo, atol=2e-3)
    np.testing.assert_allclose(x, xb, atol=2e-3)
    assert rep["kkt"] < 1e-3 * np.linalg.norm(A.T @ b)


def test_commission_device_inputs_and_errors(L):
    import torch
    rng = np.random.default_rng(1)
    A = np.abs(rng.standard_normal((50, 8)))
    b = A @ np.linspace(0.5, 1.5, 8)
    x_h, _ = L.lsm_commission(A, b)
    x_d, _ = L.lsm_commission(torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda"))
    np.testing.assert_array_equal(x_h, x_d)
    np.testing.assert_allclose(x_h, np.linspace(0.5, 1.5, 8), atol=1e-9)
    with pytest.raises(L.LSMError):
        L.lsm_commission(np.zeros((5, 2000)), np.zeros(5))


def test_async_build_and_unsynchronised_run_match_the_synchronous_ones(L):
    import torch
    wl = W.workload_full_10x10(200_000)
    ph = L.lsm_phantom_create(wl.phantom)
    out = []
    for async_, no_sync in ((False, False), (True, True), (True, False)):
        g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist // 4, async_=async_)
        t = L.lsm_tally_create(ph)
        rc = L.lsm_run(g, ph, t, 17, L.RunOpts(n_batches=4, no_sync=no_sync))
        assert rc == L.LSM_OK
        torch.cuda.synchronize()
        s1, s2, nb = L.lsm_tally_read(t)
        led, st = L.lsm_tally_ledger(t)
        out.append((s1, nb, st, g.info, g.denom))
    for s1, nb, st, info, denom in out[1:]:
        assert nb == out[0][1] and info == out[0][3] and denom == out[0][4]
        assert st["histories"] == out[0][2]["histories"] and st["photons"] == out[0][2]["photons"]
        np.testing.assert_allclose(s1, out[0][0], rtol=1e-4, atol=1e-6 * out[0][0].max())


def test_async_builds_queued_behind_work_keep_their_inputs(L):
    """Five plans of different models and fields built without host
    synchronisation while a long run holds the stream: each plan equals the
    synchronous build of its own inputs (the host staging buffers are not
    reused before their copies have run)."""
    import torch
    wl = W.workload_full_10x10(10_000_000)       # a run of about 2 ms holds the stream
    ph = L.lsm_phantom_create(wl.phantom)
    cases = [(W.psr_model(6, 10, 0.25, seed=s), W.beams(W.square_field(f))) for s, f in
             ((1, 4.0), (2, 10.0), (3, 6.0), (4, 8.0), (5, 2.0))]
    want = []
    for m, b in cases:
        g = L.lsm_build_psl(m, b, 50_000)
        want.append((g.info, g.denom, L.lsm_psl_copy(g, 0), L.lsm_psl_copy(g, 3)))
    torch.cuda.synchronize()
    t = L.lsm_tally_create(ph)
    g0 = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist // 2)
    L.lsm_run(g0, ph, t, 5, L.RunOpts(n_batches=2, no_sync=True))      # queued, still running
    got = [L.lsm_build_psl(m, b, 50_000, async_=True) for m, b in cases]
    torch.cuda.synchronize()
    for g, (info, denom, w0, c3) in zip(got, want):
        assert g.info == info and g.denom == denom
        np.testing.assert_array_equal(L.lsm_psl_copy(g, 0), w0)
        np.testing.assert_array_equal(L.lsm_psl_copy(g, 3), c3)


def test_runs_on_two_streams_match_serial_runs(L):
    """Two dose calculations queued on two CUDA streams (phantom from host
    arrays, unsynchronised plan build and run, read-back of each while the
    other runs) give the results of the same calculations run one after the
    other: counters equal, sums to FP32 atomic ordering."""
    import torch
    wl = W.workload_full_10x10(2_000_000)
    n_plan = wl.n_hist // 4

    def job(seed, stream):
        ph = L.lsm_phantom_create(wl.phantom, stream=stream)
        g = L.lsm_build_psl(wl.model, wl.beams, n_plan, async_=True, stream=stream)
        t = L.lsm_tally_create(ph, stream=stream)
        L.lsm_run(g, ph, t, seed, L.RunOpts(n_batches=4, no_sync=True), stream=stream)
        return ph, g, t, stream

    def read(j):
        ph, g, t, stream = j
        d, s = L.lsm_dose(t, ph, 1.0, stream=stream)
        led, st = L.lsm_tally_ledger(t, stream=stream)
        return d, s, st

    serial = [read(job(seed, torch.cuda.current_stream())) for seed in (41, 42)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    j0 = job(41, streams[0])
    j1 = job(42, streams[1])
    both = [read(j0), read(j1)]
    for (d, s, st), (d0, s0, st0) in zip(both, serial):
        for k in ("histories", "photons", "electrons", "rejected", "flights", "real", "esteps"):
            assert st[k] == st0[k], k
        np.testing.assert_allclose(d, d0, rtol=1e-4, atol=1e-6 * d0.max())
        np.testing.assert_allclose(s, s0, rtol=1e-3, atol=1e-5 * s0.max())


def test_more_batches_than_an_iteration_holds(L):
    """300 batches of a small plan: an iteration holds at most 255 batch slots
    (a particle carries its slot in 8 bits), so the run takes 255 + 45; the
    result equals the same run with one batch per iteration."""
    wl = W.workload_full_10x10(300 * 1000)
    ph = L.lsm_phantom_create(wl.phantom)
    g = L.lsm_build_psl(wl.model, wl.beams, 1000)
    out = []
    for chunk in (0, 1000):                 # library default (2^23): 255 + 45; one batch per iteration
        t = L.lsm_tally_create(ph)
        assert L.lsm_run(g, ph, t, 3, L.RunOpts(n_batches=300, chunk=chunk)) == L.LSM_OK
        s1, s2, nb = L.lsm_tally_read(t)
        led, st = L.lsm_tally_ledger(t)
        out.append((s1, s2, nb, st))
    (a1, a2, na, sa), (b1, b2, nb_, sb) = out
    assert na == nb_ == 300
    for k in ("histories", "photons", "electrons", "rejected", "flights", "real", "esteps"):
        assert sa[k] == sb[k], k
    assert sa["histories"] == 300_000
    np.testing.assert_allclose(a1, b1, rtol=1e-4, atol=1e-6 * b1.max())
    np.testing.assert_allclose(a2, b2, rtol=1e-3, atol=1e-6 * b2.max())


def test_async_build_reports_an_empty_plan_when_read(L):
    import torch
    wl = W.workload_full_10x10(10_000)
    far = W.beams(W.square_field(1.0, cx=60.0, cy=60.0))    # outside every PSL's sampling reach
    with pytest.raises(L.LSMError, match="non-zero weight"):
        L.lsm_build_psl(wl.model, far, 1000)
    g = L.lsm_build_psl(wl.model, far, 1000, async_=True)    # queued; nothing checked yet
    ph = L.lsm_phantom_create(wl.phantom)
    t = L.lsm_tally_create(ph)
    assert L.lsm_run(g, ph, t, 1, L.RunOpts(n_batches=2, no_sync=True)) == L.LSM_OK
    torch.cuda.synchronize()
    led, st = L.lsm_tally_ledger(t)
    assert st["histories"] == 0 and led["deposited"] == 0.0
    with pytest.raises(L.LSMError, match="non-zero weight"):
        L.lsm_psl_info(g)
    with pytest.raises(L.LSMError, match="non-zero weight"):
        L.lsm_run(g, ph, t, 1, L.RunOpts(n_batches=2))


def test_repeated_create_run_destroy_reuses_pooled_memory(L):
    """Phantoms, plans, tallies and workspaces come from the stream-ordered
    pool: a request loop neither grows device memory nor changes results."""
    import torch
    wl = W.workload_full_10x10(100_000)
    ref = None
    free0 = None
    for i in range(8):
        ph = L.lsm_phantom_create(wl.phantom)
        g = L.lsm_build_psl(wl.model, wl.beams, wl.n_hist // 2, async_=(i % 2 == 1))
        t = L.lsm_tally_create(ph)
        L.lsm_run(g, ph, t, 5, L.RunOpts(n_batches=2, chunk=1 << 20, no_sync=(i % 2 == 1)))
        d, _ = L.lsm_dose(t, ph, g.denom / (wl.n_hist // 2))
        if ref is None:
            ref = d
        else:
            np.testing.assert_allclose(d, ref, rtol=1e-4, atol=1e-6 * ref.max())
        del t, g, ph
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        if i == 2:
            free0 = free
        elif i > 2:
            assert free >= free0 - (64 << 20), (i, free0, free)


def test_checkpoint_and_resume_equal_the_uninterrupted_run(L):
    wl = W.workload_full_10x10(160_000)
    n_plan = wl.n_hist // 8
    g = L.lsm_build_psl(wl.model, wl.beams, n_plan)
    ph = L.lsm_phantom_create(wl.phantom)
    full = L.lsm_tally_create(ph)
    L.lsm_run(g, ph, full, 21, L.RunOpts(n_batches=8))
    s1, s2, nb = L.lsm_tally_read(full)
    led, st = L.lsm_tally_ledger(full)
    # the same 8 batches as 3 + checkpoint + 5
    t1 = L.lsm_tally_create(ph)
    L.lsm_run(g, ph, t1, 21, L.RunOpts(n_batches=3))
    c1, c2, cb = L.lsm_tally_read(t1)
    cled, cst = L.lsm_tally_ledger(t1)
    del t1
    t2 = L.lsm_tally_create(ph)
    L.lsm_tally_load(t2, c1, c2, cb, cled, cst)
    L.lsm_run(g, ph, t2, 21, L.RunOpts(n_batches=5, first_batch=3))
    r1, r2, rb = L.lsm_tally_read(t2)
    rled, rst = L.lsm_tally_ledger(t2)
    assert rb == nb == 8
    for k in ("histories", "photons", "electrons", "rejected", "missed", "flights", "real", "esteps"):
        assert rst[k] == st[k], k
    np.testing.assert_allclose(r1, s1, rtol=1e-5, atol=1e-7 * s1.max())
    np.testing.assert_allclose(r2, s2, rtol=1e-4, atol=1e-7 * s2.max())
    np.testing.assert_allclose(rled["source"], led["source"], rtol=1e-12)
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_run(g, ph, t2, 21, L.RunOpts(n_batches=1, first_batch=-1))


def test_energy_is_conserved_history_by_history(L):
    """Per-history ledger (test mode): for every history of a three-sub-source
    CSDA run on a heterogeneous phantom, the deposited + escaped + rejected
    energy of all its particles equals its source particle's energy (FP32
    transport arithmetic: within 1e-4); totals equal the run ledger's; the
    ledger kernels tally as the production ones (same counters, same dose to
    FP32 atomic order)."""
    import torch
    wl = W.workload_full_10x10(40_000)
    ph = W.pelvis_phantom(40, 24, 32, 1.0)
    phh = L.lsm_phantom_create(ph)
    g = L.lsm_build_psl(wl.model, W.gantry_beams([0.0, 120.0], 8.0), 20_000)
    nb = 2
    t = L.lsm_tally_create(phh)
    buf = torch.zeros((20_000 * nb, 2), dtype=torch.float64, device="cuda")
    L.lsm_tally_history_ledger(t, buf, first_history=0)
    assert L.lsm_run(g, phh, t, 9, L.RunOpts(n_batches=nb)) == L.LSM_OK
    hl = buf.cpu().numpy()
    src, acc = hl[:, 0], hl[:, 1]
    assert (src > 0).all()
    np.testing.assert_allclose(acc, src, rtol=1e-4, atol=0)
    led, st = L.lsm_tally_ledger(t)
    assert abs(src.sum() / led["source"] - 1) < 1e-9
    assert abs(acc.sum() / (led["rejected"] + led["escaped"] + led["deposited"]) - 1) < 1e-6
    s1, _, _ = L.lsm_tally_read(t)
    t2 = L.lsm_tally_create(phh)
    L.lsm_run(g, phh, t2, 9, L.RunOpts(n_batches=nb))
    r1, _, _ = L.lsm_tally_read(t2)
    led2, st2 = L.lsm_tally_ledger(t2)
    for k in ("histories", "photons", "electrons", "rejected", "missed", "flights", "real", "esteps"):
        assert st[k] == st2[k], k
    np.testing.assert_allclose(s1, r1, rtol=1e-4, atol=1e-6 * r1.max())
    # detached: the tally runs the production kernels again
    L.lsm_tally_history_ledger(t, None)
    L.lsm_tally_reset(t)
    assert L.lsm_run(g, phh, t, 9, L.RunOpts(n_batches=nb)) == L.LSM_OK
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        idx, n_rows = W.commissioning_index(W.water_phantom(16, 16, 16, 0.5))
        tb = L.lsm_tally_create(L.lsm_phantom_create(W.water_phantom(16, 16, 16, 0.5)), mode=1, idx3d=idx,
                                n_rows=n_rows, n_psr=300)
        L.lsm_tally_history_ledger(tb, buf)


def test_l2_atomic_peak(L):
    # the tally-update ceiling the bench reports transport step rates against:
    # a finite rate well above the transport's own steps per second
    r = L.lsm_l2_atomic_peak(64 ** 3 * 16, reps=3)
    assert math.isfinite(r) and r > 1e10
    small = L.lsm_l2_atomic_peak(1, reps=1)            # every update on one cell: contention, still positive
    assert 0 < small < r
    for bad in ((0, 1), (2 ** 31 + 1, 1), (1024, 0), (1024, 1001)):
        with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
            L.lsm_l2_atomic_peak(*bad)


@pytest.mark.parametrize("nb", [1, 4])
def test_dose_and_sigma_from_the_tally(L, nb):
    # lsm_dose against its definition from the tally sums: D = S1 / B * scale /
    # (rho V), sigma = sqrt(B var) / B * scale / (rho V), var the batch variance
    # max(S2 - S1^2 / B, 0) / (B - 1) (0 for one batch); FP64 to rounding
    model = W.psr_model(6, 10, 0.25, seed=2)
    ph = W.pelvis_phantom(24, 20, 16, 1.0)
    phh = L.lsm_phantom_create(ph)
    g = L.lsm_build_psl(model, W.gantry_beams([0.0, 90.0], 8.0), 20_000)
    t = L.lsm_tally_create(phh)
    L.lsm_run(g, phh, t, 3, L.RunOpts(electron_mode=1, n_batches=nb))
    s1, s2, b = L.lsm_tally_read(t)
    assert b == nb
    scale = 0.37
    d, s = L.lsm_dose(t, phh, scale)
    m = ph.rho.ravel().astype(np.float64) * (ph.dx * ph.dy * ph.dz)
    var = np.clip(s2 - s1 * s1 / nb, 0.0, None) / (nb - 1) if nb > 1 else np.zeros_like(s1)
    np.testing.assert_allclose(d.ravel(), s1 / nb * scale / m, rtol=1e-14, atol=0)
    np.testing.assert_allclose(s.ravel(), np.sqrt(nb * var) / nb * scale / m, rtol=1e-13, atol=1e-300)
    assert (d > 0).sum() > 100 and (nb == 1 or (s > 0).sum() > 100)


def test_device_philox_equals_the_oracle(L):
    # the device's Philox4x32-10 against the oracle's (itself pinned to
    # PyTorch's engine): every word of blocks at several histories, stream ids
    # and draws, including a history above 2^32 and a seed using both halves
    rng = np.random.default_rng(4)
    for seed, g0, sid, draw in ((0, 0, 0, 0), (0x1234_5678_9ABC_DEF0, 7, 1, 3),
                                (2 ** 63 + 5, 2 ** 32 - 3, 0x8000_0001, 2 ** 31 + 9), (42, 10 ** 12, 77, 0)):
        n = 257
        got = L.lsm_philox_blocks(seed, g0, sid, draw, n)
        for i in list(range(8)) + list(rng.integers(0, n, 16)) + [n - 1]:
            g = g0 + int(i)
            want = O.philox4x32_10([seed & 0xFFFFFFFF, seed >> 32],
                                   [g & 0xFFFFFFFF, g >> 32, sid, draw])
            np.testing.assert_array_equal(got[i], want, err_msg=str((seed, g, sid, draw)))
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_philox_blocks(1, 0, 0, 0, 0)


def test_transport_cutoffs_are_the_papers(L):
    # the cutoffs of tests/golden/paper_values.txt (Sec. 3.1: 200 keV electrons,
    # 50 keV photons) on the device: a particle just below its cutoff deposits
    # where it enters (no Woodcock flight, no CSDA step); just above, it moves
    import os
    import torch
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                vals[line.split()[0]] = float(line.split()[1])
    ph = W.water_phantom(16, 16, 16, 0.5)
    phh = L.lsm_phantom_create(ph)
    for kind, cut, counter in ((0, vals["photon_cutoff"], "flights"), (1, vals["electron_cutoff"], "esteps")):
        for E, moves in ((cut * (1 - 1e-5), False), (cut * (1 + 1e-3), True)):
            p = L.alloc_particles(1)
            for k, v in (("x", ph.x0 + 4.0), ("y", ph.y0 + 4.0), ("z", ph.z0), ("u", 0.0), ("v", 0.0), ("w", 1.0),
                         ("E", E)):
                p[k].fill_(v)
            p["hist"].fill_(0)
            p["psr"].fill_(0)
            p["beam"].fill_(0)
            p["type"].fill_(kind)
            p["status"].fill_(0)
            t = L.lsm_tally_create(phh)
            L.lsm_transport(phh, p, 1, 5, t, L.RunOpts(electron_mode=1))
            torch.cuda.synchronize()
            led, st = L.lsm_tally_ledger(t)
            assert (st[counter] > 0) == moves, (kind, E, st[counter])
            assert led["deposited"] + led["escaped"] == pytest.approx(E, rel=1e-5)
