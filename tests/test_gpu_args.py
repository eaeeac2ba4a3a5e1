"""Argument errors through the C ABI: each call rejects invalid input with
LSM_ERR_ARG (and a message) before any GPU work, and the library stays usable
afterwards (a valid run follows the failed calls)."""
import dataclasses

import numpy as np
import pytest

from paper_1503_01725_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    return lsm


def _arg_error(L, fn, match=None):
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG") as e:
        fn()
    assert e.value.status == L.LSM_ERR_ARG
    if match:
        assert match in str(e.value), str(e.value)


def test_phantom_arguments(L):
    ph = W.water_phantom(8, 8, 8, 0.5)
    for rho, mat in ((0.0, 0), (30.0, 0), (np.nan, 0), (1.0, 2)):
        bad = dataclasses.replace(ph, rho=np.full_like(ph.rho, 1.0), mat=np.zeros_like(ph.mat))
        bad.rho[3, 4, 5] = rho
        bad.mat[3, 4, 5] = mat
        _arg_error(L, lambda: L.lsm_phantom_create(bad), "densities")
    _arg_error(L, lambda: L.lsm_phantom_create(dataclasses.replace(ph, dx=0.0)), "voxel sizes")


def test_run_option_arguments(L):
    wl = W.workload_full_10x10(40_000)
    ph = L.lsm_phantom_create(wl.phantom)
    g = L.lsm_build_psl(wl.model, wl.beams, 10_000)
    t = L.lsm_tally_create(ph)
    base = L.RunOpts(n_batches=2)
    for bad, msg in ((dict(majorant_factor=0.5), "majorant_factor"), (dict(f_e=0.0), "f_e"),
                     (dict(f_e=1.5), "f_e"), (dict(max_steps=0), "max_steps"), (dict(chunk=(1 << 24) + 1), "chunk"),
                     (dict(ctas_per_sm=-1), "ctas_per_sm"), (dict(electron_mode=2), "electron_mode"),
                     (dict(first_batch=-3), "first_batch")):
        _arg_error(L, lambda: L.lsm_run(g, ph, t, 1, dataclasses.replace(base, **bad)), msg)
    # a tally of another phantom
    other = L.lsm_tally_create(L.lsm_phantom_create(W.water_phantom(16, 16, 16, 0.5)))
    _arg_error(L, lambda: L.lsm_run(g, ph, other, 1, base), "another phantom")
    # the failed calls left nothing behind: a valid run on the same handles
    assert L.lsm_run(g, ph, t, 1, base) == L.LSM_OK
    led, st = L.lsm_tally_ledger(t)
    assert st["histories"] == 20_000 and led["deposited"] > 0


def test_basis_tally_arguments(L):
    ph = W.water_phantom(16, 16, 16, 0.5)
    phh = L.lsm_phantom_create(ph)
    idx = np.zeros((16, 16, 16), dtype=np.uint16)
    idx[:, 8, 8] = np.arange(1, 17)
    L.lsm_tally_create(phh, mode=1, idx3d=idx, n_rows=16, n_psr=300)       # valid
    bad = idx.copy()
    bad[0, 0, 0] = 17
    _arg_error(L, lambda: L.lsm_tally_create(phh, mode=1, idx3d=bad, n_rows=16, n_psr=300), "beyond n_rows")
    # a basis tally whose PSR count does not match the plan's
    wl = W.workload_full_10x10(10_000)
    t = L.lsm_tally_create(phh, mode=1, idx3d=idx, n_rows=16, n_psr=7)
    g = L.lsm_build_psl(wl.model, wl.beams, 1000)
    _arg_error(L, lambda: L.lsm_run(g, phh, t, 1, L.RunOpts()), "basis tally shape")


def test_denoiser_arguments(L):
    w = np.zeros((24, 3, 3, 3, 16), dtype=np.float32)
    _arg_error(L, lambda: L.lsm_conv3d_create(16, 24, w), "channels")
    from oracle import denoise as DN
    net = L.lsm_unet_create(DN.init_params(0, head_scale=0.05))
    d = np.zeros((1, 12, 16, 16), dtype=np.float32)                       # 12 is not a multiple of 8
    _arg_error(L, lambda: L.lsm_unet_forward(net, d, np.ones_like(d)), "multiples of 8")
    ok = np.zeros((1, 8, 8, 8), dtype=np.float32)
    assert L.lsm_unet_forward(net, ok, np.ones_like(ok)).shape == ok.shape


def test_commission_arguments(L):
    A = np.abs(np.random.default_rng(0).standard_normal((20, 6)))
    b = A @ np.ones(6)
    _arg_error(L, lambda: L.lsm_commission(A, b, method=3), "method")
    x, rep = L.lsm_commission(A, b)
    np.testing.assert_allclose(x, np.ones(6), atol=1e-9)
