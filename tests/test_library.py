"""Host-side checks of the C-ABI library that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1503_01725_b300", "liblsm.so")
HDR = os.path.join(ROOT, "include", "lsm.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1503_01725_b300 import build
        build.build()
    return ctypes.CDLL(LIB)


def declared():
    txt = open(HDR).read()
    return re.findall(r"^\s*(?:lsm_status|void|const char\s*\*|int64_t)\s*\*?\s*(lsm_\w+)\s*\(", txt, re.M)


def test_header_declares_the_boundary():
    names = declared()
    for n in ("lsm_build_psl", "lsm_sample", "lsm_transport", "lsm_run", "lsm_commission"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing


def test_binding_covers_every_declared_symbol():
    from paper_1503_01725_b300 import lsm
    assert set(declared()) <= set(lsm.exported_symbols())


def test_no_gpu_means_loud_failure(monkeypatch):
    import torch
    from paper_1503_01725_b300 import lsm
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    monkeypatch.setattr(lsm, "_lib", None)
    with pytest.raises(RuntimeError):
        lsm.load_library()


def test_launch_counter_readable_without_gpu(lib):
    lib.lsm_launch_count.restype = ctypes.c_int64
    assert lib.lsm_launch_count() >= 0
    lib.lsm_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.lsm_last_error(), bytes)


def test_autotune_candidates():
    from paper_1503_01725_b300 import autotune as A
    c = A.candidates(625_000, 16, ctas=(0,), graphs=(False,))
    chunks = [x[0] for x in c]
    # whole-batch multiples of the plan: 1, 2, 4, 8, 16 batches per iteration
    assert chunks == [625_000 * k for k in (1, 2, 4, 8, 16)]
    big = A.candidates(50_000_000, 1, ctas=(0,), graphs=(False,))
    assert [x[0] for x in big] == [1 << 21, 1 << 22, 1 << 23, 1 << 24]
    assert all(x[0] <= A.MAX_CHUNK for x in A.candidates(3_000_000, 64))


def _model_calls(lib):
    from paper_1503_01725_b300 import lsm
    lib.lsm_model_create.argtypes = [ctypes.POINTER(lsm.lsm_psr_model), ctypes.POINTER(ctypes.c_void_p)]
    lib.lsm_model_destroy.argtypes = [ctypes.c_void_p]
    lib.lsm_model_commission.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_void_p)]
    lib.lsm_model_weights.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    return lsm


def test_model_handle_on_the_host(lib):
    """lsm_model_create / lsm_model_commission / lsm_model_weights touch no
    GPU: the handle keeps its own copy, validates the model, and the
    commissioned weights are W_R x_R with x per PSR or per Eq. 8 unknown
    (electron units of one energy bin share a factor)."""
    import numpy as np
    from paper_1503_01725_b300 import workloads as W
    lsm = _model_calls(lib)
    dp = ctypes.POINTER(ctypes.c_double)
    m = W.psr_model(4, 5, 0.3, seed=2)
    w0 = m.w.copy()
    ms, _ = lsm._marshal(m, lsm._NO_BEAMS)
    h = ctypes.c_void_p()
    assert lib.lsm_model_create(ctypes.byref(ms), ctypes.byref(h)) == 0 and h.value
    m.w[...] = -1.0                         # the caller's array changes; the handle does not
    got = np.zeros(w0.shape)
    assert lib.lsm_model_weights(h, got.ctypes.data_as(dp)) == 0
    assert np.array_equal(got, w0)
    m.w[...] = w0
    rng = np.random.default_rng(4)
    n_ph = 2 * m.n_e * m.n_r
    for n_x in (3 * m.n_e * m.n_r, n_ph + m.n_e):
        x = rng.uniform(0.5, 1.5, n_x)
        hc = ctypes.c_void_p()
        assert lib.lsm_model_commission(h, x.ctypes.data_as(dp), n_x, ctypes.byref(hc)) == 0
        assert lib.lsm_model_weights(hc, got.ctypes.data_as(dp)) == 0
        f = x if n_x == w0.size else np.concatenate([x[:n_ph], np.repeat(x[n_ph:], m.n_r)])
        assert np.array_equal(got.ravel(), w0.ravel() * f)
        lib.lsm_model_destroy(hc)
    bad = ctypes.c_void_p(1)
    x = np.ones(7)
    assert lib.lsm_model_commission(h, x.ctypes.data_as(dp), 7, ctypes.byref(bad)) == 1 and not bad.value
    x = np.ones(w0.size)
    x[3] = -0.1
    assert lib.lsm_model_commission(h, x.ctypes.data_as(dp), w0.size, ctypes.byref(bad)) == 1
    lib.lsm_model_destroy(h)
    # invalid models are rejected with LSM_ERR_ARG and no handle
    m.w[0, 0, 0] = np.nan
    ms, _ = lsm._marshal(m.with_weights(m.w.copy()), lsm._NO_BEAMS)
    h = ctypes.c_void_p(1)
    assert lib.lsm_model_create(ctypes.byref(ms), ctypes.byref(h)) == 1 and not h.value
    lib.lsm_last_error.restype = ctypes.c_char_p
    assert b"lsm_model_create" in lib.lsm_last_error()


def test_library_has_no_unresolved_own_symbols(lib):
    """Every symbol of the library's own namespace is defined in it (a helper
    declared in one file and left in another file's anonymous namespace would
    link but fail when loaded)."""
    import subprocess
    out = subprocess.check_output(["nm", "-D", "--undefined-only", LIB], text=True)
    own = [ln for ln in out.splitlines() if "_ZN3lsm" in ln or " lsm_" in ln]
    assert not own, own


def test_run_statistics_layout_agrees_across_header_binding_and_reduction():
    """lsm_tally_ledger and lsm_tally_load exchange one int64 array of run
    statistics: the header's length, the binding's keys and the multi-GPU
    reduction's keys must agree, and the header must list them in that order."""
    from paper_1503_01725_b300 import dist, lsm
    txt = open(HDR).read()
    sizes = set(re.findall(r"int64_t stats\[(\d+)\]", txt))
    assert sizes == {str(len(lsm.STAT_KEYS))}
    assert tuple(dist.STAT_KEYS) == tuple(lsm.STAT_KEYS)
    doc = re.search(r"stats: histories, accepted photons.*?Synchronises", txt, re.S).group(0)
    order = ["histories", "accepted photons", "accepted electrons", "rejected", "missed", "Woodcock flights",
             "real photon interactions", "electron steps", "step-cap hits", "queue overflows", "secondary electrons"]
    pos = [doc.find(w) for w in order]
    assert all(p >= 0 for p in pos) and pos == sorted(pos) and len(order) == len(lsm.STAT_KEYS)
