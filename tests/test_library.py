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
