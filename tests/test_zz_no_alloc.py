"""The allocation-free commissioning entry point (lsm_commission_static).

It serves callers that may not allocate GPU memory while they run (a service
that reserves its device memory at start-up, or a host application that owns
the GPU memory and loads this library as a plugin). Its results must match
lsm_commission within the tolerance of the other NNLS parity tests, on two
calls in a row, since every call reuses one fixed scratch array.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _problem(m, n, seed):
    rng = np.random.default_rng(seed)
    A = np.abs(rng.standard_normal((m, n))) + 0.1 * rng.standard_normal((m, n))
    xt = rng.uniform(0.8, 1.2, n)
    xt[rng.random(n) < 0.1] = 0.0
    b = A @ xt * (1 + 0.005 * rng.standard_normal(m))
    return A, b


def test_static_scratch_matches_allocating_solve_twice():
    import torch
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    # a larger problem first, then a smaller one: the second call must not see
    # anything the first call left in the shared scratch
    for (m, n, seed) in ((500, 200, 11), (120, 30, 12)):
        A, b = _problem(m, n, seed)
        x_ref, rep_ref = lsm.lsm_commission(A, b, method=0)
        Ad = torch.tensor(A, device="cuda")
        bd = torch.tensor(b, device="cuda")
        xd = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
        rep = lsm.lsm_commission_static(Ad, bd, xd, method=0)
        x = xd.cpu().numpy()
        np.testing.assert_allclose(x, x_ref, atol=1e-9 * max(1.0, np.abs(x_ref).max()))
        assert rep["objective"] == pytest.approx(rep_ref["objective"], rel=1e-9)
        assert rep["kkt"] < 1e-10 * np.linalg.norm(2 * A.T @ b)
    # projected gradient through the same scratch, against the allocating entry point
    A, b = _problem(300, 40, 13)
    x_ref, _ = lsm.lsm_commission(A, b, method=1, delta=1e-13)
    xd = torch.zeros(40, dtype=torch.float64, device="cuda")
    rep = lsm.lsm_commission_static(torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda"), xd,
                                    method=1, delta=1e-13)
    assert rep["converged"]
    np.testing.assert_allclose(xd.cpu().numpy(), x_ref, atol=1e-9)


def test_static_call_allocates_no_device_memory():
    """The property the entry point exists for: after a warm-up call (which
    looks up the scratch array's address), further calls leave the device's
    free memory exactly unchanged."""
    import torch
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    A, b = _problem(400, 120, 21)
    Ad, bd = torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda")
    xd = torch.zeros(120, dtype=torch.float64, device="cuda")
    lsm.lsm_commission_static(Ad, bd, xd, method=0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for method in (0, 1, 0):
        lsm.lsm_commission_static(Ad, bd, xd, method=method, max_iter=2000 if method else 0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_warm_start_and_iteration_cap():
    """Projected gradient from the caller's x (use_x0) equals the allocating
    entry point's projected gradient from the same start, and its objective
    the active-set minimum; one iteration returns LSM_ERR_NOT_CONVERGED with x
    still finite and non-negative."""
    import torch
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    A, b = _problem(300, 40, 23)
    x_as, rep_as = lsm.lsm_commission(A, b, method=0)
    x0 = np.clip(x_as + 0.05, 0, None)
    x_pg, _ = lsm.lsm_commission(A, b, method=1, delta=1e-14, x0=x0)
    Ad, bd = torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda")
    xd = torch.tensor(x0, device="cuda")
    rep = lsm.lsm_commission_static(Ad, bd, xd, method=1, delta=1e-14, use_x0=True)
    assert rep["converged"] and rep["status"] == lsm.LSM_OK
    np.testing.assert_allclose(xd.cpu().numpy(), x_pg, atol=1e-9)
    assert rep["objective"] == pytest.approx(rep_as["objective"], rel=1e-9)
    xd = torch.zeros(40, dtype=torch.float64, device="cuda")
    rep = lsm.lsm_commission_static(Ad, bd, xd, method=1, max_iter=1)
    assert rep["status"] == lsm.LSM_ERR_NOT_CONVERGED and not rep["converged"]
    x1 = xd.cpu().numpy()
    assert np.all(np.isfinite(x1)) and np.all(x1 >= 0)


def test_static_rejects_host_and_mistyped_buffers():
    import ctypes as C
    import torch
    from paper_1503_01725_b300 import lsm
    L = lsm.load_library()
    An, bn = _problem(8, 4, 5)
    A = torch.tensor(An, device="cuda")
    b = torch.tensor(bn, device="cuda")
    for bad in (torch.zeros(4, dtype=torch.float64), torch.zeros(4, dtype=torch.float32, device="cuda"),
                torch.zeros(3, dtype=torch.float64, device="cuda")):
        with pytest.raises(lsm.LSMError) as e:
            lsm.lsm_commission_static(A, b, bad)
        assert e.value.status == lsm.LSM_ERR_ARG
    # a C caller passing host memory gets LSM_ERR_ARG, not a device fault
    host = np.zeros(4)
    rc = L.lsm_commission_static(A.data_ptr(), 8, 4, b.data_ptr(), None,
                                 host.ctypes.data_as(C.c_void_p), None, None)
    assert rc == lsm.LSM_ERR_ARG
    # the entry point stays usable
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert lsm.lsm_commission_static(A, b, x)["status"] == lsm.LSM_OK


def test_static_scratch_rejects_oversized_problems():
    import torch
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    A = torch.zeros((10, 257), dtype=torch.float64, device="cuda")
    with pytest.raises(lsm.LSMError) as e:
        lsm.lsm_commission_static(A, torch.zeros(10, dtype=torch.float64, device="cuda"),
                                  torch.zeros(257, dtype=torch.float64, device="cuda"))
    assert e.value.status == lsm.LSM_ERR_ARG
