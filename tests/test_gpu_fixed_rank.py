"""End-to-end parity of rsvd_fixed_rank with the float64 oracle (same seed, same
Omega), plus argument and edge-case handling through the C ABI (GPU)."""
import ctypes

import numpy as np
import pytest

import oracle
from workloads import exp_decay_matrix, lowrank_np, poly_spectrum, exact_rank_matrix, poly_decay_matrix_np

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _np(*ts):
    return [t.cpu().numpy().astype(np.float64) for t in ts]


def test_exp_decay_2000x1000_f64(lib):
    """The 2000 x 1000 exp(-j/10) workload, k = 20, p = 10, q = 1, binary64 end to end."""
    A = exp_decay_matrix(2000, 1000, seed=1001)
    k, p, q, seed = 20, 10, 1, 1001
    U, D, V = _np(*lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=lib.RSVD_F64))
    ref = oracle.rsvd_power(A, k, p, q, seed)
    np.testing.assert_allclose(D, ref["D"], rtol=1e-12)
    np.testing.assert_allclose(U, ref["U"], atol=1e-10)
    np.testing.assert_allclose(V, ref["V"], atol=1e-10)
    err = np.linalg.norm(A - (U * D) @ V.T, 2)
    err_ref = np.linalg.norm(A - (ref["U"] * ref["D"]) @ ref["V"].T, 2)
    assert err <= 1.001 * err_ref


@pytest.mark.parametrize("m,n,k,p,q", [(2000, 1000, 20, 10, 1), (1500, 1100, 40, 24, 2), (3001, 999, 100, 28, 1),
                                       (600, 900, 7, 5, 0), (4096, 4096, 200, 56, 2)])
def test_poly_decay_f32(lib, m, n, k, p, q):
    A = lowrank_np(m, n, poly_spectrum(min(m, n), 1.5), seed=m + n).astype(np.float32)
    A64 = A.astype(np.float64)
    seed = 2000 + k
    U, D, V = _np(*lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=lib.RSVD_F32))
    ref = oracle.rsvd_power(A64, k, p, q, seed)
    d1 = ref["D"][0]
    tol = 1e-5 * ref["D"] + 16 * U32 * np.sqrt(m) * d1
    assert np.all(np.abs(D - ref["D"]) <= tol), np.max(np.abs(D - ref["D"]) / tol)
    err = oracle.fro_residual(A64, U, D, V)
    err_ref = oracle.fro_residual(A64, ref["U"], ref["D"], ref["V"])
    assert err <= 1.001 * err_ref + 16 * U32 * np.sqrt(m) * np.linalg.norm(A64)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-4)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-4)


def test_full_l_and_exact_rank(lib):
    """l > rank(A): the Gram matrices are singular; the shifted pass keeps it
    going and the rank-k part is recovered exactly (Sec. 4)."""
    A = exact_rank_matrix(700, 500, 12, seed=3)
    U, D, V = _np(*lib.fixed_rank(_t(A), 12, 8, 1, seed=5, prec=lib.RSVD_F64, full=True))
    assert U.shape == (700, 20) and D.shape == (20,)
    sig = np.linalg.svd(A, compute_uv=False)[:12]
    np.testing.assert_allclose(D[:12], sig, rtol=1e-10)
    rec = (U[:, :12] * D[:12]) @ V[:, :12].T
    assert np.linalg.norm(A - rec) <= 1e-10 * np.linalg.norm(A)
    A32 = A.astype(np.float32)
    U, D, V = _np(*lib.fixed_rank(_t(A32), 12, 8, 1, seed=5, prec=lib.RSVD_F32))
    np.testing.assert_allclose(D, sig, rtol=1e-4)


def test_argument_errors(lib):
    import torch
    A = torch.zeros(50, 40, dtype=torch.float32, device="cuda")
    h = lib.handle()
    for bad in [dict(k=45, p=0), dict(k=30, p=20), dict(k=-1, p=0)]:
        prm = lib.make_params(bad["k"], bad["p"], 1, 0, lib.RSVD_F32, lib.RSVD_FLAG_SYNC)
        out = ctypes.c_size_t()
        code = lib.load().rsvd_workspace_size(h, 50, 40, ctypes.byref(prm), ctypes.byref(out))
        assert code == lib.RSVD_E_INVALID
    prm = lib.make_params(5, 5, 1, 0, lib.RSVD_F32, 0)
    U = torch.empty(50, 5, device="cuda")
    V = torch.empty(40, 5, device="cuda")
    D = torch.empty(5, dtype=torch.float64, device="cuda")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    assert lib.rsvd_fixed_rank(h, 50, 40, A, 40, prm, U, 5, D, V, 5, small) == lib.RSVD_E_NOMEM
    assert lib.rsvd_fixed_rank(h, 50, 40, A, 39, prm, U, 5, D, V, 5, small) == lib.RSVD_E_INVALID
    prm.prec = lib.RSVD_MIXED_FP8
    assert lib.rsvd_fixed_rank(h, 50, 40, A, 40, prm, U, 5, D, V, 5, small) == lib.RSVD_E_NOMEM
    prm.prec = 9  # no such precision
    assert lib.rsvd_fixed_rank(h, 50, 40, A, 40, prm, U, 5, D, V, 5, small) == lib.RSVD_E_UNSUPPORTED
    # k = 0: nothing to compute, nothing enqueued
    prm = lib.make_params(0, 0, 0, 0, lib.RSVD_F32, 0)
    assert lib.rsvd_fixed_rank(h, 50, 40, A, 40, prm, U, 5, D, V, 5, small) == lib.RSVD_OK


def test_nonfinite_input_reports_status(lib):
    A = lowrank_np(300, 200, poly_spectrum(200, 1.0), seed=1).astype(np.float32)
    A[17, 3] = np.nan
    with pytest.raises(lib.RsvdError) as ei:
        lib.fixed_rank(_t(A), 10, 5, 1, seed=1, prec=lib.RSVD_F32)
    assert ei.value.code == lib.RSVD_E_NONFINITE


def test_deterministic_bits(lib):
    A = lowrank_np(1200, 800, poly_spectrum(800, 1.0), seed=2).astype(np.float32)
    r1 = _np(*lib.fixed_rank(_t(A), 30, 10, 2, seed=9, prec=lib.RSVD_F32))
    r2 = _np(*lib.fixed_rank(_t(A), 30, 10, 2, seed=9, prec=lib.RSVD_F32))
    for a, b in zip(r1, r2):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec_name", ["RSVD_MIXED_BF16", "RSVD_MIXED_FP8"])
def test_host_buffers_zero_copy(lib, prec_name):
    """The mixed paths read A once, in the conversion pass: a pinned host A and
    pinned host outputs give the same bits as device buffers.  Pageable host
    memory is either accepted (devices with pageable-memory access) with the
    same bits, or refused before anything is launched."""
    import torch
    prec = getattr(lib, prec_name)
    m, n, k, p, q, seed = 3000, 2048, 40, 24, 1, 3
    A = torch.from_numpy(poly_decay_matrix_np(m, n, seed=5)).cuda()
    Ud, Dd, Vd = lib.fixed_rank(A, k, p, q, seed=seed, prec=prec)
    h = lib.handle()
    prm = lib.make_params(k, p, q, seed=seed, prec=prec, flags=lib.RSVD_FLAG_SYNC)
    ws = torch.empty(lib.rsvd_workspace_size(h, m, n, prm), dtype=torch.uint8, device="cuda")
    Ah = A.cpu().pin_memory()
    U = torch.empty(m, k).pin_memory()
    D = torch.empty(k, dtype=torch.float64).pin_memory()
    V = torch.empty(n, k).pin_memory()
    assert lib.rsvd_fixed_rank(h, m, n, Ah, n, prm, U, k, D, V, k, ws) == lib.RSVD_OK
    torch.cuda.synchronize()
    assert torch.equal(D, Dd.cpu()) and torch.equal(U, Ud.cpu()) and torch.equal(V, Vd.cpu())
    Ap = A.cpu()
    D.zero_()
    code = lib.rsvd_fixed_rank(h, m, n, Ap, n, prm, U, k, D, V, k, ws)
    torch.cuda.synchronize()
    assert code in (lib.RSVD_OK, lib.RSVD_E_INVALID)
    if code == lib.RSVD_OK:
        assert torch.equal(D, Dd.cpu())
    else:
        assert "not memory the device can access" in lib.last_error(h)
