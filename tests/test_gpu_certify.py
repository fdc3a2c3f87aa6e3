"""rsvd_certify (Sec. 14: eq. infomm and Lemma thm:aposteriori) against the
oracle's certificate computed with the same 16 Gaussian columns of Philox
stream 2, and against the true residual norms."""
import numpy as np
import pytest

from oracle import controller as OC
from workloads import poly_decay_matrix_np

pytestmark = pytest.mark.gpu


def test_certify_matches_oracle_and_bounds_the_residual(lib):
    import torch
    m, n = 1500, 900
    Af = poly_decay_matrix_np(m, n, seed=4).astype(np.float64)
    A = torch.from_numpy(Af.astype(np.float32)).cuda()
    Af = A.cpu().double().numpy()
    U, D, V = lib.fixed_rank(A, 40, 10, 1, seed=2, prec=lib.RSVD_F32)
    est, bound, fa = lib.certify(A, U, D, V, seed=9)
    Uo, Do, Vo = U.cpu().double().numpy(), D.cpu().numpy(), V.cpu().double().numpy()
    e_ref, b_ref, _ = OC.residual_estimate(Af, Uo, Do, Vo, 9, r=16)
    # binary32 products against float64: the residual is ~4e-3 of A, so the
    # products' rounding (~sqrt(n) u of A's scale) stays below 1e-3 of it
    assert est == pytest.approx(e_ref, rel=1e-3)
    assert bound == pytest.approx(b_ref, rel=1e-3)
    assert fa == pytest.approx(np.linalg.norm(Af), rel=1e-6)
    R = Af - (Uo * Do) @ Vo.T
    assert 0.4 < est / np.linalg.norm(R) < 2.5
    assert bound >= np.linalg.norm(R, 2)
    # r = 0 certifies the zero approximation: the estimate of ||A||_F
    e0, _, _ = lib.certify(A, None, None, None, seed=9)
    e0_ref, _, _ = OC.residual_estimate(Af, np.zeros((m, 0)), np.zeros(0), np.zeros((n, 0)), 9, r=16)
    assert e0 == pytest.approx(e0_ref, rel=1e-5)


def test_certify_argument_errors(lib):
    import ctypes
    h = lib.handle()
    out = ctypes.c_size_t()
    assert lib.load().rsvd_certify_workspace_size(h, 0, 10, 1, ctypes.byref(out)) == lib.RSVD_E_INVALID
    assert lib.load().rsvd_certify_workspace_size(h, 10, 10, 1025, ctypes.byref(out)) == lib.RSVD_E_INVALID
    assert lib.load().rsvd_certify_workspace_size(h, 10, 10, 4, ctypes.byref(out)) == lib.RSVD_OK
