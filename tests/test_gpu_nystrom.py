"""rsvd_nystrom (Fig. nystrom) against the float64 oracle with the same Omega:
eigenvalues and eigenvectors, the Loewner order A - U Lam U^T >= 0, the
report on a rank-deficient input, and argument errors."""
import numpy as np
import pytest

import oracle
from workloads import spd_matrix_np

pytestmark = pytest.mark.gpu


def _spd(n, lam, seed):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((n, len(lam))))
    A = (V * lam[None, :]) @ V.T
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("prec_name", ["RSVD_F64", "RSVD_F32"])
def test_nystrom_matches_oracle(lib, prec_name):
    import torch
    prec = getattr(lib, prec_name)
    n, k, p, seed = 600, 20, 10, 5
    A = _spd(n, np.exp(-np.arange(n) / 8.0), 3)
    ref = oracle.nystrom(A, k, p, seed)
    dt = torch.float64 if prec == lib.RSVD_F64 else torch.float32
    At = torch.from_numpy(A).to(dt).cuda()
    U, L = lib.nystrom(At, k, p, seed=seed, prec=prec)
    U = U.cpu().double().numpy()
    L = L.cpu().numpy()
    if prec == lib.RSVD_F64:
        np.testing.assert_allclose(L, ref["L"], rtol=1e-10)
        np.testing.assert_allclose(U, ref["U"], atol=1e-8)
    else:
        # binary32 data: eigenvalues to a few u32 relative to lambda_1, vectors of
        # gaps >= 10% to ~1e-4
        np.testing.assert_allclose(L, ref["L"], rtol=1e-4, atol=1e-6 * ref["L"][0])
        np.testing.assert_allclose(U, ref["U"], atol=2e-3)
    assert np.max(np.abs(U.T @ U - np.eye(k))) < (1e-12 if prec == lib.RSVD_F64 else 1e-5)
    E = A - (U * L[None, :]) @ U.T
    assert np.linalg.eigvalsh(0.5 * (E + E.T)).min() > -(1e-10 if prec == lib.RSVD_F64 else 1e-5)


def test_nystrom_full_l_and_poly_spectrum(lib):
    import torch
    n, k, p, seed = 800, 30, 16, 11
    A = spd_matrix_np(n, seed=2)
    ref = oracle.nystrom(A, k, p, seed, full=True)
    U, L = lib.nystrom(torch.from_numpy(A).cuda(), k, p, seed=seed, prec=lib.RSVD_F64, full=True)
    np.testing.assert_allclose(L.cpu().numpy(), ref["L"], rtol=1e-9)
    assert U.shape == (n, k + p)


def test_nystrom_rank_deficient_input_is_reported(lib):
    """rank(A) = 12 < l = 24: Q^T A Q is singular to working precision.  Its
    unit-diagonal scaling turns the null block into rounding noise of order
    one, which no small shift makes positive definite, so the call reports
    RSVD_E_BREAKDOWN instead of returning a wrong factor (a shifted variant,
    A + nu I with nu subtracted from Lambda, is not part of Fig. nystrom)."""
    import torch
    h = lib.handle()
    n, k, p, seed = 300, 16, 8, 4
    A = torch.from_numpy(_spd(n, np.linspace(1.0, 0.2, 12), 6)).cuda()
    prm = lib.make_params(k, p, 0, seed, lib.RSVD_F64, lib.RSVD_FLAG_SYNC)
    U = torch.empty(n, k, dtype=torch.float64, device="cuda")
    L = torch.empty(k, dtype=torch.float64, device="cuda")
    ws = torch.empty(lib.rsvd_workspace_size(h, n, n, prm), dtype=torch.uint8, device="cuda")
    assert lib.rsvd_nystrom(h, n, A, n, prm, U, k, L, ws) == lib.RSVD_E_BREAKDOWN


def test_nystrom_argument_errors(lib):
    import torch
    h = lib.handle()
    A = torch.eye(64, dtype=torch.float32, device="cuda")
    U = torch.empty(64, 8, device="cuda")
    L = torch.empty(8, dtype=torch.float64, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    for kw, code in [(dict(q=1), lib.RSVD_E_UNSUPPORTED), (dict(prec=lib.RSVD_MIXED_BF16), lib.RSVD_E_UNSUPPORTED)]:
        prm = lib.make_params(8, 4, kw.get("q", 0), 1, kw.get("prec", lib.RSVD_F32), lib.RSVD_FLAG_SYNC)
        assert lib.rsvd_nystrom(h, 64, A, 64, prm, U, 8, L, ws) == code
    prm = lib.make_params(8, 60, 0, 1, lib.RSVD_F32, lib.RSVD_FLAG_SYNC)  # l = 68 > n
    assert lib.rsvd_nystrom(h, 64, A, 64, prm, U, 8, L, ws) == lib.RSVD_E_INVALID
