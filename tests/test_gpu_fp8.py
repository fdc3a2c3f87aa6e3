"""The e4m3 (FP8) sketch products on tcgen05 tensor cores against the oracle's
exact definition (oracle/fp8.py), and the FP8 fixed-rank solve against the
float64 oracle on a PCA-shaped matrix."""
import numpy as np
import pytest

import oracle
from oracle import fp8 as OF
from workloads import pca_matrix_np

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("block", [None, 128])
@pytest.mark.parametrize("trans,m,n,l", [(0, 1000, 700, 30), (0, 3000, 2100, 128), (0, 600, 5000, 256),
                                         (1, 1000, 700, 30), (1, 2100, 3000, 128), (1, 5000, 600, 256)])
def test_e4m3_sketch_matches_definition(lib, trans, m, n, l, block):
    """Per-row scales (RSVD_MIXED_FP8) and one scale per 128-row block
    (RSVD_MIXED_FP8_B128; 1000 and 2100 rows end in a ragged block)."""
    rng = np.random.default_rng(m + n + l)
    A = (rng.standard_normal((m, n)) * np.geomspace(1, 1e-2, m)[:, None]).astype(np.float32)
    X = rng.standard_normal((m if trans else n, l)).astype(np.float32)
    prec = lib.RSVD_MIXED_FP8 if block is None else lib.RSVD_MIXED_FP8_B128
    Y = lib.sketch(_t(A), _t(X), trans=bool(trans), prec=prec).cpu().numpy().astype(np.float64)
    if trans:
        ref = OF.sketch_fp8_t(A, X, block)
        A8, s = OF.quantize_rows(A, block)
        Q8, c = OF.quantize_cols((X * s[:, None]).astype(np.float32))
        babs = np.abs(A8).T @ np.abs(Q8) * c.astype(np.float64)[None, :]
    else:
        ref = OF.sketch_fp8(A, X, block)
        A8, s = OF.quantize_rows(A, block)
        X8, c = OF.quantize_cols(X)
        babs = (s.astype(np.float64)[:, None] * (np.abs(A8) @ np.abs(X8))) * c.astype(np.float64)[None, :]
    # the products of e4m3 values are exact; only the binary32 accumulation order differs
    K = m if trans else n
    assert np.all(np.abs(Y - ref) <= 4 * np.sqrt(K) * 6e-8 * babs + 1e-30), np.max(np.abs(Y - ref) / (babs + 1e-30))


@pytest.mark.parametrize("block", [None, 128])
def test_e4m3_conversion_is_exact(lib, block):
    """X = the first l columns of the identity picks single columns of A8:
    every converted value of A comes back (scaled), so one byte converted
    differently from the definition would show as a relative error >= 1/16
    (per-row and per-128-row-block scales)."""
    rng = np.random.default_rng(5)
    m, n, l = 777, 400, 64
    A = (rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-3, 3, (m, 1))).astype(np.float32)
    A[3] = 0.0                       # a zero row
    A[5, 7] = 1e-30                  # below e4m3's range after scaling
    X = np.zeros((n, l), dtype=np.float32)
    X[np.arange(l), np.arange(l)] = 1.0
    prec = lib.RSVD_MIXED_FP8 if block is None else lib.RSVD_MIXED_FP8_B128
    Y = lib.sketch(_t(A), _t(X), trans=False, prec=prec).cpu().numpy().astype(np.float64)
    ref = OF.sketch_fp8(A, X, block)
    np.testing.assert_allclose(Y, ref, rtol=3e-7, atol=0)
    assert np.all(Y[3] == 0)


@pytest.mark.parametrize("block", [None, 128])
def test_fp8_fixed_rank_pca(lib, block):
    """PCA-shaped matrix (rank-64 signal, singular values 100 -> 1, noise 1e-3).
    e4m3 rounding perturbs A by about 3.6% of each entry, a matrix of spectral
    norm ~ 0.036 ||A||_F (1/sqrt(n) + 1/sqrt(m)): 0.39 here (0.28 at the
    configuration's 2^20 x 4096), below the noise floor 1e-3 (sqrt(m) + sqrt(n))
    = 0.19 ... 1.09 only at full size, so the test bounds the residual against
    the float64 oracle's and the error of the well-separated singular values."""
    m, n, k, p, q, seed = 16384, 4096, 64, 64, 1, 3
    A = pca_matrix_np(m, n, seed=31)
    A64 = A.astype(np.float64)
    prec = lib.RSVD_MIXED_FP8 if block is None else lib.RSVD_MIXED_FP8_B128
    U, D, V = lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=prec)
    ref = oracle.rsvd_power(A64, k, p, q, seed)
    d = D.cpu().numpy()
    U = U.cpu().numpy().astype(np.float64)
    V = V.cpu().numpy().astype(np.float64)
    rel = np.abs(d - ref["D"]) / ref["D"]
    res = np.linalg.norm(A64 - (U * d) @ V.T)
    res_ref = np.linalg.norm(A64 - (ref["U"] * ref["D"]) @ ref["V"].T)
    Ub, Db, Vb = lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=lib.RSVD_MIXED_BF16)
    rel_b = np.abs(Db.cpu().numpy() - ref["D"]) / ref["D"]
    print("\nFP8: max rel sigma error (top 48) %.2e, residual %.4f vs oracle %.4f; bf16 %.2e"
          % (np.max(rel[:48]), res, res_ref, np.max(rel_b[:48])))
    assert np.max(rel[:48]) < 1e-3
    assert res <= 1.05 * res_ref
    assert np.max(np.abs(U.T @ U - np.eye(k))) < 1e-3 and np.max(np.abs(V.T @ V - np.eye(k))) < 1e-3
