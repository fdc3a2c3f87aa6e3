"""Implicit column centring (RSVD_FLAG_CENTER) against the oracle's
rsvd_power_centred: Fig. RSVDP_stabilized on Abar = A - 1 mu^T with every
product by A or A^T replaced by its rank-one-corrected form, on the same
seeded input and Gaussian test matrix.  The input is a PCA-shaped matrix
(rank-r signal, small noise) with column offsets of the signal's size, so the
uncentred factorization differs visibly from the centred one."""
import numpy as np
import pytest

import oracle
from workloads import haar_np

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _offset_pca(m, n, rank, seed):
    rng = np.random.default_rng(seed)
    U = haar_np(rng, m, rank)
    V = haar_np(rng, n, rank)
    s = np.linspace(10.0, 1.0, rank)
    A = (U * s[None, :]) @ V.T + 1e-4 * rng.standard_normal((m, n))
    scale = np.sqrt(np.mean(A * A))
    A += 2.0 * scale * rng.standard_normal(n)[None, :]        # column offsets
    return A


def _t(x, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x if dtype is None else x.astype(dtype))).to("cuda")


@pytest.mark.parametrize("m,n,k,p,q", [(3000, 500, 20, 10, 1), (700, 1200, 16, 16, 2), (4099, 257, 30, 2, 0)])
def test_centred_f64_matches_oracle(lib, m, n, k, p, q):
    A = _offset_pca(m, n, 40, seed=m + n)
    seed = 11
    U, D, V = lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=lib.RSVD_F64, centre=True)
    ref = oracle.rsvd_power_centred(A, k, p, q, seed)
    D = D.cpu().numpy()
    np.testing.assert_allclose(D, ref["D"], rtol=1e-10, atol=1e-13 * ref["D"][0])
    # well-separated triplets: vectors to 1e-8
    np.testing.assert_allclose(U.cpu().numpy(), ref["U"], atol=1e-8)
    np.testing.assert_allclose(V.cpu().numpy(), ref["V"], atol=1e-8)
    # U is orthogonal to the ones vector (the centred columns are)
    assert np.max(np.abs(U.cpu().numpy().sum(axis=0))) < 1e-9 * np.sqrt(m)
    # and the centring matters on this input
    D0 = lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=lib.RSVD_F64)[1].cpu().numpy()
    assert np.max(np.abs(D0 - ref["D"]) / ref["D"]) > 1e-3


@pytest.mark.parametrize("prec", ["f32", "bf16", "e4m3"])
def test_centred_binary32_and_mixed(lib, prec):
    """The binary32 path to the tolerance stated for it (1e-5 relative plus
    the binary32 rounding floor); the mixed paths, whose sketches see bf16 /
    e4m3 copies of the uncentred A, to the accuracy of their Rayleigh-Ritz
    values on a well-separated spectrum (the projection is split-bf16)."""
    m, n, k, p, q = 4096, 512, 24, 24, 1
    A = _offset_pca(m, n, 32, seed=7).astype(np.float32)
    A64 = A.astype(np.float64)
    seed = 5
    precs = {"f32": lib.RSVD_F32, "bf16": lib.RSVD_MIXED_BF16, "e4m3": lib.RSVD_MIXED_FP8}
    U, D, V = lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=precs[prec], centre=True)
    ref = oracle.rsvd_power_centred(A64, k, p, q, seed)
    D = D.cpu().numpy()
    d1 = ref["D"][0]
    if prec == "f32":
        bound = 1e-5 * ref["D"] + 16 * U32 * np.sqrt(m) * d1
    else:
        bound = 2e-4 * d1 + 0 * ref["D"]
    assert np.all(np.abs(D - ref["D"]) <= bound), float(np.max(np.abs(D - ref["D"]) / d1))
    Uc = U.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Uc.T @ Uc - np.eye(k))) < 1e-4
    # the exact u_i are orthogonal to 1.  What remains of 1 in U is the
    # sketch's rounding along 1, which scales with the uncentred entries:
    # |1^T u_i| / sqrt(m) <= u_sketch ||A||_F / ||Abar||_F (bf16 2^-9, e4m3
    # 2^-4; binary32 products over n terms, sqrt(n) 2^-24)
    Abar = A64 - A64.mean(axis=0, keepdims=True)
    ratio = np.linalg.norm(A64) / np.linalg.norm(Abar)
    u_sk = {"f32": np.sqrt(n) * U32, "bf16": 2.0 ** -9, "e4m3": 2.0 ** -4}[prec]
    assert np.max(np.abs(Uc.sum(axis=0))) / np.sqrt(m) <= u_sk * ratio, float(np.max(np.abs(Uc.sum(axis=0))))
