"""tcgen05 tensor-core sketch products and the mixed-precision solve (GPU).

The bf16 products are compared with the float64 product of the same bf16
values: each bf16 x bf16 product is exact in fp32, so the only error is fp32
accumulation, bounded by 2 K u32 sum |a||x| (u32 = 2^-24)."""
import numpy as np
import pytest

import oracle
from workloads import lowrank_np, poly_spectrum

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _bf16_pair(rng, shape, scale=1.0):
    import torch
    x = torch.from_numpy(rng.standard_normal(shape) * scale).to(torch.float32).to(torch.bfloat16)
    return x.cuda(), x.float().numpy().astype(np.float64)


def _pad8(t):
    """Copy into a buffer whose row stride is a multiple of 8 elements (TMA)."""
    import torch
    r, c = t.shape
    c8 = (c + 7) // 8 * 8
    buf = torch.zeros(r, c8, dtype=t.dtype, device=t.device)
    buf[:, :c] = t
    return buf[:, :c]


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("m,n,l", [(128, 64, 16), (1000, 777, 64), (300, 5000, 256), (4097, 130, 200),
                                   (129, 65, 30), (256, 20000, 128), (20000, 256, 96), (1, 8, 8)])
def test_tc_sketch_parity(lib, trans, m, n, l):
    rng = np.random.default_rng(m + 3 * n + l)
    A, A64 = _bf16_pair(rng, (m, n))
    X, X64 = _bf16_pair(rng, ((m if trans else n), l))
    A, X = _pad8(A), _pad8(X)
    Y = lib.sketch(A, X, trans=trans, prec=lib.RSVD_MIXED_BF16).cpu().numpy().astype(np.float64)
    Aop = A64.T if trans else A64
    ref = Aop @ X64
    K = Aop.shape[1]
    bound = 2 * K * U32 * (np.abs(Aop) @ np.abs(X64)) + 1e-30
    assert Y.shape == ref.shape
    assert np.all(np.abs(Y - ref) <= bound), float(np.max(np.abs(Y - ref) / bound))


def test_tc_sketch_deterministic(lib):
    rng = np.random.default_rng(5)
    A, _ = _bf16_pair(rng, (512, 30000))
    X, _ = _bf16_pair(rng, (512, 256))
    y1 = lib.sketch(A, X, trans=True, prec=lib.RSVD_MIXED_BF16)
    y2 = lib.sketch(A, X, trans=True, prec=lib.RSVD_MIXED_BF16)
    assert bool((y1 == y2).all())


@pytest.mark.parametrize("m,n,l", [(700, 300, 64), (3000, 1000, 256), (20000, 513, 128)])
def test_split3_projection(lib, m, n, l):
    """B^T = A^T Q with A, Q split into bf16 pairs: error about 2^-16 of |A|^T|Q|."""
    import torch
    rng = np.random.default_rng(m + n)
    A64 = rng.standard_normal((m, n))
    Q64 = rng.standard_normal((m, l))
    A = torch.from_numpy(A64.astype(np.float32)).cuda()
    Q = torch.from_numpy(Q64.astype(np.float32)).cuda()
    A64 = A.double().cpu().numpy()
    Q64 = Q.double().cpu().numpy()
    Bt = lib.project(A, Q, prec=lib.RSVD_MIXED_BF16).cpu().numpy().astype(np.float64)
    ref = A64.T @ Q64
    mag = np.abs(A64).T @ np.abs(Q64)
    err = np.abs(Bt - ref)
    assert np.all(err <= (3 * 2.0 ** -16 + 2 * m * U32) * mag)
    # and clearly better than a single bf16 product
    assert np.median(err / mag) < 2.0 ** -14


@pytest.mark.parametrize("m,n,k,p,q", [(2000, 1000, 20, 10, 1), (4096, 4096, 200, 56, 2), (6000, 2500, 64, 64, 1)])
def test_mixed_fixed_rank_vs_oracle(lib, m, n, k, p, q):
    """Mixed path: the sketches see bf16(A), so the basis differs from the
    oracle's at about 2^-9; singular values and the reconstruction error stay
    close to the float64 oracle's (second-order effect of the sketch error)."""
    import torch
    A = lowrank_np(m, n, poly_spectrum(min(m, n), 1.5), seed=m * 3 + n).astype(np.float32)
    A64 = A.astype(np.float64)
    seed = 77
    U, D, V = lib.fixed_rank(torch.from_numpy(A).cuda(), k, p, q, seed=seed, prec=lib.RSVD_MIXED_BF16)
    U, D, V = [t.cpu().numpy().astype(np.float64) for t in (U, D, V)]
    ref = oracle.rsvd_power(A64, k, p, q, seed)
    d1 = ref["D"][0]
    tol = 1e-3 * ref["D"] + 16 * U32 * np.sqrt(m) * d1
    assert np.all(np.abs(D - ref["D"]) <= tol), float(np.max(np.abs(D - ref["D"]) / tol))
    err = oracle.fro_residual(A64, U, D, V)
    err_ref = oracle.fro_residual(A64, ref["U"], ref["D"], ref["V"])
    assert err <= 1.01 * err_ref + 16 * U32 * np.sqrt(m) * np.linalg.norm(A64)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-4)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-4)
