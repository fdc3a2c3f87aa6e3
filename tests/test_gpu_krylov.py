"""Block Krylov sampling (RSVD_FLAG_KRYLOV; Sec. "Extended sampling matrix")
against the oracle's rsvd_block_krylov on the same seeded input and Gaussian
test matrix.  The oracle forms the blocks [A G, (A A^T) A G, ...] by plain
products, as the section does; the library takes each block from the previous
block's orthonormal basis and projects it against the blocks before it.  Both
span the same space, so U, D and V agree up to rounding."""
import numpy as np
import pytest

import oracle
from workloads import lowrank_np, exp_spectrum, poly_spectrum

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("m,n,k,p,q,rate", [(800, 600, 20, 12, 2, 10.0), (500, 900, 16, 8, 3, 8.0),
                                            (1201, 333, 30, 2, 2, 6.0)])
def test_krylov_f64_matches_oracle(lib, m, n, k, p, q, rate):
    A = lowrank_np(m, n, exp_spectrum(min(m, n), rate), seed=m + n + q)
    seed = 9
    U, D, V = lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=lib.RSVD_F64, krylov=True)
    ref = oracle.rsvd_block_krylov(A, k, p, q, seed)
    D = D.cpu().numpy()
    np.testing.assert_allclose(D, ref["D"], rtol=1e-8, atol=1e-12 * ref["D"][0])
    np.testing.assert_allclose(U.cpu().numpy(), ref["U"], atol=1e-6)
    np.testing.assert_allclose(V.cpu().numpy(), ref["V"], atol=1e-6)


def test_krylov_one_block_is_the_basic_rsvd(lib):
    """q = 1 block is Fig. RSVD: the same launches as the fixed-rank path with
    no power step, bit for bit."""
    A = lowrank_np(700, 500, poly_spectrum(500), seed=3).astype(np.float32)
    a = lib.fixed_rank(_t(A), 24, 8, 1, seed=4, prec=lib.RSVD_F32, krylov=True)
    b = lib.fixed_rank(_t(A), 24, 8, 0, seed=4, prec=lib.RSVD_F32)
    for x, y in zip(a, b):
        assert bool((x == y).all())


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_krylov_binary32_and_mixed(lib, prec):
    """binary32: singular values to the binary32 tolerance (1e-5 relative plus
    the rounding floor 16 u sqrt(m) d_1); bf16 sketches: the Frobenius residual
    within 1% of the oracle's and the leading values to 2e-3 (the subspace is
    that of bf16(A), 2^-9 ||A|| away)."""
    m, n, k, p, q = 3000, 2000, 48, 16, 3
    A = lowrank_np(m, n, poly_spectrum(min(m, n)), seed=12).astype(np.float32)
    A64 = A.astype(np.float64)
    seed = 21
    precs = {"f32": lib.RSVD_F32, "bf16": lib.RSVD_MIXED_BF16}
    U, D, V = lib.fixed_rank(_t(A), k, p, q, seed=seed, prec=precs[prec], krylov=True)
    ref = oracle.rsvd_block_krylov(A64, k, p, q, seed)
    D = D.cpu().numpy()
    Uc, Vc = U.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Uc.T @ Uc - np.eye(k))) < 1e-4 and np.max(np.abs(Vc.T @ Vc - np.eye(k))) < 1e-4
    res = np.linalg.norm(A64 - (Uc * D) @ Vc.T)
    res_ref = np.linalg.norm(A64 - (ref["U"] * ref["D"]) @ ref["V"].T)
    if prec == "f32":
        d1 = ref["D"][0]
        assert np.all(np.abs(D - ref["D"]) <= 1e-5 * ref["D"] + 16 * U32 * np.sqrt(m) * d1)
        assert res <= 1.001 * res_ref
    else:
        np.testing.assert_allclose(D[:10], ref["D"][:10], rtol=2e-3)
        assert res <= 1.01 * res_ref


def test_krylov_arguments(lib):
    import torch
    A = torch.zeros(300, 200, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.RsvdError):       # 3 blocks of 100 columns > min(m, n)
        lib.fixed_rank(A, 90, 10, 3, prec=lib.RSVD_F32, krylov=True)
    with pytest.raises(lib.RsvdError):       # e4m3 sketches have no Krylov mode
        lib.fixed_rank(A, 24, 8, 2, prec=lib.RSVD_MIXED_FP8, krylov=True)
    with pytest.raises(lib.RsvdError):       # bf16 blocks need k + p a multiple of 8
        lib.fixed_rank(A, 20, 5, 2, prec=lib.RSVD_MIXED_BF16, krylov=True)
