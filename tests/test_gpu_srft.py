"""The SRFT sketch (RSVD_FLAG_SRFT; Sec. 6, eq. SRFT) against the oracle's
rsvd_srft: the same Omega = D F S from the same Philox words (phases from
stream 6, the column subset from the keys of stream 7), the same complex
factors.  The library forms Omega's real and imaginary parts explicitly and
runs the complex steps on the realification; D, U and V must agree with the
oracle's complex Householder and LAPACK SVD path."""
import numpy as np
import pytest

import oracle
from workloads import lowrank_np, exp_spectrum, poly_spectrum

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("m,n,k,p,rate", [(500, 300, 16, 8, 4.0), (300, 777, 20, 12, 5.0), (1024, 1024, 40, 24, 8.0)])
def test_srft_f64_matches_oracle(lib, m, n, k, p, rate):
    A = lowrank_np(m, n, exp_spectrum(min(m, n), rate), seed=m + 3 * n)
    seed = 41
    U, D, V = lib.fixed_rank(_t(A), k, p, 0, seed=seed, prec=lib.RSVD_F64, srft=True)
    ref = oracle.rsvd_srft(A, k, p, seed)
    D = D.cpu().numpy()
    np.testing.assert_allclose(D, ref["D"], rtol=1e-9, atol=1e-12 * ref["D"][0])
    np.testing.assert_allclose(U.cpu().numpy(), ref["U"], atol=1e-7)
    np.testing.assert_allclose(V.cpu().numpy(), ref["V"], atol=1e-7)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_srft_binary32_and_mixed(lib, prec):
    """binary32: values to 1e-5 relative plus the rounding floor 16 u sqrt(m)
    d_1; bf16 sketch: the subspace of bf16(A) (Rayleigh-Ritz values, second
    order) with the split-bf16 projection, values to 2e-3 relative for the
    leading ten and the Frobenius residual within 1% of the oracle's."""
    m, n, k, p = 3000, 2048, 48, 16
    A = lowrank_np(m, n, poly_spectrum(min(m, n)), seed=33).astype(np.float32)
    A64 = A.astype(np.float64)
    seed = 29
    precs = {"f32": lib.RSVD_F32, "bf16": lib.RSVD_MIXED_BF16}
    U, D, V = lib.fixed_rank(_t(A), k, p, 0, seed=seed, prec=precs[prec], srft=True)
    ref = oracle.rsvd_srft(A64, k, p, seed)
    D = D.cpu().numpy()
    Uc, Vc = U.cpu().numpy().astype(np.complex128), V.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(Uc.conj().T @ Uc - np.eye(k))) < 1e-4
    assert np.max(np.abs(Vc.conj().T @ Vc - np.eye(k))) < 1e-4
    res = np.linalg.norm(A64 - (Uc * D) @ Vc.conj().T)
    res_ref = np.linalg.norm(A64 - (ref["U"] * ref["D"]) @ ref["V"].conj().T)
    if prec == "f32":
        assert np.all(np.abs(D - ref["D"]) <= 1e-5 * ref["D"] + 16 * U32 * np.sqrt(m) * ref["D"][0])
        assert res <= 1.001 * res_ref
    else:
        np.testing.assert_allclose(D[:10], ref["D"][:10], rtol=2e-3)
        assert res <= 1.01 * res_ref


def test_srft_arguments(lib):
    import torch
    A = torch.zeros(300, 200, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.RsvdError):       # Fig. RSVD only: no power steps
        lib.fixed_rank(A, 10, 10, 1, prec=lib.RSVD_F64, srft=True)
    with pytest.raises(lib.RsvdError):       # realified basis 2 (k + p) > 128 in binary64
        lib.fixed_rank(A, 60, 10, 0, prec=lib.RSVD_F64, srft=True)
