"""Single-pass SVD and EVD (RSVD_FLAG_SINGLE_PASS; Sec. "Single pass
algorithms", Figs. singlepass_gen and singlepass_herm) against the oracle's
singlepass_svd / singlepass_evd on the same seeded inputs and Gaussian
matrices (Gc the Omega stream, Gr Philox stream 5).  The oracle solves the
least-squares fits as written (the full over-determined system); the library
solves their normal equations (Sylvester / Lyapunov) in binary64, which has
the same unique solution."""
import numpy as np
import pytest

import oracle
from workloads import lowrank_np, exp_spectrum, haar_np

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _sym_indefinite(n, rank, seed):
    rng = np.random.default_rng(seed)
    V = haar_np(rng, n, rank)
    lam = np.exp(-np.arange(rank) / 6.0) * np.where(np.arange(rank) % 3 == 1, -1.0, 1.0)
    A = (V * lam[None, :]) @ V.T
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("m,n,k,p,rate", [(600, 400, 20, 20, 5.0), (350, 700, 16, 24, 4.0), (1000, 1000, 40, 40, 8.0)])
def test_single_pass_svd_f64_matches_oracle(lib, m, n, k, p, rate):
    A = lowrank_np(m, n, exp_spectrum(min(m, n), rate), seed=m + 2 * n)
    seed = 13
    U, D, V = lib.fixed_rank(_t(A), k, p, 0, seed=seed, prec=lib.RSVD_F64, single_pass=True)
    ref = oracle.singlepass_svd(A, k, p, seed)
    D = D.cpu().numpy()
    np.testing.assert_allclose(D, ref["D"], rtol=1e-9, atol=1e-12 * ref["D"][0])
    np.testing.assert_allclose(U.cpu().numpy(), ref["U"], atol=1e-7)
    np.testing.assert_allclose(V.cpu().numpy(), ref["V"], atol=1e-7)


@pytest.mark.parametrize("n,k,p", [(400, 20, 20), (700, 30, 30)])
def test_single_pass_evd_f64_matches_oracle(lib, n, k, p):
    A = _sym_indefinite(n, 60, seed=n + k)
    seed = 19
    U, D, V = lib.fixed_rank(_t(A), k, p, 0, seed=seed, prec=lib.RSVD_F64, single_pass=True, symmetric=True)
    ref = oracle.singlepass_evd(A, k, p, seed)
    D = D.cpu().numpy()
    np.testing.assert_allclose(D, ref["D"], rtol=1e-9, atol=1e-12 * abs(ref["D"][0]))
    assert np.any(D < 0)                            # indefinite: signed eigenvalues
    np.testing.assert_allclose(U.cpu().numpy(), ref["U"], atol=1e-7)
    assert bool((U == V).all())


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_single_pass_svd_binary32_and_mixed(lib, prec):
    """binary32: the fitted core inherits the sketches' rounding (binary32
    products over n terms) amplified by the fit's conditioning, so the values
    agree with the oracle to 1e-4 of d_1; bf16 sketches carry 2^-9 relative
    rounding into the fit, so the values agree to 1e-2 of d_1 and the
    Frobenius residual stays within 10% of the oracle's."""
    m, n, k, p = 3000, 2000, 32, 32
    A = lowrank_np(m, n, exp_spectrum(min(m, n), 10.0), seed=17).astype(np.float32)
    A64 = A.astype(np.float64)
    seed = 27
    precs = {"f32": lib.RSVD_F32, "bf16": lib.RSVD_MIXED_BF16}
    U, D, V = lib.fixed_rank(_t(A), k, p, 0, seed=seed, prec=precs[prec], single_pass=True)
    ref = oracle.singlepass_svd(A64, k, p, seed)
    D = D.cpu().numpy()
    d1 = ref["D"][0]
    tol = {"f32": 1e-4, "bf16": 1e-2}[prec]
    assert np.max(np.abs(D - ref["D"])) <= tol * d1, float(np.max(np.abs(D - ref["D"])) / d1)
    Uc, Vc = U.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
    res = np.linalg.norm(A64 - (Uc * D) @ Vc.T)
    res_ref = np.linalg.norm(A64 - (ref["U"] * ref["D"]) @ ref["V"].T)
    assert res <= {"f32": 1.001, "bf16": 1.1}[prec] * res_ref, (res, res_ref)


def test_single_pass_arguments(lib):
    import torch
    A = torch.zeros(300, 200, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.RsvdError):       # power steps do not exist in one pass
        lib.fixed_rank(A, 10, 10, 1, prec=lib.RSVD_F32, single_pass=True)
    with pytest.raises(lib.RsvdError):       # the symmetric variant needs a square A
        lib.fixed_rank(A, 10, 10, 0, prec=lib.RSVD_F32, single_pass=True, symmetric=True)
