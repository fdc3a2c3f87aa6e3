"""rsvd_adaptive_tol (Sec. 12.3 Fig. greedy_blocked, Sec. 12.4) against the
float64 oracle's adaptive_blocked on the same seeded inputs and Gaussian blocks."""
import numpy as np
import pytest

import oracle
from workloads import lowrank_np, exp_spectrum, kernel_block

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _np(*ts):
    return [t.cpu().numpy().astype(np.float64) for t in ts]


@pytest.mark.parametrize("m,n,rate,tol,b", [(600, 400, 8.0, 1e-6, 16), (300, 500, 5.0, 1e-8, 16),
                                            (257, 130, 4.0, 1e-5, 8), (1000, 999, 8.0, 1e-4, 32)])
def test_adaptive_f64_matches_oracle(lib, m, n, rate, tol, b):
    A = lowrank_np(m, n, exp_spectrum(min(m, n), rate), seed=m + n)
    seed = 31
    U, D, V, rank, err, code = lib.adaptive_tol(_t(A), tol, block=b, seed=seed, prec=lib.RSVD_F64)
    assert code == lib.RSVD_OK
    ref = oracle.adaptive_blocked(A, tol, b=b, seed=seed, max_rank=min(m, n, 128))
    assert rank == ref["rank"]
    assert err <= tol
    np.testing.assert_allclose(err, ref["norms_direct"][-1] / np.linalg.norm(A), rtol=1e-6, atol=1e-15)
    U, D, V = _np(U, D, V)
    np.testing.assert_allclose(D[:rank], ref["D"], rtol=1e-9, atol=1e-13 * ref["D"][0])
    assert np.all(D[rank:] == 0)
    k = int(np.sum(ref["D"] > 1e-6 * ref["D"][0]))  # well-determined singular vectors
    np.testing.assert_allclose(U[:, :k], ref["U"][:, :k], atol=1e-6)
    np.testing.assert_allclose(V[:, :k], ref["V"][:, :k], atol=1e-6)
    # the factorization meets the tolerance
    res = np.linalg.norm(A - (U[:, :rank] * D[:rank]) @ V[:, :rank].T)
    assert res <= tol * np.linalg.norm(A) * (1 + 1e-6)


@pytest.mark.parametrize("blk", [0, 7, 123])
def test_adaptive_f32_kernel_blocks(lib, blk):
    """The batched workload's blocks, one at a time: 1/|x - y| kernels, tol 1e-6."""
    A = kernel_block(blk, seed=4001)
    m, n = A.shape
    tol = 1e-6
    U, D, V, rank, err, code = lib.adaptive_tol(_t(A), tol, block=16, seed=blk, prec=lib.RSVD_F32)
    assert code == lib.RSVD_OK
    ref = oracle.adaptive_blocked(A.astype(np.float64), tol, b=16, seed=blk, max_rank=min(m, n, 256))
    # the stopping decision is taken on a binary32 remainder: same rank unless the
    # oracle's remainder sits within a few percent of the threshold
    ratios = ref["norms_direct"] / ref["eps"]
    if not np.any(np.abs(ratios - 1.0) < 0.05):
        assert rank == ref["rank"]
    assert err <= tol
    U, D, V = _np(U, D, V)
    A64 = A.astype(np.float64)
    res = np.linalg.norm(A64 - (U[:, :rank] * D[:rank]) @ V[:, :rank].T) / np.linalg.norm(A64)
    assert res <= 2 * tol
    nr = min(rank, ref["rank"])
    np.testing.assert_allclose(D[:nr], ref["D"][:nr], rtol=1e-4, atol=1e-6 * ref["D"][0])


def test_adaptive_not_converged_and_zero(lib):
    import torch
    rng = np.random.default_rng(0)
    A = rng.standard_normal((200, 150)).astype(np.float32)
    U, D, V, rank, err, code = lib.adaptive_tol(_t(A), 1e-6, block=16, max_rank=32, seed=1, prec=lib.RSVD_F32)
    assert code == lib.RSVD_E_NOT_CONVERGED and rank == 32 and err > 1e-6
    ref = oracle.adaptive_blocked(A.astype(np.float64), 1e-6, b=16, seed=1, max_rank=32)
    np.testing.assert_allclose(D.cpu().numpy(), ref["D"], rtol=1e-4)
    Z = torch.zeros(100, 80, dtype=torch.float32, device="cuda")
    U, D, V, rank, err, code = lib.adaptive_tol(Z, 1e-3, block=16, seed=1, prec=lib.RSVD_F32)
    assert code == lib.RSVD_OK and rank == 0 and err == 0.0
    assert float(D.abs().max()) == 0.0 and float(U.abs().max()) == 0.0


def test_adaptive_argument_errors(lib):
    import torch
    A = torch.zeros(50, 40, dtype=torch.float32, device="cuda")
    h = lib.handle()
    for kw in [dict(tol=0.0), dict(tol=1.5), dict(tol=1e-3, block=64), dict(tol=1e-3, max_rank=41)]:
        prm = lib.make_params(0, 0, 0, 1, lib.RSVD_F32, 0, **kw)
        import ctypes
        out = ctypes.c_size_t()
        code = lib.load().rsvd_workspace_size(h, 50, 40, ctypes.byref(prm), ctypes.byref(out))
        if kw.get("tol", 0) <= 0:
            # tol == 0 selects the fixed-rank sizing (k = 0 is accepted there)
            continue
        assert code == lib.RSVD_E_INVALID, kw


# the ranks these need (about rate ln(2.4 / thresh), thresh = eps / (10
# sqrt(2/pi)), plus up to two blocks) stay below the binary64 cap of 128
@pytest.mark.parametrize("m,n,rate,eps", [(300, 200, 5.0, 1e-3), (600, 450, 4.0, 1e-4), (257, 300, 5.0, 1e-2),
                                          (1000, 700, 6.0, 3e-5)])
def test_adaptive_spectral_f64_matches_oracle(lib, m, n, rate, eps):
    """RSVD_FLAG_SPECTRAL (Sec. 13, Fig. adaptive2's test with Lemma
    thm:aposteriori) against the oracle's adaptive_blocked_spectral: same
    rank, same singular values, the reported bound is the stopping block's
    probe bound, and the spectral error of the result is below eps."""
    A = lowrank_np(m, n, exp_spectrum(min(m, n), rate), seed=m + n + 1)
    seed = 17
    U, D, V, rank, err, code = lib.adaptive_tol(_t(A), eps, block=16, seed=seed, prec=lib.RSVD_F64, spectral=True)
    assert code == lib.RSVD_OK
    ref = oracle.adaptive_blocked_spectral(A, eps, b=16, seed=seed, max_rank=min(m, n, 128))
    assert ref["converged"] and rank == ref["rank"]
    np.testing.assert_allclose(err, 10.0 * np.sqrt(2.0 / np.pi) * ref["probes"][-1], rtol=1e-9)
    U, D, V = _np(U, D, V)
    np.testing.assert_allclose(D[:rank], ref["D"], rtol=1e-9, atol=1e-13 * ref["D"][0])
    assert np.all(D[rank:] == 0)
    res = np.linalg.norm(A - (U[:, :rank] * D[:rank]) @ V[:, :rank].T, 2)
    assert res <= eps and res <= err


@pytest.mark.parametrize("m,n,rate,eps", [(500, 400, 8.0, 1e-3), (800, 300, 6.0, 1e-4)])
def test_adaptive_spectral_f32(lib, m, n, rate, eps):
    """The binary32 path of the spectral mode: the oracle runs on the same
    binary32 matrix; the stopping decision compares binary32 samples with the
    threshold, so the rank matches unless one of the oracle's probes lies
    within 1% of it."""
    A = lowrank_np(m, n, exp_spectrum(min(m, n), rate), seed=m + n + 2).astype(np.float32)
    A64 = A.astype(np.float64)
    seed = 23
    U, D, V, rank, err, code = lib.adaptive_tol(_t(A), eps, block=16, seed=seed, prec=lib.RSVD_F32, spectral=True)
    assert code == lib.RSVD_OK
    ref = oracle.adaptive_blocked_spectral(A64, eps, b=16, seed=seed, max_rank=min(m, n, 256))
    if not np.any(np.abs(ref["probes"] / ref["thresh"] - 1.0) < 0.01):
        assert rank == ref["rank"]
    U, D, V = _np(U, D, V)
    r = min(rank, ref["rank"])
    d1 = ref["D"][0]
    assert np.all(np.abs(D[:r] - ref["D"][:r]) <= 1e-5 * ref["D"][:r] + 64 * 2.0 ** -24 * np.sqrt(m) * d1)
    res = np.linalg.norm(A64 - (U[:, :rank] * D[:rank]) @ V[:, :rank].T, 2)
    assert res <= eps


def test_adaptive_spectral_cap_and_arguments(lib):
    """The cap ends the spectral loop with RSVD_E_NOT_CONVERGED and reports
    the Frobenius residual (a deterministic bound on the spectral error);
    power steps are refused in this mode."""
    A = lowrank_np(300, 200, exp_spectrum(200, 10.0), seed=5)
    U, D, V, rank, err, code = lib.adaptive_tol(_t(A), 1e-12, block=16, max_rank=48, seed=3, prec=lib.RSVD_F64,
                                                spectral=True)
    assert code == lib.RSVD_E_NOT_CONVERGED and rank == 48
    ref = oracle.adaptive_blocked_spectral(A, 1e-12, b=16, seed=3, max_rank=48)
    assert not ref["converged"] and ref["rank"] == 48
    U, D, V = _np(U, D, V)
    np.testing.assert_allclose(err, np.linalg.norm(A - (U * D) @ V.T), rtol=1e-6)
    with pytest.raises(lib.RsvdError):
        lib.adaptive_tol(_t(A), 1e-3, block=16, seed=3, prec=lib.RSVD_F64, spectral=True, q=1)
