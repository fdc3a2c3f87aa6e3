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
