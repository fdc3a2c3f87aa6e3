"""Pins of the single-pass oracles (Sec. "Single pass algorithms", Figs.
singlepass_herm and singlepass_gen) by facts other than their own code: exact
recovery of rank-k inputs (where Q Q* A = A, the fitted C equals Q* A Q), the
stationarity conditions of both least-squares fits solved in closed form as
Sylvester equations, the ordering of the constrained, symmetrized and free
fits, and the loss of accuracy against two passes that the section remarks on."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import gaussian, rsvd_basic, STREAM_SKETCH
from oracle.philox import STREAM_ROW
from oracle.singlepass import singlepass_evd, singlepass_svd


def _sym_rank_k(n, lam, seed):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((n, len(lam))))
    return (V * lam[None, :]) @ V.T


def _decaying(m, n, seed, power=2.0):
    rng = np.random.default_rng(seed)
    r = min(m, n)
    sig = 1.0 / (1.0 + np.arange(r)) ** power
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return (U * sig[None, :]) @ V.T, sig


def test_evd_exact_on_rank_k_indefinite():
    n, k, p = 120, 10, 10
    lam = np.array([5.0, -4.0, 3.0, -2.5, 2.0, 1.5, -1.2, 1.0, 0.8, -0.5])
    A = _sym_rank_k(n, lam, 0)
    r = singlepass_evd(A, k, p, seed=1)
    assert np.allclose((r["U"] * r["D"][None, :]) @ r["U"].T, A, atol=1e-12)
    assert np.allclose(r["D"], lam, rtol=1e-10)              # ordered by |lambda|
    assert np.allclose(r["U"].T @ r["U"], np.eye(k), atol=1e-12)
    # with Q Q* A = A the one-pass fit is the two-pass core Q* A Q
    assert np.allclose(r["C"], r["Q"].T @ A @ r["Q"], atol=1e-12)
    idx = np.argmax(np.abs(r["U"]), axis=0)
    assert np.all(r["U"][idx, np.arange(k)] > 0)


def test_symmetric_fit_is_the_constrained_minimizer():
    """d/dC ||C M - N||^2 over symmetric C vanishes iff
    C (M M*) + (M M*) C = N M* + M N*, a Lyapunov equation solved here by
    scipy's Bartels-Stewart routine."""
    n, k, p = 90, 8, 8
    A = _sym_rank_k(n, np.linspace(3.0, 0.5, 8), 2)
    E = np.random.default_rng(3).standard_normal((n, n))
    A = A + 1e-3 * 0.5 * (E + E.T)
    r = singlepass_evd(A, k, p, seed=4)
    M, N, C = r["M"], r["N"], r["C"]
    S = M @ M.T
    C_ref = sla.solve_sylvester(S, S, N @ M.T + M @ N.T)
    assert np.array_equal(C, C.T)
    assert np.allclose(C, C_ref, rtol=1e-9, atol=1e-12)
    # free fit <= constrained fit <= symmetrized free fit
    Cu = N @ np.linalg.pinv(M)
    res = lambda X: np.linalg.norm(X @ M - N)
    assert res(Cu) <= res(C) <= res(0.5 * (Cu + Cu.T))


def test_svd_exact_on_rank_k():
    m, n, k, p = 150, 100, 10, 10
    rng = np.random.default_rng(5)
    U0, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, k)))
    s0 = np.linspace(3.0, 0.5, k)
    A = (U0 * s0[None, :]) @ V0.T
    r = singlepass_svd(A, k, p, seed=3)
    assert np.allclose((r["U"] * r["D"][None, :]) @ r["V"].T, A, atol=1e-12)
    assert np.allclose(r["D"], s0, rtol=1e-12)
    assert np.allclose(r["C"], r["Qc"].T @ A @ r["Qr"], atol=1e-12)
    assert np.allclose(r["U"].T @ r["U"], np.eye(k), atol=1e-12)
    assert np.allclose(r["V"].T @ r["V"], np.eye(k), atol=1e-12)


def test_joint_fit_is_the_least_squares_solution():
    """The joint fit's normal equations, P*P C + C M M* = P* R1 + R2 M*, solved
    as a Sylvester equation, on an input that is not exactly low rank."""
    A, _ = _decaying(110, 80, 6, power=1.0)
    r = singlepass_svd(A, 9, 9, seed=7)
    P, R1, M, R2 = r["P"], r["R1"], r["M"], r["R2"]
    C_ref = sla.solve_sylvester(P.T @ P, M @ M.T, P.T @ R1 + R2 @ M.T)
    assert np.allclose(r["C"], C_ref, rtol=1e-9, atol=1e-12)


def test_two_sketches_are_independent_streams():
    r = singlepass_svd(np.eye(40, 30), 4, 4, seed=9)
    assert np.array_equal(r["Gc"], gaussian(30, 8, 9, STREAM_SKETCH))
    assert np.array_equal(r["Gr"], gaussian(40, 8, 9, STREAM_ROW))
    assert not np.allclose(r["Gr"][:30], r["Gc"])


@pytest.mark.parametrize("kind", ["svd", "evd"])
def test_one_pass_loses_accuracy_against_two(kind):
    """Remark "Loss of accuracy": on a fast-decaying spectrum the one-pass
    error exceeds the two-pass error at the same k and p = k, yet stays a small
    multiple of sigma_{k+1}."""
    m, n, k = 150, 100, 10
    if kind == "svd":
        A, sig = _decaying(m, n, 8)
    else:
        A, sig = _decaying(n, n, 8)
        A = 0.5 * (A + A.T)
        sig = np.sort(np.abs(np.linalg.eigvalsh(A)))[::-1]
    one, two = [], []
    for seed in range(6):
        if kind == "svd":
            r = singlepass_svd(A, k, k, seed)
            E1 = A - (r["U"] * r["D"][None, :]) @ r["V"].T
        else:
            r = singlepass_evd(A, k, k, seed)
            E1 = A - (r["U"] * r["D"][None, :]) @ r["U"].T
        b = rsvd_basic(A, k, k, seed)
        one.append(np.linalg.norm(E1, 2))
        two.append(np.linalg.norm(A - (b["U"] * b["D"][None, :]) @ b["V"].T, 2))
    one, two = np.array(one), np.array(two)
    assert np.mean(one) > 1.2 * np.mean(two)
    assert np.all(two >= sig[k] * (1 - 1e-12))
    assert np.all(one < 10.0 * sig[k])


def test_fits_refuse_systems_beyond_small_cases():
    from oracle.singlepass import joint_lsq, symmetric_lsq
    k, l = 200, 400
    with pytest.raises(ValueError):
        joint_lsq(np.zeros((l, k)), np.zeros((l, k)), np.zeros((k, l)), np.zeros((k, l)))
    with pytest.raises(ValueError):
        symmetric_lsq(np.zeros((k, 3 * l)), np.zeros((k, 3 * l)))
