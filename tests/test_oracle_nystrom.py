"""Pins of the Nystrom oracle (Fig. nystrom) by facts other than its own
formulas: exact recovery when rank(A) = k + p, the Loewner order
F F* <= A (the Nystrom approximation is a Schur-complement lower bound), the
closed form A - F F* = A^1/2 (I - P) A^1/2 with P the projector onto
range(A^1/2 Q), and the explicit-inverse form (A Q)(Q* A Q)^-1 (A Q)*."""
import numpy as np
import pytest

from oracle import gaussian, STREAM_SKETCH
from oracle.nystrom import nystrom


def _spd(n, lam, seed):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((n, len(lam))))
    return (V * lam[None, :]) @ V.T, V


def test_exact_recovery_when_rank_equals_l():
    n, k, p = 200, 20, 10
    lam = np.linspace(1.0, 0.1, k + p)
    A, V = _spd(n, lam, 1)
    r = nystrom(A, k, p, seed=3, full=True)
    assert np.allclose(r["F"] @ r["F"].T, A, atol=1e-12)
    assert np.allclose(r["L"], lam, rtol=1e-10)
    rk = nystrom(A, k, p, seed=3)
    assert np.allclose(rk["L"], lam[:k], rtol=1e-10)
    U = rk["U"]
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-12)
    assert np.allclose(A @ U, U * rk["L"][None, :], atol=1e-11)
    # sign convention: the largest-magnitude entry of each u_i is positive
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(k)] > 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_loewner_order_and_eigenvalue_bounds(seed):
    n, k, p = 150, 10, 5
    lam = np.exp(-np.arange(n) / 12.0)
    A, _ = _spd(n, lam, 10 + seed)
    r = nystrom(A, k, p, seed=seed, full=True)
    E = A - r["F"] @ r["F"].T
    assert np.linalg.eigvalsh(0.5 * (E + E.T)).min() > -1e-12
    # hence each Nystrom eigenvalue lies below the matching eigenvalue of A
    assert np.all(r["L"] <= lam[:k + p] * (1 + 1e-10) + 1e-14)


def test_closed_form_residual_and_explicit_inverse():
    n, k, p = 120, 8, 6
    lam = 1.0 / (1.0 + np.arange(n)) ** 2
    A, _ = _spd(n, lam, 5)
    r = nystrom(A, k, p, seed=7, full=True)
    # A - F F* = A^1/2 (I - P) A^1/2, P the projector onto range(A^1/2 Q)
    w, Vw = np.linalg.eigh(A)
    Ah = (Vw * np.sqrt(np.clip(w, 0, None))[None, :]) @ Vw.T
    M = Ah @ r["Q"]
    Qm, _ = np.linalg.qr(M)
    E_closed = Ah @ (np.eye(n) - Qm @ Qm.T) @ Ah
    assert np.allclose(A - r["F"] @ r["F"].T, E_closed, atol=1e-12)
    # the explicit-inverse form of eq. spd_nystrom
    B1 = A @ r["Q"]
    N = B1 @ np.linalg.inv(r["Q"].T @ B1) @ B1.T
    assert np.allclose(r["F"] @ r["F"].T, N, atol=1e-12)
    # the same Omega as the fixed-rank path
    assert np.array_equal(r["G"], gaussian(n, k + p, 7, STREAM_SKETCH))


def test_nystrom_beats_the_standard_hermitian_form_on_average():
    """The figure's claim (one power step "for free"): over seeds, the
    Nystrom residual is below that of Q (Q* A Q) Q* (eq. spd_standard)."""
    n, k, p = 300, 15, 5
    lam = 1.0 / (1.0 + np.arange(n)) ** 1.5
    A, _ = _spd(n, lam, 9)
    ny, st = [], []
    for seed in range(8):
        r = nystrom(A, k, p, seed=seed, full=True)
        Q = r["Q"]
        ny.append(np.linalg.norm(A - r["F"] @ r["F"].T, 2))
        st.append(np.linalg.norm(A - Q @ (Q.T @ A @ Q) @ Q.T, 2))
    assert np.mean(ny) < 0.5 * np.mean(st)
