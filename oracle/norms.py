"""Residual norms and the a-posteriori estimators, float64.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

* ``fro_residual``     exact Frobenius norm of A - U D V*, computed blockwise.
* ``spectral_residual`` block power iteration on T = A - U D V* applied
                       implicitly (T x = A x - U (D (V* x))); the spectral norm
                       is the quantity in Remark 3.1 / eq. (8:error_SVD).
* ``certificate``      Sec. 14: E = (A - A_approx) G with a thin Gaussian G,
                       bound (1/alpha) sqrt(2/pi) max_i ||E(:, i)|| (Lemma
                       "thm:aposteriori", Sec. 13), which holds with
                       probability at least 1 - alpha^r.
"""
import numpy as np

from .philox import gaussian, STREAM_CERTIFY, STREAM_NORM


def fro_residual(A, U, D, V, block=4096):
    A = np.asarray(A, dtype=np.float64)
    s = 0.0
    UD = U * D[None, :]
    for r0 in range(0, A.shape[0], block):
        T = A[r0:r0 + block] - UD[r0:r0 + block] @ V.T
        s += float(np.sum(T * T))
    return np.sqrt(s)


def _apply(A, U, D, V, X):
    return A @ X - U @ (D[:, None] * (V.T @ X))


def _apply_t(A, U, D, V, Y):
    return A.T @ Y - V @ (D[:, None] * (U.T @ Y))


def spectral_residual(A, U, D, V, iters=30, block=4, seed=7):
    """Estimate ||A - U D V*||_2 by `iters` block power steps (start block from
    the STREAM_NORM Gaussian stream).  Returns (estimate, last relative change)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    X = gaussian(n, block, seed, STREAM_NORM)
    X, _ = np.linalg.qr(X)
    est, prev = 0.0, 0.0
    for _ in range(iters):
        Y = _apply(A, U, D, V, X)
        est = float(np.linalg.norm(Y, 2))
        Z = _apply_t(A, U, D, V, Y)
        X, _ = np.linalg.qr(Z)
        change = abs(est - prev) / max(est, 1e-300)
        prev = est
    return est, change


def certificate(A, U, D, V, seed, r=10, alpha=0.1):
    """Sec. 14: draw G (n x r, STREAM_CERTIFY), E = (A - U D V*) G.

    Returns (bound, column norms of E).  With alpha = 1/10 and r = 10 the bound
    holds with probability >= 1 - 1e-10.
    """
    A = np.asarray(A, dtype=np.float64)
    G = gaussian(A.shape[1], r, seed, STREAM_CERTIFY)
    E = _apply(A, U, D, V, G)
    cn = np.linalg.norm(E, axis=0)
    return (1.0 / alpha) * np.sqrt(2.0 / np.pi) * float(cn.max()), cn


def theorem_bounds(sigma, k, p, q=0):
    """Right-hand sides of the paper's error bounds for given singular values.

    Returns a dict with
    * ``fro_mean``  eq. (8:expectationbound), q = 0, Frobenius;
    * ``spec_mean`` eq. (expectationboundspectral), q = 0;
    * ``spec_tail`` eq. (8:tailbound), q = 0, p >= 4, failure prob <= 3 e^-p;
    * ``power_mean`` eq. (averageerrorpower) for the given q.
    """
    s = np.asarray(sigma, dtype=np.float64)
    tail = s[k:]
    fro_tail = np.sqrt(np.sum(tail ** 2))
    sk1 = s[k] if len(s) > k else 0.0
    out = {}
    out["fro_mean"] = np.sqrt(1.0 + k / (p - 1.0)) * fro_tail
    out["spec_mean"] = (1.0 + np.sqrt(k / (p - 1.0))) * sk1 + np.e * np.sqrt(k + p) / p * fro_tail
    out["spec_tail"] = (1.0 + 17.0 * np.sqrt(1.0 + k / p)) * sk1 + 8.0 * np.sqrt(k + p) / (p + 1.0) * fro_tail
    e = 2 * q + 1
    out["power_mean"] = ((1.0 + np.sqrt(k / (p - 1.0))) * sk1 ** e
                         + np.e * np.sqrt(k + p) / p * np.sqrt(np.sum(tail ** (2 * e)))) ** (1.0 / e)
    return out
