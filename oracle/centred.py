"""Randomized SVD of the column-centred matrix without forming it, float64.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

The paper names PCA as an application (Sec. 1) without spelling out how the
data are centred.  The centred matrix is Abar = A - 1 mu* with mu the vector
of column means, mu = A* 1 / m.  Forming Abar costs a pass over A and a copy
of it; applying it implicitly costs one rank-1 correction per product:
    Abar X  = A X  - 1 (mu* X)
    Abar* Y = A* Y - mu (1* Y)
This module runs Fig. RSVDP_stabilized (Sec. 8.1), step by step as the
fixed-rank oracle does, with every product by A or A* replaced by the
corrected product; Stage B's B = Q* Abar is one more corrected product.

Every column of Abar is orthogonal to the ones vector (1* Abar = 1* A - m mu*
= 0), so every Q the solve forms lies in that complement and the correction
of Abar* Q, mu (1* Q), vanishes in exact arithmetic: only the forward
correction changes results.  The oracle applies both, as the definition does.
"""
import numpy as np

from .philox import gaussian, STREAM_SKETCH
from .rsvd import orth, sign_normalize


def column_means(A):
    m = A.shape[0]
    return A.T @ np.ones(m) / m


def centred_apply(A, mu, X):
    """Abar X = A X - 1 (mu* X)."""
    return A @ X - np.outer(np.ones(A.shape[0]), mu @ X)


def centred_apply_t(A, mu, Y):
    """Abar* Y = A* Y - mu (1* Y)."""
    return A.T @ Y - np.outer(mu, Y.sum(axis=0))


def rsvd_power_centred(A, k, p, q, seed, full=False):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    mu = column_means(A)
    G = gaussian(n, k + p, seed, STREAM_SKETCH)
    Q, _ = orth(centred_apply(A, mu, G))
    for _ in range(q):
        W, _ = orth(centred_apply_t(A, mu, Q))
        Q, _ = orth(centred_apply(A, mu, W))
    B = centred_apply_t(A, mu, Q).T                         # Q* Abar
    Uh, D, Vt = np.linalg.svd(B, full_matrices=False)
    U, V = Q @ Uh, Vt.T
    if not full:
        U, D, V = U[:, :k], D[:k], V[:, :k]
    U, V = sign_normalize(U, V)
    return dict(U=U, D=D, V=V, Q=Q, B=B, G=G, mu=mu)
