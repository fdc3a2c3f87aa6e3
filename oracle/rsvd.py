"""Fixed-rank randomized SVD, float64, written from the paper's figures.

TEST INFRASTRUCTURE ONLY: this is the oracle that the CUDA path is checked
against.  Nothing in the product path may import it.

Each function follows one figure of Martinsson, "Randomized methods for matrix
computations" (arXiv:1607.01649):

* ``orth``            Sec. 2.3 (orthonormalization, unpivoted QR).
* ``rsvd_basic``      Sec. 4, Fig. RSVD (basic randomized SVD).
* ``rsvd_power_plain``  Sec. 8.1, Fig. RSVDP (power scheme, no re-orth).
* ``rsvd_power``      Sec. 8.1, Fig. RSVDP_stabilized (orth after every product)
                      -- the path the GPU library implements.

LAPACK (through numpy) serves as the QR and dense-SVD primitives; the steps
around them are the paper's, in its order.
"""
import numpy as np

from .philox import gaussian, STREAM_SKETCH


def orth(Y):
    """Sec. 2.3: orthonormal basis of col(Y), unpivoted.

    Householder QR (LAPACK geqrf/orgqr via numpy), then each column's sign is
    chosen so that diag(R) > 0.  With that sign rule Q is unique whenever Y
    has full column rank, which is what makes stage-by-stage comparison with
    another orthonormalizer (e.g. CholeskyQR) meaningful.
    Returns (Q, R) with Y = Q R.
    """
    Q, R = np.linalg.qr(Y, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def sign_normalize(U, V):
    """Fix each singular pair's sign: the largest-|.| entry of v_i is positive.

    The SVD (Sec. 2.2) determines u_i, v_i only up to a common sign.
    """
    if V.shape[1] == 0:
        return U, V
    idx = np.argmax(np.abs(V), axis=0)
    s = np.sign(V[idx, np.arange(V.shape[1])])
    s[s == 0] = 1.0
    return U * s[None, :], V * s[None, :]


def stage_b(A, Q):
    """Sec. 3, Stage B: B = Q* A, B = Uhat D V*, U = Q Uhat."""
    B = Q.T @ A
    Uhat, D, Vt = np.linalg.svd(B, full_matrices=False)
    U = Q @ Uhat
    return U, D, Vt.T, B


def _finish(U, D, V, k, full):
    """Remark "How many basis vectors": keep the k leading triplets."""
    if not full:
        U, D, V = U[:, :k], D[:k], V[:, :k]
    U, V = sign_normalize(U, V)
    return U, D, V


def rsvd_basic(A, k, p, seed, full=False, stream=STREAM_SKETCH):
    """Fig. RSVD (Sec. 4): G = randn(n, k+p); Y = A G; Q = orth(Y); Stage B."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    G = gaussian(n, k + p, seed, stream)
    Q, _ = orth(A @ G)
    U, D, V, B = stage_b(A, Q)
    U, D, V = _finish(U, D, V, k, full)
    return dict(U=U, D=D, V=V, Q=Q, B=B, G=G)


def rsvd_power_plain(A, k, p, q, seed, full=False):
    """Fig. RSVDP (Sec. 8.1): Y = (A A*)^q A G with no orth between products.

    Kept only as the ablation that shows the round-off loss described in the
    remark after that figure.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    G = gaussian(n, k + p, seed, STREAM_SKETCH)
    Y = A @ G
    for _ in range(q):
        Z = A.T @ Y
        Y = A @ Z
    Q, _ = orth(Y)
    U, D, V, B = stage_b(A, Q)
    U, D, V = _finish(U, D, V, k, full)
    return dict(U=U, D=D, V=V, Q=Q, B=B, G=G)


def rsvd_power(A, k, p, q, seed, full=False):
    """Fig. RSVDP_stabilized (Sec. 8.1), the library's path.

    G = randn(n, k+p); Q = orth(A G);
    q times: W = orth(A* Q), Q = orth(A W);
    B = Q* A; [Uhat, D, V] = svd(B); U = Q Uhat;
    then truncation to k (Remark "How many basis vectors").

    Returns the outputs and every intermediate (Y, W, Q per step, B) so that
    tests can compare stage by stage.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    G = gaussian(n, l, seed, STREAM_SKETCH)
    Y0 = A @ G
    Q, R0 = orth(Y0)
    Qs, Ws, Ys, Zs = [Q], [], [Y0], []
    for _ in range(q):
        Z = A.T @ Q
        W, _ = orth(Z)
        Y = A @ W
        Q, _ = orth(Y)
        Zs.append(Z); Ws.append(W); Ys.append(Y); Qs.append(Q)
    U, D, V, B = stage_b(A, Q)
    U, D, V = _finish(U, D, V, k, full)
    return dict(U=U, D=D, V=V, Q=Q, B=B, G=G, Qs=Qs, Ws=Ws, Ys=Ys, Zs=Zs)
