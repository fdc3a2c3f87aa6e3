"""Single-pass randomized EVD and SVD (Sec. "Single pass algorithms"), float64.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

Both methods touch each entry of A once: every product with A is a sketch
taken before any basis exists, and the small core matrix C is fitted to the
sketches by least squares instead of being formed as Q* A Q.

Hermitian A (Fig. singlepass_herm), real symmetric here:
  1. G = randn(n, k + p)                        (the Omega stream)
  2. Y = A G
  3. Q = the k dominant left singular vectors of Y
  4. C = the symmetric k x k least-squares solution of C (Q* G) = Q* Y
  5. C = Uhat D Uhat*                           (symmetric EVD)
  6. U = Q Uhat

General A (Fig. singlepass_gen):
  1. G_c = randn(n, k + p) (the Omega stream), G_r = randn(m, k + p) (row stream)
  2. Y_c = A G_c,  Y_r = A* G_r
  3. Q_c, Q_r = the k dominant left singular vectors of Y_c, Y_r
  4. C = the k x k least-squares solution of the joint system
         (G_r* Q_c) C = Y_r* Q_r   and   C (Q_r* G_c) = Q_c* Y_c
  5. C = Uhat D Vhat*
  6. U = Q_c Uhat,  V = Q_r Vhat

Readings where the section leaves a choice:
* "Least squares" minimizes the Frobenius norm of the residual; in the general
  case the two equations enter with equal weight.
* The symmetric fit parametrizes C by its upper triangle (C = sum over i < j
  of c_ij (e_i e_j* + e_j e_i*) plus sum over i of c_ii e_i e_i*) and solves the
  resulting over-determined system as it stands: the definition written out,
  with no closed form substituted for it.
* Real arithmetic (A real, so A* = A^T).
* The EVD keeps its k pairs ordered by decreasing |lambda| (A may be
  indefinite); each u_i (and in the SVD each v_i, u_i with it) is signed so
  that its largest-magnitude entry is positive.
"""
import numpy as np

from .philox import gaussian, STREAM_SKETCH, STREAM_ROW


def dominant_left(Y, k):
    """Step 3 of both figures: the k dominant left singular vectors of Y."""
    U, _, _ = np.linalg.svd(Y, full_matrices=False)
    return U[:, :k]


def _sign_by_largest(X):
    """+-1 per column: the largest-magnitude entry of that column positive."""
    if X.shape[1] == 0:
        return np.ones(0)
    idx = np.argmax(np.abs(X), axis=0)
    s = np.sign(X[idx, np.arange(X.shape[1])])
    s[s == 0] = 1.0
    return s


# The fits below write the least-squares system out in full: k(k+1)/2 or k^2
# unknowns over k l or 2 k l equations.  That is the definition, meant for the
# small cases an oracle serves; past this many matrix entries they refuse.
MAX_SYSTEM_ENTRIES = 1 << 27


def _check_system(rows, cols):
    if rows * cols > MAX_SYSTEM_ENTRIES:
        raise ValueError("least-squares system of %d x %d entries is beyond the oracle's "
                         "small-case limit" % (rows, cols))


def symmetric_lsq(M, N):
    """argmin over symmetric C (k x k) of ||C M - N||_F, M and N k x l."""
    k = M.shape[0]
    pairs = [(i, j) for i in range(k) for j in range(i, k)]
    _check_system(N.size, len(pairs))
    K = np.zeros((N.size, len(pairs)))
    for t, (i, j) in enumerate(pairs):
        E = np.zeros((k, k))
        E[i, j] = 1.0
        E[j, i] = 1.0
        K[:, t] = (E @ M).ravel()
    x, *_ = np.linalg.lstsq(K, N.ravel(), rcond=None)
    C = np.zeros((k, k))
    for t, (i, j) in enumerate(pairs):
        C[i, j] = x[t]
        C[j, i] = x[t]
    return C


def joint_lsq(P, R1, M, R2):
    """argmin over C (k x k) of ||P C - R1||_F^2 + ||C M - R2||_F^2."""
    k = P.shape[1]
    _check_system(P.shape[0] * k + M.shape[1] * k, k * k)
    # column-major vec: vec(P C) = (I kron P) vec(C), vec(C M) = (M^T kron I) vec(C)
    K = np.vstack([np.kron(np.eye(k), P), np.kron(M.T, np.eye(k))])
    rhs = np.concatenate([R1.ravel(order="F"), R2.ravel(order="F")])
    x, *_ = np.linalg.lstsq(K, rhs, rcond=None)
    return x.reshape(k, k, order="F")


def singlepass_evd(A, k, p, seed):
    """Fig. singlepass_herm for a real symmetric n x n A: returns U (n x k), D (k)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    G = gaussian(n, k + p, seed, STREAM_SKETCH)
    Y = A @ G
    Q = dominant_left(Y, k)
    M = Q.T @ G
    N = Q.T @ Y
    C = symmetric_lsq(M, N)
    lam, Uh = np.linalg.eigh(C)
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, Uh = lam[order], Uh[:, order]
    U = Q @ Uh
    U = U * _sign_by_largest(U)[None, :]
    return dict(U=U, D=lam, Q=Q, C=C, M=M, N=N, G=G, Y=Y)


def singlepass_svd(A, k, p, seed):
    """Fig. singlepass_gen for an m x n A: returns U (m x k), D (k), V (n x k)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    Gc = gaussian(n, l, seed, STREAM_SKETCH)
    Gr = gaussian(m, l, seed, STREAM_ROW)
    Yc = A @ Gc
    Yr = A.T @ Gr
    Qc = dominant_left(Yc, k)
    Qr = dominant_left(Yr, k)
    P, R1 = Gr.T @ Qc, Yr.T @ Qr
    M, R2 = Qr.T @ Gc, Qc.T @ Yc
    C = joint_lsq(P, R1, M, R2)
    Uh, D, Vht = np.linalg.svd(C)
    U, V = Qc @ Uh, Qr @ Vht.T
    s = _sign_by_largest(V)
    U, V = U * s[None, :], V * s[None, :]
    return dict(U=U, D=D, V=V, Qc=Qc, Qr=Qr, C=C, P=P, R1=R1, M=M, R2=R2,
                Gc=Gc, Gr=Gr, Yc=Yc, Yr=Yr)
