"""Eigenvalue decomposition of a symmetric positive semi-definite matrix by
the Nystrom method, float64.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

Follows Fig. nystrom (Sec. "The Nystrom method for symmetric positive
definite matrices"), step by step:
  1. G = randn(n, k + p)               (the Omega stream of the fixed-rank path)
  2. Y = A G
  3. Q = orth(Y)
  4. B1 = A Q,  B2 = Q* B1
  5. B2 = C* C                         (Cholesky, C upper triangular)
  6. F = B1 C^-1                       (triangular solve)
  7. [U, Sigma, ~] = svd(F, 'econ')
  8. Lambda = Sigma^2
so that A ~ U Lambda U* = F F* = (A Q)(Q* A Q)^-1 (A Q)*.

Readings where the figure leaves a choice:
* B2 is symmetric in exact arithmetic only; it is symmetrized, (B2 + B2*)/2,
  before the Cholesky factorization.
* The output keeps the k leading pairs (the fixed-rank path's convention;
  all k + p with full=True), each u_i signed so that its largest-magnitude
  entry is positive.
"""
import numpy as np

from .philox import gaussian, STREAM_SKETCH
from .rsvd import orth


def nystrom(A, k, p, seed, full=False):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    l = k + p
    G = gaussian(n, l, seed, STREAM_SKETCH)
    Y = A @ G
    Q, _ = orth(Y)
    B1 = A @ Q
    B2 = Q.T @ B1
    B2 = 0.5 * (B2 + B2.T)
    C = np.linalg.cholesky(B2).T           # B2 = C^T C, C upper triangular
    F = np.linalg.solve(C.T, B1.T).T       # F C = B1
    Uf, S, _ = np.linalg.svd(F, full_matrices=False)
    lam = S * S
    if not full:
        Uf, lam = Uf[:, :k], lam[:k]
    if Uf.shape[1]:
        idx = np.argmax(np.abs(Uf), axis=0)
        s = np.sign(Uf[idx, np.arange(Uf.shape[1])])
        s[s == 0] = 1.0
        Uf = Uf * s[None, :]
    return dict(U=Uf, L=lam, Q=Q, B1=B1, B2=B2, C=C, F=F, G=G)
