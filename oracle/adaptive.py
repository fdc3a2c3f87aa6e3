"""Adaptive-rank range finders, float64.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

* ``adaptive_blocked``   Sec. 12.3, Fig. "greedy_blocked": draw an n x b
  Gaussian block, Q_new = qr(A G), B_new = Q_new* A, append, A <- A - Q_new B_new,
  until ||A||_Fro <= eps.  The optional power variant is the one in that
  figure's caption, with orth between products.  The residual norm is
  computed directly from the updated A; the Sec. 12.4 downdate
  sqrt(a^2 - ||B_j||_Fro^2) is recorded beside it as a cross-check.
* ``single_vector_range_finder``  Sec. 13, Fig. "singlevecrangefinder".
* ``adaptive_range_finder``  Sec. 13, Fig. "adaptive2" with the threshold
  eps / (10 sqrt(2/pi)) and an r-vector window.
* ``adaptive_blocked_spectral``  the blocked scheme with Fig. adaptive2's
  spectral-norm stopping test applied to each fresh block (its b samples are
  the test's r = b probes).

Readings taken where the paper is silent:
* the relative tolerance: eps = tol * ||A||_Fro;
* the step follows Fig. greedy_blocked with one deflation, A_j <- A_j -
  Q_new B_new, and one addition: before qr(A_j G) the sample is projected
  against the current Q, (I - Q Q*) A_j G, as Fig. adaptive2 does with its
  own samples.  In exact arithmetic A_j G already lies in the orthogonal
  complement of Q, so this changes only round-off; without it the float64
  basis loses orthogonality (1e-10 at tol = 1e-6: near the end A_j is small
  and its sample carries rounding components along Q of relative size
  u ||A|| / ||A_j||).  (A binary32 implementation also deflates twice: there
  a CholeskyQR2 block is orthonormal only to about 1e-6, and a single
  deflation leaves that much of A_j inside span(Q_new), hidden from every
  later sample by the projection.);
* Gaussian blocks come from STREAM_ADAPTIVE, block t holding columns
  t b .. t b + b - 1 of that stream;
* the loop stops with converged=False at max_rank or min(m, n).
"""
import numpy as np

from .philox import gaussian, STREAM_ADAPTIVE, STREAM_ADAPTIVE2
from .rsvd import orth, sign_normalize


def adaptive_blocked(A, tol, b=16, seed=0, q=0, max_rank=None):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    rmax = min(m, n) if max_rank is None else min(max_rank, m, n)
    Aj = A.copy()
    a2 = float(np.sum(A * A))
    eps = tol * np.sqrt(a2)
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    norms_direct = [np.sqrt(a2)]
    norms_downdate = [np.sqrt(a2)]
    t = 0
    converged = norms_direct[-1] <= eps
    while not converged and Q.shape[1] < rmax:
        bb = min(b, rmax - Q.shape[1])
        G = gaussian(n, bb, seed, STREAM_ADAPTIVE, col0=t * b)
        Y = Aj @ G
        for _ in range(q):
            Y, _ = orth(Y)
            Z, _ = orth(Aj.T @ Y)
            Y = Aj @ Z
        Y = Y - Q @ (Q.T @ Y)
        Qn, _ = orth(Y)
        Bn = Qn.T @ Aj
        Aj = Aj - Qn @ Bn
        Q = np.hstack([Q, Qn])
        B = np.vstack([B, Bn])
        nd = float(np.sqrt(np.sum(Aj * Aj)))
        norms_direct.append(nd)
        norms_downdate.append(float(np.sqrt(max(a2 - np.sum(B * B), 0.0))))
        converged = nd <= eps
        t += 1
    Uhat, D, Vt = np.linalg.svd(B, full_matrices=False)
    U, V = sign_normalize(Q @ Uhat, Vt.T)
    return dict(Q=Q, B=B, U=U, D=D, V=V, rank=Q.shape[1], converged=converged,
                norms_direct=np.array(norms_direct), norms_downdate=np.array(norms_downdate),
                eps=eps, steps=t)


def adaptive_blocked_spectral(A, eps, b=16, seed=0, max_rank=None):
    """The blocked scheme of Fig. greedy_blocked (q = 0) stopped by the
    spectral-norm test of Fig. adaptive2 and Lemma thm:aposteriori instead of
    the Frobenius norm: at the start of step t the fresh block G_t (drawn
    independently of the current Q) gives Y = A_j G_t = (I - Q Q*) A G_t; if
    every column of Y has norm at most eps / (10 sqrt(2/pi)), then
    ||A - Q B||_2 <= eps except with probability 10^-b, and the step stops
    without appending; otherwise the step goes on exactly as in
    adaptive_blocked with the same block.  eps is absolute."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    rmax = min(m, n) if max_rank is None else min(max_rank, m, n)
    thresh = eps / (10.0 * np.sqrt(2.0 / np.pi))
    Aj = A.copy()
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    probes = []
    t = 0
    converged = False
    while Q.shape[1] < rmax:
        bb = min(b, rmax - Q.shape[1])
        G = gaussian(n, bb, seed, STREAM_ADAPTIVE, col0=t * b)
        Y = Aj @ G
        probes.append(float(np.max(np.linalg.norm(Y, axis=0))))
        if probes[-1] <= thresh:
            converged = True
            break
        Y = Y - Q @ (Q.T @ Y)
        Qn, _ = orth(Y)
        Bn = Qn.T @ Aj
        Aj = Aj - Qn @ Bn
        Q = np.hstack([Q, Qn])
        B = np.vstack([B, Bn])
        t += 1
    Uhat, D, Vt = np.linalg.svd(B, full_matrices=False)
    U, V = sign_normalize(Q @ Uhat, Vt.T)
    return dict(Q=Q, B=B, U=U, D=D, V=V, rank=Q.shape[1], converged=converged,
                probes=np.array(probes), thresh=thresh, steps=t)


def truncate_to_tol(D, resid_fro, tol_abs):
    """Smallest r with resid^2 + sum_{i>r} d_i^2 <= tol_abs^2 (Stage-B truncation
    of an adaptive result; Eckart-Young, eq. (minerrors))."""
    D = np.asarray(D, dtype=np.float64)
    tail = np.concatenate([np.cumsum((D ** 2)[::-1])[::-1], [0.0]])  # tail[r] = sum_{i>=r} d_i^2
    for r in range(len(D) + 1):
        if resid_fro ** 2 + tail[r] <= tol_abs ** 2:
            return r
    return len(D)


def single_vector_range_finder(A, steps, seed, stream=STREAM_ADAPTIVE2):
    """Fig. singlevecrangefinder: q_j from (I - Q Q*) A g_j, one vector at a time."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    G = gaussian(n, steps, seed, stream)
    Q = np.zeros((m, 0))
    Bs = []
    for j in range(steps):
        y = A @ G[:, j]
        z = y - Q @ (Q.T @ y)
        qj = z / np.linalg.norm(z)
        Q = np.hstack([Q, qj[:, None]])
        Bs.append(qj @ A)
    return Q, np.array(Bs), G


def adaptive_range_finder(A, eps, r=10, seed=0, max_rank=None):
    """Fig. adaptive2 (Sec. 13).  Returns Q (m x j) and the number of draws."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    rmax = min(m, n) if max_rank is None else min(max_rank, m, n)
    thresh = eps / (10.0 * np.sqrt(2.0 / np.pi))
    # columns of the STREAM_ADAPTIVE2 stream, drawn on demand: g_1 .. g_r first
    G = gaussian(n, r, seed, STREAM_ADAPTIVE2, col0=0)
    ys = [A @ G[:, i] for i in range(r)]          # ys[i] holds y_{i+1}
    Q = np.zeros((m, 0))
    j = 0
    while max(np.linalg.norm(ys[i]) for i in range(j, j + r)) > thresh and j < rmax:
        j += 1
        yj = ys[j - 1]
        yj = yj - Q @ (Q.T @ yj)
        qj = yj / np.linalg.norm(yj)
        Q = np.hstack([Q, qj[:, None]])
        g = gaussian(n, 1, seed, STREAM_ADAPTIVE2, col0=j + r - 1)[:, 0]
        y = A @ g
        ys.append(y - Q @ (Q.T @ y))
        for i in range(j, j + r - 1):
            ys[i] = ys[i] - qj * (qj @ ys[i])
    return Q, j + r
