"""Subsampled randomized Fourier transform (SRFT) sketch (Sec. "A method with
complexity O(mn log k) for general dense matrices", eq. SRFT), float64 /
complex128.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

Omega = D F S (n x l):
* D: diagonal, entries e^{i theta_j} with theta_j uniform on [0, 2 pi);
* F: the unitary DFT, F(p, q) = n^-1/2 exp(-2 pi i p q / n), p, q = 0 .. n-1;
* S: l distinct columns of the n x n identity, drawn without replacement.
The range finder then runs as in Fig. RSVD with Omega in place of G:
Y = A Omega, Q = orth(Y), B = Q* A, B = Uhat D V*, U = Q Uhat.

Readings where the section leaves a choice:
* The random quantities come from the same counter-based Philox4x32-10
  generator as the Gaussian test matrices (its definition is in philox.py):
  - theta_j = 2 pi (w >> 8) 2^-24, with w word (j mod 4) of counter
    (j div 4, 0, STREAM_SRFT_D, 0);
  - S takes the l indices j with the smallest 64-bit keys
    (w0 << 32) | w1 of counter (j, 0, STREAM_SRFT_S, 0), ties broken by the
    smaller j, in increasing key order.  This is a uniform draw without
    replacement, and the first l' columns of an l-column draw equal the
    l'-column draw (the prefix property of the Gaussian stream).
* Stage B is the two-pass Q* A of Fig. RSVD (the section's other options,
  the single-pass fit and row extraction by an ID, are other rows).
* A real A still gives a complex Y, Q, B, U and V (the singular values D are
  real); all of them stay complex.  Each singular pair is phased so that the
  largest-magnitude entry of v_i is real and positive.
* F is applied as the dense matrix of its definition; the exponent p q is
  reduced mod n in integer arithmetic first, which changes no entry.
"""
import numpy as np

from .philox import philox4x32_10, omega_words, seed_key, STREAM_SRFT_D, STREAM_SRFT_S


def srft_phases(n, seed):
    """theta_0 .. theta_{n-1} of D, in [0, 2 pi)."""
    if n == 0:
        return np.zeros(0)
    ng = (n + 3) // 4
    w = omega_words(ng, 1, seed, STREAM_SRFT_D)[0]           # (ng, 4): [g, word]
    v = (w.reshape(-1)[:n].astype(np.uint64) >> np.uint64(8)).astype(np.float64)
    return 2.0 * np.pi * v * 2.0 ** -24


def srft_subset(n, l, seed):
    """The l column indices of S, in draw order."""
    if l > n:
        raise ValueError("l > n")
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n, dtype=np.uint64)
    ctr[:, 2] = STREAM_SRFT_S
    w = philox4x32_10(ctr, seed_key(seed)).astype(np.uint64)
    keys = (w[:, 0] << np.uint64(32)) | w[:, 1]
    order = np.lexsort((np.arange(n), keys))                  # by key, then index
    return order[:l]


def dft_matrix(n):
    """F(p, q) = n^-1/2 exp(-2 pi i p q / n)."""
    pq = np.outer(np.arange(n, dtype=np.int64), np.arange(n, dtype=np.int64)) % n
    return np.exp(-2j * np.pi * pq / n) / np.sqrt(n)


def srft_omega(n, l, seed):
    """Omega = D F S, n x l complex."""
    d = np.exp(1j * srft_phases(n, seed))
    S = srft_subset(n, l, seed)
    return (d[:, None] * dft_matrix(n))[:, S]


def orth_c(Y):
    """Orthonormal basis of col(Y) (Sec. 2.3) for complex Y: Householder QR,
    each column phased so that diag(R) is real and positive."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    d = np.diag(R)
    s = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * s[None, :], np.conj(s)[:, None] * R


def rsvd_srft(A, k, p, seed, full=False):
    """Fig. RSVD with the SRFT Omega: returns complex U (m x k), real D (k),
    complex V (n x k) with A ~ U diag(D) V*."""
    A = np.asarray(A)
    m, n = A.shape
    l = k + p
    Om = srft_omega(n, l, seed)
    Y = A @ Om
    Q, _ = orth_c(Y)
    B = np.conj(Q.T) @ A
    Uh, D, Vh = np.linalg.svd(B, full_matrices=False)
    U, V = Q @ Uh, np.conj(Vh.T)
    if not full:
        U, D, V = U[:, :k], D[:k], V[:, :k]
    if V.shape[1]:
        idx = np.argmax(np.abs(V), axis=0)
        piv = V[idx, np.arange(V.shape[1])]
        ph = np.conj(piv) / np.abs(piv)
        U, V = U * ph[None, :], V * ph[None, :]
    return dict(U=U, D=D, V=V, Q=Q, B=B, Y=Y, Omega=Om)
