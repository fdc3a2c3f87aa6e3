"""Randomized SVD on the extended (block Krylov) sampling matrix (Sec.
"Extended sampling matrix", eq. red), float64.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

Steps, in the section's order:
  1. G = randn(n, k + p)                                   (the Omega stream)
  2. Y = [A G, (A A*) A G, ..., (A A*)^(q-1) A G]          (q blocks, q l columns)
  3. Q = orth(Y)                                           (qr of the section)
  4. B = Q* A,  [Uhat, D, V] = svd(B, 'econ'),  U = Q Uhat
then the k leading triplets are kept (Remark "How many basis vectors").

Readings where the section leaves a choice:
* The section writes the blocks as A^j G, which has a meaning only for a
  square A; for a general A block j is (A A*)^(j-1) A G, the same reading the
  power scheme of Sec. 8.1 takes, and the two agree when A is symmetric.
* The blocks are formed by repeated products with no orthonormalization in
  between, as the section states; the loss of accuracy that the remark after
  Fig. RSVDP describes applies to them as well, so the oracle is meant for
  small q and well-scaled test matrices.
* q counts blocks: q = 1 is Fig. RSVD itself.
"""
import numpy as np

from .philox import gaussian, STREAM_SKETCH
from .rsvd import orth, stage_b, sign_normalize


def krylov_blocks(A, G, q):
    """Step 2: the list [A G, (A A*) A G, ..., (A A*)^(q-1) A G]."""
    blocks = [A @ G]
    for _ in range(q - 1):
        blocks.append(A @ (A.T @ blocks[-1]))
    return blocks


def rsvd_block_krylov(A, k, p, q, seed, full=False):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    if q < 1 or q * l > min(m, n):
        raise ValueError("need q >= 1 and q (k + p) <= min(m, n)")
    G = gaussian(n, l, seed, STREAM_SKETCH)
    Y = np.hstack(krylov_blocks(A, G, q))
    Q, _ = orth(Y)
    U, D, V, B = stage_b(A, Q)
    if not full:
        U, D, V = U[:, :k], D[:k], V[:, :k]
    U, V = sign_normalize(U, V)
    return dict(U=U, D=D, V=V, Q=Q, B=B, Y=Y, G=G)
