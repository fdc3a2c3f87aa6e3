"""Counter-based Gaussian test matrices for the oracle.

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The paper only says ``G = randn(n, k+p)`` (Sec. 4, Fig. RSVD; Sec. 8,
Fig. "Accuracy enhanced randomized SVD (with orthonormalization)") and
draws further Gaussian blocks in Fig. "greedy_blocked" (Sec. 12.3) and
Fig. "adaptive2" (Sec. 13).  It fixes neither a generator nor a layout, so this
project reads ``randn`` as:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a 4x32-bit counter, a 2x32-bit key, ten rounds of two
  32x32->64 multiplies with the multipliers 0xD2511F53 and 0xCD9E8D57, and a
  Weyl key schedule with increments 0x9E3779B9 and 0xBB67AE85.
* Key = (seed mod 2^32, seed div 2^32).
* Entry (i, j) of an n x l test matrix comes from counter
  (i div 4, col0 + j, stream, 0); its four output words w0..w3 feed two
  Box-Muller pairs, (w0, w1) -> rows 4g, 4g+1 and (w2, w3) -> rows 4g+2, 4g+3.
  So the first l' columns of a wider draw equal a narrower draw (prefix
  property), and so do the first n' rows.
* Uniforms carry 24 bits: v = w >> 8, u1 = (v + 1) 2^-24 in (0, 1],
  u2 = v 2^-24 in [0, 1); z_even = sqrt(-2 ln u1) cos(2 pi u2),
  z_odd = sqrt(-2 ln u1) sin(2 pi u2).  Both uniforms are exact in binary32,
  so a binary32 consumer and this binary64 reference start from the same
  numbers.

The oracle computes the Box-Muller step in float64.
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

# Random streams used by the method.  Each stream is an independent counter
# space, so blocks drawn for different purposes never overlap.
STREAM_SKETCH = 0       # Omega of the fixed-rank path (and the 16-column probe)
STREAM_ADAPTIVE = 1     # G blocks of the blocked adaptive range finder
STREAM_CERTIFY = 2      # thin G of the a-posteriori certificate
STREAM_ADAPTIVE2 = 3    # g_j of the vector-at-a-time adaptive range finder
STREAM_NORM = 4         # start block of the spectral-norm estimator
STREAM_ROW = 5          # G_r (row-space sketch) of the single-pass SVD
STREAM_SRFT_D = 6       # phases of the SRFT's diagonal D
STREAM_SRFT_S = 7       # sort keys that draw the SRFT's column subset S


def philox4x32_10(counters, key):
    """Apply ten Philox4x32 rounds to each row of ``counters`` ((N, 4) uint32).

    ``key`` is a pair of 32-bit integers.  Returns an (N, 4) uint32 array.
    """
    c = np.asarray(counters, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0 = np.uint64(int(key[0]) & MASK32)
    k1 = np.uint64(int(key[1]) & MASK32)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    mask = np.uint64(MASK32)
    s32 = np.uint64(32)
    for _ in range(10):
        p0 = m0 * c0          # exact: both factors < 2^32
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(PHILOX_W0)) & mask
        k1 = (k1 + np.uint64(PHILOX_W1)) & mask
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & MASK32, seed >> 32)


def omega_words(n_groups, l, seed, stream=0, col0=0):
    """Raw Philox words for counters (g, col0 + j, stream, 0).

    Returns an array of shape (l, n_groups, 4): [j, g, w].
    """
    g = np.arange(n_groups, dtype=np.uint64)
    ctr = np.zeros((l, n_groups, 4), dtype=np.uint64)
    ctr[:, :, 0] = g[None, :]
    ctr[:, :, 1] = (np.arange(l, dtype=np.uint64) + np.uint64(col0))[:, None]
    ctr[:, :, 2] = np.uint64(stream)
    out = philox4x32_10(ctr.reshape(-1, 4), seed_key(seed))
    return out.reshape(l, n_groups, 4)


def box_muller(w_a, w_b):
    """Two uint32 words -> two standard normals (float64), 24-bit uniforms."""
    va = (np.asarray(w_a, dtype=np.uint64) >> np.uint64(8)).astype(np.float64)
    vb = (np.asarray(w_b, dtype=np.uint64) >> np.uint64(8)).astype(np.float64)
    u1 = (va + 1.0) * 2.0 ** -24
    u2 = vb * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    return r * np.cos(th), r * np.sin(th)


def gaussian(n, l, seed, stream=0, col0=0):
    """n x l Gaussian test matrix (float64) under the counter layout above."""
    if n == 0 or l == 0:
        return np.zeros((n, l))
    ng = (n + 3) // 4
    w = omega_words(ng, l, seed, stream, col0)          # (l, ng, 4)
    z0, z1 = box_muller(w[:, :, 0], w[:, :, 1])
    z2, z3 = box_muller(w[:, :, 2], w[:, :, 3])
    cols = np.stack([z0, z1, z2, z3], axis=2).reshape(l, 4 * ng)  # rows 4g+r
    return np.ascontiguousarray(cols[:, :n].T)
