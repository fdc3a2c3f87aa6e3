"""FP8 (e4m3) sketch products, float64 reference.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

The paper samples with a Gaussian test matrix in whatever arithmetic is at
hand (Sec. 4, Fig. RSVD; Sec. 8.1); the FP8 sketch is a reading of that step
for a GPU whose tensor cores take 8-bit operands.  This module states exactly
what such a sketch computes, so that the CUDA product can be compared with it
element by element:

* e4m3 is the 8-bit format with 1 sign bit, 4 exponent bits (bias 7) and 3
  mantissa bits, no infinities, the all-ones pattern (S.1111.111) as NaN:
  normal values 2^(e - 7) (1 + m / 8) for e = 1..15 (m <= 6 when e = 15),
  subnormals 2^-6 (m / 8); largest finite value 448.
* Conversion rounds to the nearest value, ties to the even mantissa, and
  saturates finite values beyond 448 to +-448.
* A is scaled per row: r_i = 448 / max_j |A_ij| (binary32 division; 1 for a
  zero row), A8 = e4m3(binary32(A_ij r_i)), s_i = 1 / r_i, so A ~ diag(s) A8.
  (A scale per row is one instance of a diagonal row scaling A = S A8; a row
  fits in on-chip memory, so one pass over A finds the scale and converts.)
  With block=b the maximum is taken over the b rows of i's block (rows
  b floor(i / b) .. + b - 1), one scale for the whole block: the
  per-128-row-block scaling, block=128.
* A thin operand X (K x N) is scaled per column the same way:
  X ~ X8 diag(c), c_j = 1 / (448 / max_i |X_ij|).
* Y = A X is computed as diag(s) (A8 X8) diag(c); the products of two e4m3
  values are exact, so the only rounding left is in the accumulation.
* A^T Q is computed as A8^T (S Q): Q' = binary32(s_i Q_ij) is scaled per column
  and converted, Z = (A8^T Q'8) diag(c').
"""
import numpy as np

E4M3_MAX = 448.0


def e4m3_values():
    """All 127 non-negative finite e4m3 values, ascending, with their codes."""
    vals, codes = [], []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue  # NaN
            v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
            vals.append(v)
            codes.append((e << 3) | m)
    order = np.argsort(vals, kind="stable")
    return np.array(vals)[order], np.array(codes)[order]


_VALS, _CODES = e4m3_values()


def e4m3_decode(code):
    """Value of an 8-bit e4m3 code (uint8 array); NaN for S.1111.111."""
    code = np.asarray(code, dtype=np.uint8).astype(np.int64)
    s = np.where(code & 0x80, -1.0, 1.0)
    e = (code >> 3) & 0xF
    m = code & 0x7
    v = np.where(e == 0, (m / 8.0) * 2.0 ** -6, (1.0 + m / 8.0) * 2.0 ** (e - 7.0))
    v = np.where((e == 15) & (m == 7), np.nan, v)
    return s * v


def e4m3_round(x):
    """Round float64/float32 values to e4m3 (nearest, ties to even mantissa,
    saturating finite values at +-448); returns the rounded values as float64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    i = np.clip(np.searchsorted(_VALS, a), 1, len(_VALS) - 1)  # _VALS[i-1] < a <= _VALS[i]
    lo, hi = _VALS[i - 1], _VALS[i]
    dlo, dhi = a - lo, hi - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((_CODES[i] & 1) == 0))
    r = np.where(pick_hi, hi, lo)
    r = np.where(a == 0.0, 0.0, r)
    out = np.sign(x) * r
    return np.where(np.isnan(x), np.nan, out)


def row_scale(A, block=None):
    """r_i = 448 / max |A| in binary32 (1 for a zero maximum); returns (r, s = 1/r).
    block=None: the maximum of row i; block=b: the maximum over the b rows of
    i's block (rows b floor(i / b) .. + b - 1, all columns), one scale for the
    whole block."""
    A = np.asarray(A, dtype=np.float32)
    amax = np.max(np.abs(A), axis=1).astype(np.float32)
    if block is not None:
        for b0 in range(0, A.shape[0], block):
            amax[b0:b0 + block] = np.max(amax[b0:b0 + block])
    r = np.where(amax > 0, np.float32(E4M3_MAX) / np.where(amax > 0, amax, np.float32(1)), np.float32(1))
    r = r.astype(np.float32)
    return r, (np.float32(1) / r).astype(np.float32)


def quantize_rows(A, block=None):
    """(A8 values as float64, s) with A ~ diag(s) A8 (per-row scales, or one
    scale per block of `block` rows)."""
    A = np.asarray(A, dtype=np.float32)
    r, s = row_scale(A, block)
    return e4m3_round((A * r[:, None]).astype(np.float32)), s


def quantize_cols(X):
    """(X8 values as float64, c) with X ~ X8 diag(c)."""
    X8t, c = quantize_rows(np.asarray(X, dtype=np.float32).T)
    return X8t.T, c


def sketch_fp8(A, X, block=None):
    """Y = diag(s) (A8 X8) diag(c) in float64 (the exact value the e4m3
    tensor-core product approximates with binary32 accumulation)."""
    A8, s = quantize_rows(A, block)
    X8, c = quantize_cols(X)
    return (s.astype(np.float64)[:, None] * (A8 @ X8)) * c.astype(np.float64)[None, :]


def sketch_fp8_t(A, Q, block=None):
    """Z = A8^T Q'8 diag(c'), Q' = binary32(s_i Q_ij) (the transposed sketch)."""
    A8, s = quantize_rows(A, block)
    Qs = (np.asarray(Q, dtype=np.float32) * s[:, None]).astype(np.float32)
    Q8, c = quantize_cols(Qs)
    return (A8.T @ Q8) * c.astype(np.float64)[None, :]
