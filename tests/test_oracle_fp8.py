"""Pins of the FP8 (e4m3) sketch oracle: the format's values from its
definition, rounding against brute force, ties, saturation, and the scaled
products against exact arithmetic where the operands are representable."""
import numpy as np
import pytest

from oracle import fp8
from oracle import fp8 as OF


def test_e4m3_value_set():
    v, c = fp8.e4m3_values()
    assert len(v) == 127 and len(np.unique(v)) == 127
    assert v[0] == 0.0 and v[1] == 2.0 ** -9 and v[-1] == 448.0
    # normals: 1.0 is code 0x38 (e = 7, m = 0); 1.125 is the next value
    assert c[np.searchsorted(v, 1.0)] == 0x38 and v[np.searchsorted(v, 1.0) + 1] == 1.125
    codes = np.arange(256, dtype=np.uint8)
    d = fp8.e4m3_decode(codes)
    assert np.isnan(d[0x7F]) and np.isnan(d[0xFF]) and np.sum(np.isnan(d)) == 2
    fin = d[~np.isnan(d)]
    assert np.array_equal(np.sort(np.unique(np.abs(fin))), v)
    assert d[0xB8] == -1.0 and d[0x7E] == 448.0 and d[0x01] == 2.0 ** -9


def test_round_trip_and_ties():
    v, c = fp8.e4m3_values()
    assert np.array_equal(fp8.e4m3_round(v), v)
    assert np.array_equal(fp8.e4m3_round(-v[1:]), -v[1:])
    mid = 0.5 * (v[:-1] + v[1:])
    r = fp8.e4m3_round(mid)
    even_hi = (c[1:] & 1) == 0
    assert np.array_equal(r, np.where(even_hi, v[1:], v[:-1]))
    eps = 1e-9 * mid
    assert np.array_equal(fp8.e4m3_round(mid + eps), v[1:])
    assert np.array_equal(fp8.e4m3_round(mid - eps), v[:-1])


def test_saturation_zero_nan():
    assert fp8.e4m3_round(np.array([1e6, -500.0, 460.0, 448.0]))[0] == 448.0
    r = fp8.e4m3_round(np.array([1e6, -500.0, 460.0, -1e30, 0.0, 2.0 ** -11]))
    assert list(r[:4]) == [448.0, -448.0, 448.0, -448.0] and r[4] == 0.0 and r[5] == 0.0
    assert np.isnan(fp8.e4m3_round(np.array([np.nan]))[0])


def test_rounding_matches_brute_force():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.uniform(-4, 3, 5000),
                        rng.uniform(-450, 450, 3000)])
    v, c = fp8.e4m3_values()
    allv = np.concatenate([-v[::-1], v[1:]])
    allc = np.concatenate([c[::-1], c[1:]])
    got = fp8.e4m3_round(x)
    for xi, gi in zip(x, got):
        a = min(max(xi, -448.0), 448.0)
        d = np.abs(allv - a)
        best = np.flatnonzero(d == d.min())
        if len(best) > 1:
            best = [b for b in best if allc[b] % 2 == 0]
        assert gi == allv[best[0]], (xi, gi, allv[best])


def test_scaled_sketch_exact_on_representable_operands():
    rng = np.random.default_rng(1)
    v, _ = fp8.e4m3_values()
    # rows of A on the e4m3 grid with max |.| = 448 (scale 1), X likewise per column
    A = rng.choice(np.concatenate([-v, v]), size=(40, 64)).astype(np.float32)
    A[:, 0] = 448.0
    X = rng.choice(np.concatenate([-v, v]), size=(64, 12)).astype(np.float32)
    X[0, :] = -448.0
    Y = fp8.sketch_fp8(A, X)
    assert np.array_equal(Y, A.astype(np.float64) @ X.astype(np.float64))
    Z = fp8.sketch_fp8_t(A, rng.choice(v, size=(40, 5)).astype(np.float32) * 0 + 448.0)
    assert np.allclose(Z, A.astype(np.float64).T @ np.full((40, 5), 448.0))


def test_scaled_sketch_error_is_fp8_sized():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((300, 200)).astype(np.float32) * np.geomspace(1, 1e-3, 300)[:, None].astype(np.float32)
    X = rng.standard_normal((200, 16)).astype(np.float32)
    Y = fp8.sketch_fp8(A, X)
    ex = A.astype(np.float64) @ X.astype(np.float64)
    # per-row scaling keeps every row's relative error at the e4m3 level: each
    # operand carries up to 2^-4 relative rounding (rms about 2^-4 / sqrt 3),
    # so a product row is off by about sqrt(2) x 3.6% whatever the row's size
    rel = np.linalg.norm(Y - ex, axis=1) / np.linalg.norm(ex, axis=1)
    assert np.all(rel < 0.1) and 0.02 < np.median(rel) < 0.07
    Q = rng.standard_normal((300, 8)).astype(np.float32)
    Z = fp8.sketch_fp8_t(A, Q)
    exz = A.astype(np.float64).T @ Q.astype(np.float64)
    assert np.linalg.norm(Z - exz) / np.linalg.norm(exz) < 0.1


def test_block_scaling_of_rows():
    """Per-block scaling (one scale per 128 rows): every block's largest
    magnitude maps to exactly 448 and nothing exceeds it; a block of one row
    is the per-row scaling; rows that share their maximum within each block
    give the per-row result bit for bit; otherwise the smaller rows of a block
    are quantized on the coarser grid of the block's scale."""
    rng = np.random.default_rng(11)
    A = (rng.standard_normal((300, 70)) * 10.0 ** rng.uniform(-2, 2, (300, 1))).astype(np.float32)
    A8, s = OF.quantize_rows(A, block=128)
    for b0 in range(0, 300, 128):
        blk = A8[b0:b0 + 128]
        assert np.max(np.abs(blk)) == 448.0
        assert np.all(s[b0:b0 + 128] == s[b0])
    one8, one_s = OF.quantize_rows(A, block=1)
    row8, row_s = OF.quantize_rows(A)
    assert np.array_equal(one8, row8) and np.array_equal(one_s, row_s)
    # equal row maxima inside each block: block and row scaling coincide
    B = A.copy()
    B[:, 0] = np.float32(1000.0)
    Bb8, Bbs = OF.quantize_rows(B, block=128)
    Br8, Brs = OF.quantize_rows(B)
    assert np.array_equal(Bb8, Br8) and np.array_equal(Bbs, Brs)
    # with unequal rows the block grid is coarser: larger reconstruction error
    err_b = np.abs(s[:, None] * A8 - A).max(axis=1) / np.abs(A).max(axis=1)
    err_r = np.abs(row_s[:, None] * row8 - A).max(axis=1) / np.abs(A).max(axis=1)
    assert np.mean(err_b) > np.mean(err_r)
    # the sketch with block scales is the exact product of the block-quantized operands
    X = rng.standard_normal((70, 9)).astype(np.float32)
    X8, c = OF.quantize_cols(X)
    ref = (s.astype(np.float64)[:, None] * (A8 @ X8)) * c.astype(np.float64)[None, :]
    np.testing.assert_array_equal(OF.sketch_fp8(A, X, block=128), ref)
