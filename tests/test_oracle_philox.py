"""Pins for the oracle's Gaussian test-matrix generator (the paper's randn)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import philox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _triton_words(counters, seed):
    """Philox4x32-10 from an independent implementation: Triton's tl.philox,
    executed by Triton's CPU interpreter in a child process."""
    code = textwrap.dedent("""
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import numpy as np, torch, triton, triton.language as tl
        @triton.jit
        def k(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
            i = tl.arange(0, N)
            r0, r1, r2, r3 = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i),
                                       tl.load(c2p + i), tl.load(c3p + i))
            tl.store(out + 4 * i, r0); tl.store(out + 4 * i + 1, r1)
            tl.store(out + 4 * i + 2, r2); tl.store(out + 4 * i + 3, r3)
        d = json.loads(sys.stdin.read())
        c = np.array(d["c"], dtype=np.uint32)
        N = c.shape[0]
        cols = [torch.from_numpy(c[:, j].view(np.int32).copy()) for j in range(4)]
        out = torch.zeros(4 * N, dtype=torch.int32)
        k[(1,)](out, *cols, d["seed"], N=N)
        print(json.dumps(out.numpy().view(np.uint32).tolist()))
    """)
    import json
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", code], input=json.dumps({"c": counters.tolist(), "seed": int(seed)}),
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    return np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint32).reshape(-1, 4)


def test_philox_matches_independent_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    N = 64
    c = rng.integers(0, 2 ** 32, size=(N, 4), dtype=np.uint64).astype(np.uint32)
    c[0] = 0
    c[1] = [0xFFFFFFFF] * 4
    for seed in (0, 1234567, (77 << 32) | 99):
        ref = _triton_words(c, seed)
        got = philox.philox4x32_10(c, philox.seed_key(seed))
        np.testing.assert_array_equal(got, ref)


def test_gaussian_moments_and_ks():
    from scipy import stats
    z = philox.gaussian(4096, 256, seed=11).ravel()   # 1,048,576 draws
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(stats.skew(z)) < 5.0 * np.sqrt(6.0 / n)
    assert abs(stats.kurtosis(z)) < 5.0 * np.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert np.all(np.isfinite(z))


def test_gaussian_pairs_uncorrelated_and_each_row_phase_normal():
    from scipy import stats
    G = philox.gaussian(4000, 200, seed=3)
    # rows 4g+r for each r in 0..3 are each N(0,1) (cos and sin branches)
    for r in range(4):
        assert stats.kstest(G[r::4].ravel(), "norm").pvalue > 1e-4
    # the two members of a Box-Muller pair are uncorrelated
    c = np.corrcoef(G[0::4].ravel(), G[1::4].ravel())[0, 1]
    assert abs(c) < 5.0 / np.sqrt(G[0::4].size)
    # neighbouring columns are uncorrelated
    c = np.corrcoef(G[:, :-1].ravel(), G[:, 1:].ravel())[0, 1]
    assert abs(c) < 5.0 / np.sqrt(G.size)


def test_uniform_extremes_are_finite():
    w_max = np.array([0xFFFFFFFF], dtype=np.uint32)
    w_min = np.array([0], dtype=np.uint32)
    for a in (w_min, w_max):
        for b in (w_min, w_max):
            z0, z1 = philox.box_muller(a, b)
            assert np.isfinite(z0).all() and np.isfinite(z1).all()
    # u1 = 1 exactly when the word's top 24 bits are all ones: radius 0
    z0, z1 = philox.box_muller(w_max, w_min)
    assert z0[0] == 0.0 and z1[0] == 0.0


def test_prefix_property_and_offsets():
    G = philox.gaussian(103, 40, seed=9)
    np.testing.assert_array_equal(philox.gaussian(103, 17, seed=9), G[:, :17])
    np.testing.assert_array_equal(philox.gaussian(50, 40, seed=9), G[:50])
    np.testing.assert_array_equal(philox.gaussian(103, 10, seed=9, col0=30), G[:, 30:40])
    assert not np.array_equal(philox.gaussian(103, 40, seed=10), G)


def test_streams_are_distinct():
    a = philox.gaussian(2048, 16, seed=1, stream=0).ravel()
    b = philox.gaussian(2048, 16, seed=1, stream=1).ravel()
    assert abs(np.corrcoef(a, b)[0, 1]) < 5.0 / np.sqrt(a.size)
