"""The seeded input generators shared by the oracle side and the GPU side,
checked against the recipe they state: Haar factors (Q00^2 ~ Beta(1/2,
(m - 1) / 2) and a symmetric sign, which a missing diagonal-sign fix breaks),
exact spectra, column centring, the kernel-block geometry, the controller
stream's sizes and spectra, and the torch builders reproducing the numpy ones
on the CPU."""
import numpy as np
import pytest
from scipy import stats

import workloads as W


def test_haar_factors_are_haar():
    m, r = 40, 3
    q00 = []
    for seed in range(600):
        Q = W.haar_np(np.random.default_rng(seed), m, r)
        if seed < 5:
            assert np.allclose(Q.T @ Q, np.eye(r), atol=1e-13)
        q00.append(Q[0, 0])
    q00 = np.array(q00)
    # the first column is uniform on the sphere: its first entry squared is Beta(1/2, (m-1)/2)
    assert stats.kstest(q00 ** 2, stats.beta(0.5, (m - 1) / 2.0).cdf).pvalue > 1e-3
    # and symmetric in sign (QR without the sign fix gives one sign only)
    assert 0.42 < np.mean(q00 > 0) < 0.58


def test_lowrank_and_named_spectra():
    s = np.array([3.0, 1.0, 0.5, 1e-3])
    A = W.lowrank_np(60, 40, s, seed=1)
    assert np.allclose(np.linalg.svd(A, compute_uv=False)[:4], s, atol=1e-13)
    assert np.allclose(W.exp_spectrum(5), np.exp(-np.arange(1, 6) / 10.0))
    assert np.allclose(W.poly_spectrum(4, 2.0), [1.0, 0.25, 1 / 9.0, 1 / 16.0])
    assert np.array_equal(W.step_spectrum(5, 2), [1.0, 1.0, 1e-6, 1e-6, 1e-6])
    P = W.poly_decay_matrix_np(80, 60, seed=3)
    assert P.dtype == np.float32
    assert np.allclose(np.linalg.svd(P.astype(np.float64), compute_uv=False), W.poly_spectrum(60), atol=1e-6)
    E = W.exp_decay_matrix(200, 100, seed=4)
    assert np.allclose(np.linalg.svd(E, compute_uv=False), W.exp_spectrum(100), atol=1e-13)
    R = W.exact_rank_matrix(50, 40, 7, seed=5, cond=10.0)
    sv = np.linalg.svd(R, compute_uv=False)
    assert np.allclose(sv[:7], np.geomspace(1.0, 0.1, 7), atol=1e-13) and sv[7] < 1e-13


def test_spd_and_pca_families():
    S = W.spd_matrix_np(100, seed=6)
    assert np.array_equal(S, S.T)
    assert np.allclose(np.linalg.eigvalsh(S)[::-1], W.poly_spectrum(100), atol=1e-13)
    m, n = 4096, 256
    A = W.pca_matrix_np(m, n, seed=7).astype(np.float64)
    assert np.abs(A.mean(axis=0)).max() < 1e-6
    sv = np.linalg.svd(A, compute_uv=False)
    # the rank-64 signal 100 -> 1, moved by the centring and by the 1e-3 noise
    assert np.allclose(sv[:48], np.linspace(100.0, 1.0, 64)[:48], rtol=2e-3)
    assert sv[64] < 1e-3 * (np.sqrt(m) + np.sqrt(n)) * 1.1


def test_kernel_blocks_geometry():
    shapes = W.kernel_block_shapes(64, seed=11)
    assert len(set(W.block_seed(11, b) for b in range(4096))) == 4096
    for b in (0, 1, 37):
        x, y = W.kernel_block_points(b, seed=11)
        A = W.kernel_block(b, seed=11)
        assert A.shape == shapes[b] == (len(x), len(y))
        assert 64 <= A.shape[0] <= 1024 and 64 <= A.shape[1] <= 1024
        assert np.all((x >= 0) & (x < 1)) and np.all((y[:, 0] >= 3) & (y[:, 0] < 4))
        i, j = 5, A.shape[1] - 1
        assert A[i, j] == np.float32(1.0 / np.linalg.norm(x[i] - y[j]))
        # unit cubes 3 apart: distances in [2, sqrt(18)]
        assert A.min() >= 1.0 / np.sqrt(18.0) - 1e-6 and A.max() <= 0.5 + 1e-6
    ms = np.array([s[0] for s in W.kernel_block_shapes(2000, seed=4001)])
    assert stats.kstest((ms - 63.5) / 961.0, "uniform").pvalue > 1e-3


def test_kernel_block_torch_is_bit_identical():
    import torch
    for b in (0, 3):
        A = W.kernel_block(b, seed=4001)
        out = torch.empty(A.shape, dtype=torch.float32)
        W.kernel_block_torch(b, out, seed=4001)
        assert np.array_equal(out.numpy(), A)


def test_controller_stream_cases():
    ns, kinds = [], set()
    for seed in range(400):
        n, sig, kind, par = W.controller_case(seed, 512, 16384)
        assert 512 <= n <= 16384 and len(sig) == n and np.all(np.diff(sig) <= 0)
        kinds.add(kind)
        if kind == "poly":
            assert 0.5 <= par <= 2.0
        else:
            assert 16 <= par <= 256
        ns.append(n)
    assert kinds == set(W.CONTROLLER_KINDS)
    u = (np.log(ns) - np.log(512)) / (np.log(16384) - np.log(512))     # log-uniform sizes
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    C = W.dct_factor_np(np.random.default_rng(1), 37)
    assert np.allclose(C.T @ C, np.eye(37), atol=1e-13)


def test_controller_matrix_np_and_torch_agree():
    import torch
    for seed in (2, 9):
        A, (n, kind, par) = W.controller_matrix_np(seed, lo=64, hi=300)
        _, sig, _, _ = W.controller_case(seed, 64, 300)
        assert np.allclose(np.linalg.svd(A.astype(np.float64), compute_uv=False), sig, atol=1e-6)
        At, meta = W.controller_matrix(seed, lo=64, hi=300, device="cpu")
        assert meta == (n, kind, par) and At.dtype == torch.float32
        assert np.allclose(At.numpy(), A, atol=1e-6)


def test_torch_builders_on_cpu():
    import torch
    A = W.poly_decay_matrix(96, 64, seed=2, device="cpu")
    assert A.dtype == torch.float32 and A.is_contiguous()
    assert np.allclose(np.linalg.svd(A.double().numpy(), compute_uv=False), W.poly_spectrum(64), atol=1e-5)
    S = W.spd_matrix(80, seed=3, device="cpu")
    assert torch.equal(S, S.T)
    assert np.allclose(np.linalg.eigvalsh(S.double().numpy())[::-1], W.poly_spectrum(80), atol=1e-5)
    P = W.pca_matrix(2048, 128, seed=4, device="cpu")
    assert float(P.double().mean(dim=0).abs().max()) < 1e-5
    sv = np.linalg.svd(P.double().numpy(), compute_uv=False)
    assert np.allclose(sv[:40], np.linspace(100.0, 1.0, 64)[:40], rtol=3e-3)


def test_mlp_init_layout():
    th = W.mlp_init(7)
    d, h, o = 17, 128, 20
    assert th.shape == (d * h + h + h * h + h + o * h + o,)
    W1 = th[:d * h]
    b1 = th[d * h:d * h + h]
    assert np.all(b1 == 0) and np.all(th[-o:] == 0)
    assert abs(W1.std() / np.sqrt(2.0 / d) - 1.0) < 0.1
