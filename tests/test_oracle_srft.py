"""Pins of the SRFT oracle (eq. SRFT): Omega has orthonormal columns (they
are columns of the unitary D F); A Omega equals the subsampled FFT of A D
computed by numpy's FFT; D's phases are uniform and S is a uniform draw
without replacement with the prefix property; the SRFT range finder recovers
rank-k matrices exactly and, on a decaying spectrum, is about as accurate as
the Gaussian one (the section's observation), for n not a power of two."""
import numpy as np
import pytest
from scipy import stats

from oracle import rsvd_basic
from oracle.srft import srft_phases, srft_subset, srft_omega, dft_matrix, rsvd_srft


@pytest.mark.parametrize("n,l", [(300, 40), (64, 64), (97, 5)])
def test_omega_columns_orthonormal(n, l):
    Om = srft_omega(n, l, seed=5)
    assert Om.shape == (n, l)
    assert np.allclose(np.conj(Om.T) @ Om, np.eye(l), atol=1e-12)


def test_dft_matches_numpy_fft_and_sketch_is_a_subsampled_fft():
    n, l = 300, 40
    F = dft_matrix(n)
    assert np.allclose(F, np.fft.fft(np.eye(n), axis=0) / np.sqrt(n), atol=1e-13)
    A = np.random.default_rng(1).standard_normal((50, n))
    d = np.exp(1j * srft_phases(n, 5))
    S = srft_subset(n, l, 5)
    Y_fft = (np.fft.fft(A * d[None, :], axis=1) / np.sqrt(n))[:, S]
    assert np.allclose(A @ srft_omega(n, l, 5), Y_fft, atol=1e-12)


def test_phases_uniform_and_subset_uniform_without_replacement():
    th = srft_phases(1 << 14, seed=1)
    assert th.min() >= 0.0 and th.max() < 2 * np.pi
    assert stats.kstest(th / (2 * np.pi), "uniform").pvalue > 1e-3
    n, l, draws = 64, 8, 2000
    cnt = np.zeros(n)
    for seed in range(draws):
        S = srft_subset(n, l, seed)
        assert len(set(S.tolist())) == l
        cnt[S] += 1
    assert stats.chisquare(cnt).pvalue > 1e-3
    S = srft_subset(500, 60, 3)
    assert np.array_equal(srft_subset(500, 12, 3), S[:12])     # prefix property
    assert not np.array_equal(srft_subset(500, 12, 4), S[:12])
    with pytest.raises(ValueError):
        srft_subset(10, 11, 0)


def test_exact_recovery_of_rank_k():
    m, n, k = 200, 300, 12
    rng = np.random.default_rng(2)
    U0, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, k)))
    s0 = np.linspace(2.0, 0.3, k)
    A = (U0 * s0[None, :]) @ V0.T
    r = rsvd_srft(A, k, k, seed=3)
    assert np.allclose((r["U"] * r["D"][None, :]) @ np.conj(r["V"].T), A, atol=1e-12)
    assert np.allclose(r["D"], s0, rtol=1e-12)
    assert np.allclose(np.conj(r["U"].T) @ r["U"], np.eye(k), atol=1e-12)
    idx = np.argmax(np.abs(r["V"]), axis=0)
    piv = r["V"][idx, np.arange(k)]
    assert np.allclose(piv.imag, 0.0, atol=1e-15) and np.all(piv.real > 0)


def test_accuracy_close_to_gaussian_on_decaying_spectrum():
    m, n, k = 200, 300, 12
    rng = np.random.default_rng(4)
    sig = 1.0 / (1.0 + np.arange(m)) ** 1.5
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, m)))
    A = (U * sig[None, :]) @ V.T
    srft, gauss = [], []
    for seed in range(6):
        r = rsvd_srft(A, k, k, seed)
        srft.append(np.linalg.norm(A - (r["U"] * r["D"][None, :]) @ np.conj(r["V"].T), 2))
        b = rsvd_basic(A, k, k, seed)
        gauss.append(np.linalg.norm(A - (b["U"] * b["D"][None, :]) @ b["V"].T, 2))
    srft = np.array(srft) / sig[k]
    assert np.all(srft >= 1 - 1e-12)                    # never below the optimum
    assert np.mean(srft) < 1.5 * np.mean(np.array(gauss) / sig[k])
