"""Pins for the oracle's fixed-rank randomized SVD against what the paper and
the mathematics fix (no pin re-types the oracle's own formula)."""
import numpy as np
import pytest

import oracle
from workloads import lowrank_np, exact_rank_matrix, exp_spectrum, poly_spectrum, exp_decay_matrix


def mgs_orth(Y):
    """Modified Gram-Schmidt in plain loops (textbook, independent of LAPACK)."""
    Y = np.array(Y, dtype=np.float64)
    m, l = Y.shape
    Q = np.zeros((m, l))
    R = np.zeros((l, l))
    for j in range(l):
        v = Y[:, j].copy()
        for i in range(j):
            R[i, j] = Q[:, i] @ v
            v -= R[i, j] * Q[:, i]
        # second pass (reorthogonalization) so the brute-force reference is tight
        for i in range(j):
            c = Q[:, i] @ v
            R[i, j] += c
            v -= c * Q[:, i]
        R[j, j] = np.linalg.norm(v)
        Q[:, j] = v / R[j, j]
    return Q, R


def test_orth_matches_gram_schmidt_and_is_unique():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((60, 12)) @ np.diag(np.geomspace(1, 1e-3, 12))
    Q, R = oracle.orth(Y)
    Qg, Rg = mgs_orth(Y)
    np.testing.assert_allclose(Q, Qg, atol=1e-10)
    np.testing.assert_allclose(R, Rg, atol=1e-10)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    np.testing.assert_allclose(Q @ R, Y, atol=1e-13)


def test_exact_recovery_of_rank_k_matrix():
    """Sec. 4: if A has exact rank k, k samples span its range (w.p. 1)."""
    for (m, n, k, p) in [(120, 80, 15, 5), (80, 120, 10, 0), (200, 50, 20, 10)]:
        A = exact_rank_matrix(m, n, k, seed=m + n)
        for q in (0, 1):
            r = oracle.rsvd_power(A, k, p, q, seed=3)
            err = np.linalg.norm(A - (r["U"] * r["D"]) @ r["V"].T)
            assert err <= 1e-12 * np.linalg.norm(A), (m, n, k, p, q, err)


def test_full_width_sketch_gives_exact_svd():
    """l = min(m, n): Q spans everything, so Stage B returns the exact SVD."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 25))
    r = oracle.rsvd_power(A, 25, 0, 1, seed=5)
    # singular values by brute force: square roots of eigenvalues of A^T A
    ev = np.sqrt(np.clip(np.sort(np.linalg.eigvalsh(A.T @ A))[::-1], 0, None))
    np.testing.assert_allclose(r["D"], ev, rtol=1e-10)
    np.testing.assert_allclose((r["U"] * r["D"]) @ r["V"].T, A, atol=1e-12)
    np.testing.assert_allclose(r["U"].T @ r["U"], np.eye(25), atol=1e-12)
    np.testing.assert_allclose(r["V"].T @ r["V"], np.eye(25), atol=1e-12)


def test_stage_b_identity_and_interlacing():
    """Remark 3.1: ||A - U D V*|| = ||A - Q Q* A||; Remark 3.2: |sigma_i - d_i| <= eps,
    with 0 <= sigma_i - d_i (d_i are singular values of Q*A, a compression of A)."""
    A = lowrank_np(150, 100, poly_spectrum(100, 1.0), seed=4)
    sig = np.linalg.svd(A, compute_uv=False)
    for q in (0, 1, 2):
        r = oracle.rsvd_power(A, 12, 6, q, seed=7, full=True)
        Q = r["Q"]
        P = A - Q @ (Q.T @ A)
        R = A - (r["U"] * r["D"]) @ r["V"].T
        assert abs(np.linalg.norm(R, 2) - np.linalg.norm(P, 2)) <= 1e-12 * np.linalg.norm(A, 2)
        assert abs(np.linalg.norm(R) - np.linalg.norm(P)) <= 1e-12 * np.linalg.norm(A)
        eps = np.linalg.norm(P, 2)
        d = r["D"]
        diff = sig[:len(d)] - d
        assert np.all(diff >= -1e-13) and np.all(diff <= eps + 1e-13)


def test_eckart_young_lower_bounds():
    """eq. (minerrors): no rank-j approximation beats sigma_{j+1} (2-norm) or the
    Frobenius tail."""
    A = lowrank_np(120, 90, exp_spectrum(90, 6.0), seed=8)
    sig = np.linalg.svd(A, compute_uv=False)
    for (k, p, q) in [(10, 5, 0), (10, 5, 1), (20, 0, 0)]:
        r = oracle.rsvd_power(A, k, p, q, seed=2)
        R = A - (r["U"] * r["D"]) @ r["V"].T
        assert np.linalg.norm(R, 2) >= sig[k] * (1 - 1e-12)
        assert np.linalg.norm(R) >= np.sqrt(np.sum(sig[k:] ** 2)) * (1 - 1e-12)


def test_bound_helpers_match_paper_special_cases():
    """Special cases the paper states in words: p = k + 1 puts the Frobenius bound
    within sqrt(2) of optimal (Sec. 7.1); for a flat tail the power bound reduces
    to [1 + sqrt(k/(p-1)) + e sqrt(k+p)/p sqrt(min(m,n) - k)]^(1/(2q+1)) sigma_{k+1}
    (Sec. 8.2)."""
    k, N = 20, 300
    s = np.concatenate([np.linspace(10, 2, k), np.full(N - k, 0.3)])
    b = oracle.theorem_bounds(s, k, k + 1)
    tail = np.sqrt(np.sum(s[k:] ** 2))
    assert abs(b["fro_mean"] / tail - np.sqrt(2.0)) < 1e-12
    for q in (0, 1, 2, 3):
        p = 7
        b = oracle.theorem_bounds(s, k, p, q)
        flat = (1 + np.sqrt(k / (p - 1)) + np.e * np.sqrt(k + p) / p * np.sqrt(N - k)) ** (1.0 / (2 * q + 1)) * 0.3
        assert abs(b["power_mean"] - flat) <= 1e-12 * flat
    # q = 0 power bound equals the q = 0 spectral expectation bound
    b = oracle.theorem_bounds(s, k, 7, 0)
    assert abs(b["power_mean"] - b["spec_mean"]) <= 1e-12 * b["spec_mean"]


@pytest.mark.parametrize("q", [0, 1, 2])
def test_expectation_bounds_over_seeds(q):
    """Theorem 7.1 (q = 0, Frobenius and spectral) and eq. (averageerrorpower)."""
    m, n, k, p = 200, 150, 10, 6
    A = lowrank_np(m, n, poly_spectrum(150, 0.6), seed=21)
    sig = np.linalg.svd(A, compute_uv=False)
    b = oracle.theorem_bounds(sig, k, p, q)
    fro, spec = [], []
    for s in range(64):
        r = oracle.rsvd_power(A, k, p, q, seed=100 + s, full=True)
        P = A - r["Q"] @ (r["Q"].T @ A)
        fro.append(np.linalg.norm(P))
        spec.append(np.linalg.norm(P, 2))
    if q == 0:
        assert np.mean(fro) <= b["fro_mean"]
        assert np.mean(spec) <= b["spec_mean"]
    assert np.mean(spec) <= b["power_mean"]
    # and never below the optimum
    assert min(spec) >= sig[k + p] * (1 - 1e-12)


def test_tail_bound_every_seed():
    """eq. (8:tailbound): holds except with probability <= 3 e^-p (p >= 4)."""
    m, n, k, p = 120, 100, 8, 8
    A = lowrank_np(m, n, poly_spectrum(100, 0.5), seed=31)
    sig = np.linalg.svd(A, compute_uv=False)
    bound = oracle.theorem_bounds(sig, k, p)["spec_tail"]
    for s in range(200):
        r = oracle.rsvd_basic(A, k, p, seed=500 + s, full=True)
        P = A - r["Q"] @ (r["Q"].T @ A)
        assert np.linalg.norm(P, 2) <= bound


def test_power_scheme_closed_form():
    """Sec. 8.1: A^(q) = (A A*)^q A = U D^(2q+1) V*; the unstabilized scheme's
    sample space equals orth(U D^(2q+1) V* G)."""
    A = lowrank_np(80, 60, np.geomspace(1, 0.2, 60), seed=12)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    for q in (1, 2):
        Aq = (U * s ** (2 * q + 1)) @ Vt
        r = oracle.rsvd_power_plain(A, 8, 4, q, seed=4, full=True)
        Qref, _ = oracle.orth(Aq @ r["G"])
        np.testing.assert_allclose(np.abs(Qref.T @ r["Q"]), np.eye(12), atol=1e-8)


def test_roundoff_ablation_stabilized_vs_plain():
    """Remark after Fig. RSVDP: without orth between products, information for
    sigma_j / sigma_1 <= eps_mach^(1/(2q+1)) is lost; Fig. RSVDP_stabilized keeps it."""
    m, n = 300, 200
    s = np.geomspace(1.0, 1e-14, 200)
    A = lowrank_np(m, n, s, seed=13)
    # eps^(1/7) ~ 5.8e-3 while sigma_81 ~ 2.5e-6: the plain scheme cannot see
    # the singular directions between them
    k, p, q = 80, 10, 3
    st = oracle.rsvd_power(A, k, p, q, seed=1)
    pl = oracle.rsvd_power_plain(A, k, p, q, seed=1)
    e_st = np.linalg.norm(A - (st["U"] * st["D"]) @ st["V"].T, 2)
    e_pl = np.linalg.norm(A - (pl["U"] * pl["D"]) @ pl["V"].T, 2)
    assert e_st <= 10 * s[k]
    assert e_pl >= 100 * e_st


def test_rsvd_power_intermediates_are_orthonormal_and_consistent():
    A = exp_decay_matrix(300, 200, seed=5)
    r = oracle.rsvd_power(A, 20, 10, 2, seed=1001)
    for Q in r["Qs"] + r["Ws"]:
        np.testing.assert_allclose(Q.T @ Q, np.eye(30), atol=1e-12)
    # each Q spans A W (and the first spans A G)
    Ys = [A @ r["G"]] + [A @ W for W in r["Ws"]]
    for Y, Q in zip(Ys, r["Qs"]):
        np.testing.assert_allclose(Q @ (Q.T @ Y), Y, atol=1e-10 * np.linalg.norm(Y))
    np.testing.assert_allclose(r["B"], r["Q"].T @ A, atol=1e-12)


def test_spectral_residual_estimator_matches_direct_norm():
    A = lowrank_np(90, 70, poly_spectrum(70, 1.0), seed=14)
    r = oracle.rsvd_power(A, 6, 4, 0, seed=2)
    est, change = oracle.spectral_residual(A, r["U"], r["D"], r["V"], iters=60)
    direct = np.linalg.norm(A - (r["U"] * r["D"]) @ r["V"].T, 2)
    assert abs(est - direct) <= 1e-6 * direct
    fro = oracle.fro_residual(A, r["U"], r["D"], r["V"], block=17)
    assert abs(fro - np.linalg.norm(A - (r["U"] * r["D"]) @ r["V"].T)) <= 1e-12 * fro
