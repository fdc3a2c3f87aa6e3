"""Pins for the oracle's adaptive range finders and a-posteriori estimators."""
import numpy as np

import oracle
from workloads import lowrank_np, exp_spectrum, poly_spectrum, kernel_block


def eps_rank(sig, eps):
    """Brute force: min k with (sum_{j>k} sigma_j^2)^(1/2) <= eps."""
    tail = np.sqrt(np.concatenate([np.cumsum((sig ** 2)[::-1])[::-1], [0.0]]))
    return int(np.argmax(tail <= eps))


def test_blocked_adaptive_frobenius_identity_and_stop():
    """Sec. 12.4: ||A||^2 = ||B_j||^2 + ||A_j||^2 and A = Q_j B_j + A_j;
    Fig. greedy_blocked stops once ||A_j||_Fro <= eps."""
    A = lowrank_np(200, 160, exp_spectrum(160, 8.0), seed=3)
    tol = 1e-6
    r = oracle.adaptive_blocked(A, tol, b=16, seed=5)
    a = np.linalg.norm(A)
    assert r["converged"]
    assert r["norms_direct"][-1] <= tol * a
    # identity holds to round-off at every step (in squares)
    d2 = r["norms_direct"] ** 2 - r["norms_downdate"] ** 2
    assert np.max(np.abs(d2)) <= 1e-12 * a * a
    # A = Q B + A_j and the final residual equals ||A - Q B||
    np.testing.assert_allclose(np.linalg.norm(A - r["Q"] @ r["B"]), r["norms_direct"][-1], rtol=1e-6, atol=1e-14 * a)
    np.testing.assert_allclose(r["Q"].T @ r["Q"], np.eye(r["rank"]), atol=1e-12)
    sig = np.linalg.svd(A, compute_uv=False)
    k_opt = eps_rank(sig, tol * a)
    assert k_opt <= r["rank"] <= k_opt + 2 * 16
    assert r["rank"] % 16 == 0


def test_blocked_adaptive_power_variant_and_kernel_block():
    A = kernel_block(0, seed=4001, lo=64, hi=160).astype(np.float64)
    tol = 1e-6
    for q in (0, 1):
        r = oracle.adaptive_blocked(A, tol, b=16, seed=2, q=q)
        a = np.linalg.norm(A)
        assert r["converged"] and r["norms_direct"][-1] <= tol * a
        sig = np.linalg.svd(A, compute_uv=False)
        assert r["rank"] >= eps_rank(sig, tol * a)
        # Stage B on the adaptive basis: U D V* reproduces Q B
        np.testing.assert_allclose((r["U"] * r["D"]) @ r["V"].T, r["Q"] @ r["B"], atol=1e-12 * a)


def test_blocked_adaptive_not_converged_at_max_rank():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((64, 48))          # noise: no low-rank structure
    r = oracle.adaptive_blocked(A, 1e-6, b=16, seed=1, max_rank=32)
    assert not r["converged"] and r["rank"] == 32


def test_truncate_to_tol_brute_force():
    D = np.array([5.0, 3.0, 1.0, 0.5, 0.1])
    for resid in (0.0, 0.05, 0.3):
        for tol in (0.2, 0.6, 1.3, 6.0):
            r = oracle.truncate_to_tol(D, resid, tol)
            ok = [rr for rr in range(6) if resid ** 2 + np.sum(D[rr:] ** 2) <= tol ** 2]
            assert r == (ok[0] if ok else 5)


def test_single_vector_finder_spans_block_sketch():
    """Fig. singlevecrangefinder: q_1..q_p form an ON basis of A G(:, 1:p), the
    same as the block method (caption of that figure)."""
    A = lowrank_np(100, 70, poly_spectrum(70, 1.0), seed=6)
    Q1, B1, G = oracle.single_vector_range_finder(A, 12, seed=4)
    Q2, _ = oracle.orth(A @ G)
    np.testing.assert_allclose(Q1, Q2, atol=1e-10)
    np.testing.assert_allclose(B1, Q1.T @ A, atol=1e-12)


def test_adaptive_range_finder_meets_tolerance():
    """Fig. adaptive2: ||A - Q Q* A|| <= eps w.p. >= 1 - min(m,n) 10^-r."""
    A = lowrank_np(150, 120, exp_spectrum(120, 5.0), seed=9)
    for s in range(10):
        eps = 1e-4 * np.linalg.norm(A, 2)
        Q, draws = oracle.adaptive_range_finder(A, eps, r=10, seed=s)
        np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)
        assert np.linalg.norm(A - Q @ (Q.T @ A), 2) <= eps
        assert draws == Q.shape[1] + 10


def test_gaussian_norm_estimator_identity():
    """eq. (infomm): E ||T g||^2 = ||T||_Fro^2."""
    T = lowrank_np(60, 50, poly_spectrum(50, 0.7), seed=11)
    G = oracle.gaussian(50, 4000, seed=3, stream=2)
    vals = np.sum((T @ G) ** 2, axis=0)
    fro2 = np.sum(T * T)
    assert abs(vals.mean() - fro2) <= 5 * vals.std() / np.sqrt(vals.size)


def test_certificate_bounds_the_error():
    """Lemma thm:aposteriori with alpha = 1/10, r = 10 (Sec. 14): the certificate
    upper-bounds ||A - A_approx|| (fails w.p. <= 1e-10)."""
    A = lowrank_np(120, 90, poly_spectrum(90, 1.0), seed=12)
    r = oracle.rsvd_power(A, 10, 5, 0, seed=1)
    true = np.linalg.norm(A - (r["U"] * r["D"]) @ r["V"].T, 2)
    for s in range(100):
        bound, cn = oracle.certificate(A, r["U"], r["D"], r["V"], seed=1000 + s)
        assert bound >= true
        assert len(cn) == 10


def test_blocked_with_spectral_stop():
    """adaptive_blocked_spectral: the blocked scheme with Fig. adaptive2's test
    on each fresh block.  Its basis is the blocked scheme's own (same blocks,
    same steps, bit for bit); where it stops, the spectral error is below eps
    on every seed (Lemma thm:aposteriori, failure probability 10^-16 per
    test), so its rank is at least the spectral eps-rank; and it stops within
    two blocks of the rank where the Frobenius tail falls below a quarter of
    the threshold (a Gaussian probe of a remainder that small stays under the
    threshold)."""
    import numpy as np
    from oracle.adaptive import adaptive_blocked_spectral, adaptive_blocked
    from workloads import lowrank_np, exp_spectrum
    sig = exp_spectrum(200)
    A = lowrank_np(300, 200, sig, seed=1)
    tail = np.sqrt(np.concatenate([np.cumsum((sig ** 2)[::-1])[::-1], [0.0]]))    # tail[r] = ||A - A_r||_F
    for eps in (1e-2, 1e-3, 1e-4):
        th = eps / (10.0 * np.sqrt(2.0 / np.pi))
        lo, hi = int(np.sum(sig > eps)), int(np.argmax(tail <= th / 4)) + 32
        for seed in range(8):
            r = adaptive_blocked_spectral(A, eps, b=16, seed=seed)
            assert r["converged"] and r["probes"][-1] <= th < r["probes"][:-1].min()
            assert np.linalg.norm(A - r["Q"] @ r["B"], 2) <= eps
            assert lo <= r["rank"] <= hi, (eps, seed, r["rank"], lo, hi)
            if seed < 2:
                ref = adaptive_blocked(A, 1e-300, b=16, seed=seed, max_rank=r["rank"])
                assert np.array_equal(ref["Q"], r["Q"]) and np.array_equal(ref["B"], r["B"])
    z = adaptive_blocked_spectral(np.zeros((40, 30)), 1e-6, seed=0)
    assert z["rank"] == 0 and z["converged"]
    capped = adaptive_blocked_spectral(A, 1e-12, b=16, seed=0, max_rank=48)
    assert capped["rank"] == 48 and not capped["converged"]
