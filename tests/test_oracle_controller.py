"""Pins of the controller oracle (oracle/controller.py) against closed forms,
invariants, finite differences and brute force.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import controller as C
from workloads import haar_np, lowrank_np, step_spectrum, mlp_init, controller_matrix_np, controller_case


def test_probe_of_orthogonal_matrix_sees_the_gaussian_block():
    # sigma(c Q G) = c sigma(G) for orthogonal Q; the reference values come
    # from the eigenvalues of G^T G (a different LAPACK routine than the SVD).
    n, seed = 64, 11
    Q = haar_np(np.random.default_rng(3), n, n)
    sig = C.probe_singular_values(3.5 * Q, seed)
    G = oracle.gaussian(n, 16, seed, oracle.STREAM_SKETCH)
    ev = np.sort(np.linalg.eigvalsh(G.T @ G))[::-1]
    assert np.allclose(sig, 3.5 * np.sqrt(ev), rtol=1e-12)
    f = C.features(sig, n, n)
    assert np.allclose(f[:15], np.log10(np.sqrt(ev[1:] / ev[0])), atol=1e-12)
    assert f[15] == pytest.approx(6.0 / 16.0) and f[16] == pytest.approx(6.0 / 16.0)


def test_features_rank_deficient_scale_invariant_and_zero():
    A = lowrank_np(120, 90, np.geomspace(1, 0.1, 5), seed=4)
    f = C.probe_features(A, 5)
    assert np.all(f[4:15] == C.FEAT_FLOOR) and np.all(f[:4] > -2.0)
    assert np.all(f[:15] >= C.FEAT_FLOOR)
    assert np.allclose(C.probe_features(7.0 * A, 5), f, atol=1e-12)
    z = C.probe_features(np.zeros((40, 30)), 5)
    assert np.all(z[:15] == C.FEAT_FLOOR)
    assert z[15] == pytest.approx(np.log2(40) / 16) and z[16] == pytest.approx(np.log2(30) / 16)


def test_forward_closed_forms():
    X = np.random.default_rng(0).standard_normal((7, C.D_IN))
    # (a) zero weights: logits equal b3
    P = {name: np.zeros(shape) for name, shape in C.SHAPES}
    P["b3"] = np.arange(C.N_OUT, dtype=np.float64)
    Z, _, _ = C.forward(C.pack(P), X)
    assert np.array_equal(Z, np.tile(P["b3"], (7, 1)))
    # (b) a hand-built network whose logit 0 is ||x||_1 and logit 1 is max(x_0, 0)
    P = {name: np.zeros(shape) for name, shape in C.SHAPES}
    for i in range(C.D_IN):
        P["W1"][i, i] = 1.0
        P["W1"][C.D_IN + i, i] = -1.0
        P["W2"][i, i] = 1.0
        P["W2"][i, C.D_IN + i] = 1.0
    P["W3"][0, :C.D_IN] = 1.0
    P["W2"][100, 0] = 1.0
    P["W3"][1, 100] = 1.0
    Z, _, _ = C.forward(C.pack(P), X)
    assert np.allclose(Z[:, 0], np.abs(X).sum(axis=1), atol=1e-14)
    assert np.allclose(Z[:, 1], np.maximum(X[:, 0], 0.0), atol=1e-14)
    # (c) without biases the ReLU network is positively homogeneous
    th = mlp_init(1)
    Z1, _, _ = C.forward(th, X)
    Z2, _, _ = C.forward(th, 2.5 * X)
    assert np.allclose(Z2, 2.5 * Z1, rtol=1e-12, atol=1e-12)


def test_loss_at_uniform_logits():
    X = np.random.default_rng(1).standard_normal((6, C.D_IN))
    th = mlp_init(2)
    P = C.unpack(th.copy())
    P["W3"][:] = 0.0
    P["b3"][:] = 0.0
    yl = np.array([0, 3, 7, 15, 2, 9])
    yq = np.array([0, 1, 2, 3, 0, 1])
    lam = 0.7
    loss, _ = C.loss_and_grad(C.pack(P), X, yl, yq, lam)
    expect = np.log(16.0) + np.log(4.0) + lam * np.mean(yl / 16.0)
    assert loss == pytest.approx(expect, rel=1e-13)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    th = mlp_init(3) + 0.05 * rng.standard_normal(C.n_params())
    X = rng.standard_normal((5, C.D_IN))
    yl = rng.integers(0, C.N_L, 5)
    yq = rng.integers(0, C.N_Q, 5)
    lam = 0.5
    _, g = C.loss_and_grad(th, X, yl, yq, lam)
    idx = np.concatenate([rng.choice(C.n_params(), 300, replace=False),
                          np.arange(C.n_params() - C.N_OUT, C.n_params())])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (C.loss_and_grad(th + e, X, yl, yq, lam)[0] - C.loss_and_grad(th - e, X, yl, yq, lam)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_adam_first_step_is_a_signed_step():
    rng = np.random.default_rng(6)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m1, m2 = C.adam_step(th, g, np.zeros(50), np.zeros(50), 1, 0.01)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_decide_quantile_and_ties():
    z = np.full(C.N_OUT, -50.0)
    z[5] = 50.0
    z[C.N_L + 2] = 1.0
    assert C.decide(z) == (96, 2)
    # l probabilities 0.5 on class 1, 0.5 on class 6: the 0.9 quantile is class 6
    z = np.full(C.N_OUT, -50.0)
    z[1] = z[6] = 10.0
    z[C.N_L:] = 0.0  # all q tie -> the lowest
    assert C.decide(z, 0.9) == (112, 0)
    assert C.decide(z, 0.4) == (32, 0)


def test_label_from_ranks_brute_force():
    assert C.label_from_ranks([64, 48, 48, 48], [True] * 4) == (3, 0)
    assert C.label_from_ranks([160, 48, 32, 32], [True] * 4) == (2, 1)   # 192 == 192 -> q = 1
    assert C.label_from_ranks([256, 256, 256, 256], [False] * 4) == (15, 2)
    assert C.label_from_ranks([256, 200, 100, 80], [False, True, True, True]) == (6, 2)
    # brute force over every small case: the chosen (q, l) minimizes the cost
    rng = np.random.default_rng(7)
    for _ in range(200):
        ranks = list(rng.integers(1, 17, 4) * 16)
        conv = list(rng.random(4) < 0.7)
        c, q = C.label_from_ranks(ranks, conv)
        feas = [(2 * qq + 2) * r for qq, (r, ok) in enumerate(zip(ranks, conv)) if ok]
        if feas:
            assert conv[q] and (2 * q + 2) * ranks[q] == min(feas) and c == ranks[q] // 16 - 1
        else:
            assert (c, q) == (15, 2)


def test_adaptive_labels_on_a_step_spectrum():
    # step at rank 24 then 1e-6: the eps-rank at tol 1e-4 is 24, so the blocked
    # finder (b = 16) stops at rank 32 for every q, and q = 0 is the cheapest.
    A = lowrank_np(200, 160, step_spectrum(160, 24), seed=8)
    ranks, conv = C.adaptive_ranks(A, 1e-4, seed=9, R=96)
    assert conv == [True] * 4 and ranks == [32] * 4
    assert C.label_from_ranks(ranks, conv) == (1, 0)


def test_adaptive_labels_bracket_the_eps_rank():
    # brute force: eps-rank from a full SVD; each l_q lies in [eps-rank, eps-rank + 2b]
    for seed in (10, 11):
        A, (n, kind, par) = controller_matrix_np(seed, lo=96, hi=160)
        A = A.astype(np.float64)
        s = np.linalg.svd(A, compute_uv=False)
        eps2 = (1e-4 ** 2) * np.sum(s * s)
        tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
        k_eps = int(np.argmax(tail <= eps2))
        ranks, conv = C.adaptive_ranks(A, 1e-4, seed=seed, R=min(n, 256))
        for r, ok in zip(ranks, conv):
            if ok:
                assert k_eps <= r <= k_eps + 32, (kind, par, k_eps, ranks)


def test_residual_estimate_is_unbiased_and_bounds_the_norm():
    A = lowrank_np(150, 100, np.geomspace(1, 1e-3, 100), seed=12)
    out = oracle.rsvd_power(A, 10, 0, 0, seed=1)
    T = A - out["U"] @ np.diag(out["D"]) @ out["V"].T
    fro, spec = np.linalg.norm(T), np.linalg.norm(T, 2)
    est2 = []
    for seed in range(200):
        f, b, _ = C.residual_estimate(A, out["U"], out["D"], out["V"], seed)
        est2.append(f * f)
        assert b >= spec
    assert np.mean(est2) == pytest.approx(fro * fro, rel=0.05)


def test_controller_stream_spectra():
    for seed in range(30):
        n, s, kind, par = controller_case(seed, 512, 16384)
        assert 512 <= n <= 16384 and len(s) == n and np.all(np.diff(s) <= 0)
        if kind == "exp":
            assert 16 <= par <= 256
        elif kind == "poly":
            assert 0.5 <= par <= 2.0
        else:
            assert s[int(par) - 1] == 1.0 and s[int(par)] == 1e-6
