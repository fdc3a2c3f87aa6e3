"""Pins of the extended-sampling (block Krylov) oracle (Sec. "Extended
sampling matrix") and of the implicitly centred solver: q = 1 is Fig. RSVD;
a rank-r input with l < r <= q l is recovered exactly, which one block
cannot do; the basis spans the same space as a block-by-block
orthonormalized Krylov basis; nesting (the last block is the power scheme's
sample) makes the truncated Frobenius residual no larger than that of
Fig. RSVDP_stabilized with q - 1 steps and the same G.  The centred solver
equals the fixed-rank oracle run on the explicitly centred matrix, and its U
is orthogonal to the ones vector."""
import numpy as np
import pytest

from oracle import rsvd_basic, rsvd_power, orth
from oracle.krylov import rsvd_block_krylov
from oracle.centred import rsvd_power_centred


def _rank_r(m, n, s, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, len(s))))
    V, _ = np.linalg.qr(rng.standard_normal((n, len(s))))
    return (U * s[None, :]) @ V.T


def _fro_trunc(A, r):
    return np.linalg.norm(A - (r["U"] * r["D"][None, :]) @ r["V"].T)


def test_one_block_is_the_basic_rsvd():
    A = np.random.default_rng(0).standard_normal((160, 120))
    a = rsvd_block_krylov(A, 8, 4, 1, seed=3)
    b = rsvd_basic(A, 8, 4, seed=3)
    for key in ("U", "D", "V", "Q"):
        assert np.array_equal(a[key], b[key])


def test_exact_recovery_beyond_one_block():
    k, p, r = 8, 4, 30                        # l = 12 < r = 30 <= 3 l
    A = _rank_r(160, 120, np.linspace(1.0, 0.5, r), 1)
    kr = rsvd_block_krylov(A, k, p, 3, seed=1, full=True)
    assert np.allclose((kr["U"] * kr["D"][None, :]) @ kr["V"].T, A, atol=1e-12)
    assert np.allclose(kr["D"][:r], np.linspace(1.0, 0.5, r), rtol=1e-12)
    b = rsvd_basic(A, k, p, seed=1, full=True)
    assert np.abs((b["U"] * b["D"][None, :]) @ b["V"].T - A).max() > 1e-2


def test_span_equals_blockwise_orthonormalized_krylov_space():
    m, n, k, p, q = 150, 110, 6, 4, 3
    A = _rank_r(m, n, 1.0 / (1.0 + np.arange(100)) ** 0.5, 2)
    kr = rsvd_block_krylov(A, k, p, q, seed=4)
    G = kr["G"]
    blocks = [orth(A @ G)[0]]
    for _ in range(q - 1):
        blocks.append(orth(A @ (A.T @ blocks[-1]))[0])
    Qs, _ = np.linalg.qr(np.hstack(blocks))
    assert np.allclose(kr["Q"] @ kr["Q"].T, Qs @ Qs.T, atol=1e-9)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_nested_space_never_worse_than_power_scheme(seed):
    m, n, k, p = 160, 120, 8, 4
    sig = 1.0 / (1.0 + np.arange(n))
    A = _rank_r(m, n, sig, 5)
    opt = np.sqrt(np.sum(sig[k:] ** 2))
    ek = _fro_trunc(A, rsvd_block_krylov(A, k, p, 3, seed))
    ep = _fro_trunc(A, rsvd_power(A, k, p, 2, seed))
    eb = _fro_trunc(A, rsvd_basic(A, k, p, seed))
    assert opt * (1 - 1e-12) <= ek <= ep * (1 + 1e-12) <= eb * (1 + 1e-12)


def test_block_count_checked():
    with pytest.raises(ValueError):
        rsvd_block_krylov(np.ones((40, 30)), 6, 4, 4, seed=0)    # q l = 40 > 30
    with pytest.raises(ValueError):
        rsvd_block_krylov(np.ones((40, 30)), 6, 4, 0, seed=0)


@pytest.mark.parametrize("q", [0, 2])
def test_centred_equals_explicit_centring(q):
    m, n, k, p = 160, 120, 8, 4
    rng = np.random.default_rng(6)
    A = rng.standard_normal((m, n)) + 3.0 + np.outer(np.ones(m), 5.0 * rng.standard_normal(n))
    c = rsvd_power_centred(A, k, p, q, seed=5)
    mu = A.mean(axis=0)
    assert np.allclose(c["mu"], mu, atol=1e-13)
    d = rsvd_power(A - np.outer(np.ones(m), mu), k, p, q, seed=5)
    for key in ("U", "D", "V"):
        assert np.allclose(c[key], d[key], atol=1e-11)
    assert np.abs(c["U"].sum(axis=0)).max() < 1e-11          # 1* Abar = 0
    # the mean is a rank-one spike that the uncentred solver spends a triplet on
    u = rsvd_power(A, k, p, q, seed=5)
    assert u["D"][0] > 10 * c["D"][0]


def test_centred_products_match_the_formed_matrix():
    from oracle.centred import centred_apply, centred_apply_t, column_means
    rng = np.random.default_rng(7)
    A = rng.standard_normal((50, 30)) + 2.0
    Abar = A - A.mean(axis=0)[None, :]
    mu = column_means(A)
    X, Y = rng.standard_normal((30, 4)), rng.standard_normal((50, 4))
    assert np.allclose(centred_apply(A, mu, X), Abar @ X, atol=1e-12)
    assert np.allclose(centred_apply_t(A, mu, Y), Abar.T @ Y, atol=1e-12)
