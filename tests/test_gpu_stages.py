"""Stage-by-stage parity of the CUDA path with the float64 oracle (GPU)."""
import numpy as np
import pytest

import oracle
from oracle import philox
from workloads import lowrank_np, poly_spectrum

pytestmark = pytest.mark.gpu


def _t(x, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


@pytest.mark.parametrize("ng,l,seed,stream,col0", [(1, 1, 0, 0, 0), (257, 33, 12345, 0, 0),
                                                   (64, 16, (9 << 32) | 7, 2, 40), (1000, 3, 1, 4, 5)])
def test_philox_words_bit_exact(lib, ng, l, seed, stream, col0):
    got = lib.philox_words(ng, l, seed, stream, col0).cpu().numpy().view(np.uint32).reshape(l, ng, 4)
    ref = philox.omega_words(ng, l, seed, stream, col0)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n,l", [(1, 1), (7, 5), (1001, 30), (4096, 256), (3, 300)])
def test_gaussian_parity(lib, n, l):
    import torch
    seed = 1000 + n
    ref = philox.gaussian(n, l, seed, stream=0)
    g64 = lib.gaussian(n, l, seed, dtype=torch.float64).cpu().numpy()
    np.testing.assert_allclose(g64, ref, rtol=0, atol=4e-15 * np.maximum(1.0, np.abs(ref)).max())
    g32 = lib.gaussian(n, l, seed, dtype=torch.float32).cpu().numpy().astype(np.float64)
    # binary32 Box-Muller from the same 24-bit uniforms: a few ulp of the radius (<= 5.8)
    assert np.max(np.abs(g32 - ref)) <= 8 * 2.0 ** -21
    gbf = lib.gaussian(n, l, seed, dtype=torch.bfloat16).float().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gbf - ref) / np.maximum(np.abs(ref), 1e-30)) <= 2.0 ** -8 + 1e-6
    # column offset and prefix property
    sub = lib.gaussian(n, max(1, l // 2), seed, col0=l - max(1, l // 2), dtype=torch.float64).cpu().numpy()
    np.testing.assert_array_equal(sub, g64[:, l - max(1, l // 2):])


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("m,n,l", [(1, 1, 1), (300, 200, 30), (1000, 777, 61), (129, 4100, 256), (4500, 70, 64)])
def test_sketch_simt_parity(lib, trans, m, n, l):
    import torch
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n))
    X = rng.standard_normal((m if trans else n, l))
    ref = (A.T if trans else A) @ X
    Y64 = lib.sketch(_t(A), _t(X), trans=trans, prec=lib.RSVD_F64).cpu().numpy()
    K = m if trans else n
    bound64 = 4 * K * 2.0 ** -53 * (np.abs(A.T if trans else A) @ np.abs(X))
    assert np.all(np.abs(Y64 - ref) <= bound64 + 1e-300)
    A32, X32 = A.astype(np.float32), X.astype(np.float32)
    ref32 = (A32.astype(np.float64).T if trans else A32.astype(np.float64)) @ X32.astype(np.float64)
    Y32 = lib.sketch(_t(A32), _t(X32), trans=trans, prec=lib.RSVD_F32).cpu().numpy().astype(np.float64)
    absprod = (np.abs(A32.astype(np.float64)).T if trans else np.abs(A32.astype(np.float64))) @ np.abs(X32)
    assert np.all(np.abs(Y32 - ref32) <= 2 * K * 2.0 ** -24 * absprod + 1e-30)


@pytest.mark.parametrize("rows,l,cond", [(50, 1, 1e2), (300, 30, 1e3), (2000, 64, 1e5), (5000, 256, 1e3),
                                         (4099, 100, 1e6)])
def test_orth_parity(lib, rows, l, cond):
    rng = np.random.default_rng(rows + l)
    G = rng.standard_normal((rows, l))
    Qg, _ = np.linalg.qr(G)
    W, _ = np.linalg.qr(rng.standard_normal((l, l)))
    Y = (Qg * np.geomspace(1.0, 1.0 / cond, l)[None, :]) @ W.T
    Qref, Rref = oracle.orth(Y)
    # binary64 path (l <= 128)
    if l <= 128:
        Q, R = lib.orth(_t(Y), prec=lib.RSVD_F64)
        Q, R = Q.cpu().numpy(), R.cpu().numpy()
        np.testing.assert_allclose(Q.T @ Q, np.eye(l), atol=1e-12)
        assert np.max(np.abs(Q - Qref)) <= 1e-15 * cond * 100 + 1e-13
        np.testing.assert_allclose(Q @ R, Y, atol=1e-13 * np.abs(Y).max())
    else:
        with pytest.raises(lib.RsvdError) as ei:
            lib.orth(_t(Y), prec=lib.RSVD_F64)
        assert ei.value.code == lib.RSVD_E_UNSUPPORTED
    # binary32 path: orthonormal to binary32 accuracy, same Q up to the conditioning
    Y32 = Y.astype(np.float32)
    Qref32, _ = oracle.orth(Y32.astype(np.float64))
    Q32, R32 = lib.orth(_t(Y32), prec=lib.RSVD_F32)
    Q32, R32 = Q32.cpu().numpy().astype(np.float64), R32.cpu().numpy()
    assert np.linalg.norm(Q32.T @ Q32 - np.eye(l), 2) <= 10 * 2.0 ** -24 * np.sqrt(l) * l
    assert np.max(np.abs(Q32 - Qref32)) <= 2.0 ** -24 * cond * 50 * np.sqrt(l)
    assert np.linalg.norm(Q32 @ R32 - Y32, 2) <= 1e-5 * np.linalg.norm(Y32, 2)
    assert np.all(np.diag(R32) > 0)
