"""rsvd_sketch_noalloc: the bf16 tensor-core sketch product for callers that
cannot allocate device memory -- code running inside another framework's
memory pool, an allocation-free real-time loop, or a plugin that is handed only
its input and output buffers.  It takes no workspace: its scratch is a fixed
array inside the library.

Each case runs the call twice in a row (the second call reuses the scratch the
first one left behind) and checks every element of Y against the exact
float64 product of the same bf16 operands, within the binary32 accumulation
bound the other tensor-core tests use, and against rsvd_sketch (the entry
point with a caller workspace) within the same bound.  The cases cover both
operand layouts, a ragged M, K long enough that every tile is split between
many CTAs (partial tiles in the fixed array, added by the fix-up kernel) and a
K long enough that one CTA adds several TMEM segments of a tile.  This file is
collected last on purpose: a failure here leaves every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _bf16(rng, shape):
    import torch
    x = torch.from_numpy(rng.standard_normal(shape, dtype=np.float32)).to(torch.bfloat16).cuda()
    r, c = shape
    c8 = (c + 7) // 8 * 8
    buf = torch.zeros(r, c8, dtype=torch.bfloat16, device="cuda")
    buf[:, :c] = x
    return buf[:, :c]


@pytest.mark.parametrize("trans,m,n,l", [
    (False, 3000, 2000, 128),     # NN, ragged M (3000 = 23 x 128 + 56)
    (True, 5000, 700, 96),        # TN (A^T X), ragged M = 700
    (False, 256, 20000, 64),      # two tiles, each split between ~76 CTAs
    (False, 128, 1 << 21, 16),    # one tile, ~215 k-blocks per CTA: two TMEM segments each
])
def test_noalloc_matches_exact_product_and_workspace_entry_point(lib, trans, m, n, l):
    import torch
    h = lib.handle()
    rng = np.random.default_rng(m + n + l)
    A = _bf16(rng, (m, n))
    X = _bf16(rng, ((m if trans else n), l))
    M = n if trans else m
    K = m if trans else n
    A64 = A.float().cpu().numpy().astype(np.float64)
    X64 = X.float().cpu().numpy().astype(np.float64)
    Aop = A64.T if trans else A64
    exact = Aop @ X64
    bound = 2 * K * U32 * (np.abs(Aop) @ np.abs(X64)) + 1e-30
    del A64, Aop
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        Y = torch.full((M, l), float("nan"), dtype=torch.float32, device="cuda")
        code = lib.rsvd_sketch_noalloc(h, int(trans), m, n, l, A, A.stride(0), X, X.stride(0), Y, Y.stride(0),
                                       status=status)
        assert code == lib.RSVD_OK, lib.last_error(h)
        torch.cuda.synchronize()
        assert int(status.item()) == lib.RSVD_OK
        got = Y.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got)), call
        err = np.abs(got - exact)
        assert np.all(err <= bound), (call, float(np.max(err / bound)))
        ref = lib.sketch(A, X, trans=trans, prec=lib.RSVD_MIXED_BF16).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref) <= bound), (call, float(np.max(np.abs(got - ref) / bound)))


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    h = lib.handle()
    A = torch.zeros(256, 256, dtype=torch.bfloat16, device="cuda")
    X = torch.zeros(256, 136, dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros(256, 136, dtype=torch.float32, device="cuda")
    code = lib.rsvd_sketch_noalloc(h, 0, 256, 256, 136, A, 256, X, 136, Y, 136)
    assert code == lib.RSVD_E_INVALID
    assert "128" in lib.last_error(h)
