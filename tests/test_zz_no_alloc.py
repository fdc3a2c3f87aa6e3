"""rsvd_sketch_noalloc: the bf16 tensor-core sketch product for callers that
cannot allocate device memory (no workspace argument; the scratch is a fixed
array in the library).  Checked against rsvd_sketch, the entry point that takes
a caller workspace, on two calls in a row (the second call reuses the scratch
the first one left behind).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _bf16(rng, shape):
    import torch
    x = torch.from_numpy(rng.standard_normal(shape)).to(torch.float32).to(torch.bfloat16).cuda()
    r, c = shape
    c8 = (c + 7) // 8 * 8
    buf = torch.zeros(r, c8, dtype=torch.bfloat16, device="cuda")
    buf[:, :c] = x
    return buf[:, :c]


@pytest.mark.parametrize("trans,m,n,l", [(False, 3000, 2000, 128), (True, 5000, 700, 96), (False, 256, 20000, 64)])
def test_noalloc_matches_workspace_entry_point(lib, trans, m, n, l):
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
    bound = 2 * K * U32 * (np.abs(Aop) @ np.abs(X64)) + 1e-30
    for call in range(2):
        ref = lib.sketch(A, X, trans=trans, prec=lib.RSVD_MIXED_BF16).cpu().numpy().astype(np.float64)
        Y = torch.full((M, l), float("nan"), dtype=torch.float32, device="cuda")
        code = lib.rsvd_sketch_noalloc(h, int(trans), m, n, l, A, A.stride(0), X, X.stride(0), Y, Y.stride(0))
        assert code == lib.RSVD_OK, lib.last_error(h)
        got = Y.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
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
