"""rsvd_batched: many tolerance-driven problems (Sec. 12.3 Fig. greedy_blocked,
then Stage B of Sec. 3) in one persistent launch, each checked against the
float64 oracle's adaptive_blocked with the same Gaussian blocks (Philox stream
1, key = seed + problem index)."""
import numpy as np
import pytest

import oracle
from workloads import kernel_block, kernel_block_torch, kernel_block_shapes, lowrank_np, exp_spectrum

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _check_problem(A, res, p, tol, seed, b=16, R=64, rank_exact=True):
    """Compare problem p of a finished plan with the oracle."""
    A64 = np.asarray(A, dtype=np.float64)
    m, n = A64.shape
    U, D, V = [t.cpu().numpy().astype(np.float64) for t in res.result(p)]
    rank = int(res.rank[p])
    err = float(res.err[p])
    ref = oracle.adaptive_blocked(A64, tol, b=b, seed=seed + p, max_rank=min(R, m, n))
    nA = np.linalg.norm(A64)
    # The stopping test runs on a binary32 remainder, whose rounding adds a
    # floor of a few u ||A||_F to the float64 one; the rank must agree unless
    # the oracle's remainder lies within 5% of the threshold or that floor
    # could carry it across.
    eps = ref["eps"]
    floor = 8 * U32 * nA
    r = ref["norms_direct"]
    ambiguous = np.any(np.abs(r - eps) < 0.05 * eps) or np.any((r <= eps) & (np.hypot(r, floor) > 0.95 * eps))
    if rank_exact and not ambiguous:
        assert rank == ref["rank"], (p, rank, ref["rank"])
    else:
        assert ref["rank"] <= rank <= ref["rank"] + b or rank == min(R, m, n), (p, rank, ref["rank"])
    resid = np.linalg.norm(A64 - (U[:, :rank] * D[:rank]) @ V[:, :rank].T) / nA if nA > 0 else 0.0
    # When the oracle needs every column it may take (rank = min(R, m, n) and
    # the remainder of an exactly low-rank matrix), its remainder is zero while
    # the binary32 one is the round-off of a last Gaussian block with no
    # oversampling over that remainder's rank: allow a 200 u floor there.
    full = ref["rank"] == min(R, m, n) and min(m, n) <= R
    if full:
        assert rank == ref["rank"]
        assert int(res.status[p]) in (0, 5) and err <= max(tol, 200 * U32), (p, err)
    elif ref["converged"] and not ambiguous:
        assert int(res.status[p]) == 0, (p, (m, n), rank, ref["rank"], err, r / nA)
        assert err <= tol
        assert resid <= 2 * tol
    # the reported remainder is the factorization's error to binary32 accuracy
    assert abs(resid - err) <= 0.05 * tol + 64 * U32, (resid, err)
    nr = min(rank, ref["rank"])
    np.testing.assert_allclose(D[:nr], ref["D"][:nr], rtol=1e-4, atol=1e-6 * ref["D"][0] + 1e-30)
    assert np.all(D[rank:] == 0) and np.all(U[:, rank:] == 0) and np.all(V[:, rank:] == 0)
    if rank:
        for X in (U[:, :rank], V[:, :rank]):
            np.testing.assert_allclose(X.T @ X, np.eye(rank), atol=2e-5)
        # singular vectors with a clear gap agree (signs fixed by the convention)
        d = ref["D"][:nr]
        gap = np.minimum(np.abs(np.diff(d, prepend=np.inf)), np.abs(np.diff(d, append=-np.inf)))
        well = np.nonzero(gap > 1e-2 * d[0])[0]
        for k in well:
            assert np.max(np.abs(U[:, k] - ref["U"][:, k])) < 1e-3, k
            assert np.max(np.abs(V[:, k] - ref["V"][:, k])) < 1e-3, k
    return rank, ref


def _plan(lib, blocks, R=64):
    import torch
    plan = lib.BatchPlan([b.shape for b in blocks], R=R)
    for p, b in enumerate(blocks):
        plan.block(p).copy_(torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)))
    return plan


def test_batched_kernel_blocks_match_oracle(lib):
    """The workload's first blocks (1/|x - y| kernels, tol 1e-6) against the oracle."""
    blocks = [kernel_block(b, seed=4001) for b in range(12)]
    plan = _plan(lib, blocks)
    code = lib.batched_run(plan, 1e-6, block=16, seed=100, flags=lib.RSVD_FLAG_SYNC)
    assert code == lib.RSVD_OK, lib.last_error(lib.handle())
    for p, A in enumerate(blocks):
        _check_problem(A, plan, p, 1e-6, 100)


@pytest.mark.parametrize("b,R,tol", [(16, 64, 1e-6), (8, 40, 1e-5), (5, 17, 1e-4)])
def test_batched_ragged_shapes_and_blocks(lib, b, R, tol):
    """Low-rank test matrices of ragged shapes (several tiles and tails of the
    row and column passes, sizes below b and below the rank cap)."""
    shapes = [(300, 200), (64, 1024), (1024, 64), (257, 255), (33, 700), (700, 31), (12, 400), (400, 9),
              (3, 3), (1, 50), (129, 1000)]
    blocks = [lowrank_np(m, n, exp_spectrum(min(m, n), 3.0), seed=7 * m + n).astype(np.float32)
              for m, n in shapes]
    plan = _plan(lib, blocks, R=R)
    lib.batched_run(plan, tol, block=b, seed=5, flags=lib.RSVD_FLAG_SYNC)
    for p, A in enumerate(blocks):
        _check_problem(A, plan, p, tol, 5, b=b, R=R)


def test_batched_cap_zero_invalid_and_nonfinite(lib):
    """Per-problem outcomes: rank cap reached, zero matrix, a size out of range
    and a NaN entry each stay within their own problem."""
    import torch
    rng = np.random.default_rng(3)
    good = kernel_block(5, seed=4001)
    noise = rng.standard_normal((200, 150)).astype(np.float32)
    zero = np.zeros((90, 70), np.float32)
    nan = kernel_block(6, seed=4001).copy()
    nan[3, 4] = np.nan
    blocks = [good, noise, zero, nan, good]
    plan = _plan(lib, blocks, R=32)
    # problem 4 claims n = 2000 (beyond the 1024 limit)
    plan.n[4] = 2000
    plan.lda[4] = 2000
    code = lib.batched_run(plan, 1e-6, seed=9, flags=lib.RSVD_FLAG_SYNC)
    assert code != lib.RSVD_OK
    st = plan.status.cpu().tolist()
    assert st[0] == lib.RSVD_OK
    assert st[1] == lib.RSVD_E_NOT_CONVERGED and int(plan.rank[1]) == 32 and float(plan.err[1]) > 1e-6
    ref = oracle.adaptive_blocked(noise.astype(np.float64), 1e-6, b=16, seed=9 + 1, max_rank=32)
    np.testing.assert_allclose(plan.result(1)[1].cpu().numpy(), ref["D"], rtol=1e-4)
    assert st[2] == lib.RSVD_OK and int(plan.rank[2]) == 0 and float(plan.result(2)[1].abs().max()) == 0.0
    assert st[3] == lib.RSVD_E_NONFINITE and int(plan.rank[3]) == 0
    assert st[4] == lib.RSVD_E_INVALID and int(plan.rank[4]) == 0
    _check_problem(good, plan, 0, 1e-6, 9, R=32)


def test_batched_deterministic_and_graph_replay(lib):
    """Results do not depend on which CTA takes a problem: two eager runs and a
    CUDA-graph replay of the same plan agree bit for bit."""
    import torch
    blocks = [kernel_block(b, seed=4001) for b in range(20, 40)]
    plan = _plan(lib, blocks)
    lib.batched_run(plan, 1e-6, seed=1, flags=lib.RSVD_FLAG_SYNC)
    first = [t.clone() for t in (plan.U, plan.D, plan.V, plan.rank, plan.err)]
    lib.batched_run(plan, 1e-6, seed=1, flags=lib.RSVD_FLAG_SYNC)
    for a, b in zip(first, (plan.U, plan.D, plan.V, plan.rank, plan.err)):
        assert torch.equal(a, b)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lib.batched_run(plan, 1e-6, seed=1, stream=s)  # warm-up on the capture stream
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    for t in (plan.U, plan.V, plan.D, plan.err):
        t.zero_()
    plan.rank.zero_()
    with torch.cuda.graph(g, stream=s):
        code = lib.batched_run(plan, 1e-6, seed=1, stream=s)
    assert code == lib.RSVD_OK
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(first, (plan.U, plan.D, plan.V, plan.rank, plan.err)):
        assert torch.equal(a, b)


def test_batched_argument_errors(lib):
    import ctypes
    h = lib.handle()
    for kw, code in [(dict(tol=0.0), lib.RSVD_E_INVALID), (dict(tol=1e-3, block=17), lib.RSVD_E_INVALID),
                     (dict(tol=1e-3, max_rank=65), lib.RSVD_E_INVALID)]:
        prm = lib.make_params(0, 0, 0, 1, lib.RSVD_F32, 0, **kw)
        out = ctypes.c_size_t()
        assert lib.load().rsvd_batched_workspace_size(h, 4, ctypes.byref(prm), ctypes.byref(out)) == code, kw
    prm = lib.make_params(0, 0, 1, 1, lib.RSVD_F32, 0, tol=1e-3)
    out = ctypes.c_size_t()
    assert lib.load().rsvd_batched_workspace_size(h, 4, ctypes.byref(prm), ctypes.byref(out)) == \
        lib.RSVD_E_UNSUPPORTED
    prm = lib.make_params(0, 0, 0, 1, lib.RSVD_F64, 0, tol=1e-3)
    assert lib.load().rsvd_batched_workspace_size(h, 4, ctypes.byref(prm), ctypes.byref(out)) == \
        lib.RSVD_E_UNSUPPORTED


@pytest.mark.slow
def test_batched_full_workload_sampled(lib):
    """All 4096 blocks of the batched workload (m, n ~ U{64..1024}) in the
    launch configuration the benchmark times; every problem converges, and a
    sample of blocks matches the oracle."""
    import torch
    shapes = kernel_block_shapes(4096, seed=4001)
    plan = lib.BatchPlan(shapes, R=64)
    for p in range(len(shapes)):
        kernel_block_torch(p, plan.block(p), seed=4001)
    code = lib.batched_run(plan, 1e-6, block=16, seed=0, flags=lib.RSVD_FLAG_SYNC)
    assert code == lib.RSVD_OK, lib.last_error(lib.handle())
    assert int(plan.status.abs().max()) == 0
    assert float(plan.err.max()) <= 1e-6
    rng = np.random.default_rng(11)
    for p in list(rng.choice(len(shapes), 6, replace=False)) + [int(np.argmax([m * n for m, n in shapes]))]:
        _check_problem(plan.block(int(p)).cpu().numpy(), plan, int(p), 1e-6, 0)


def test_batched_variants_bit_identical_and_autotune(lib):
    """Every launch variant (loads in flight per thread) gives the same bits;
    the autotuner keeps the fastest and rsvd_batched launches it."""
    import torch
    blocks = [kernel_block(b, seed=4001) for b in range(40, 64)]
    plan = _plan(lib, blocks)
    h = lib.handle()
    nv = lib.rsvd_batched_variants()
    assert nv >= 2
    with pytest.raises(lib.RsvdError):
        lib.rsvd_batched_set_variant(h, nv)
    outs = []
    try:
        for v in range(nv):
            lib.rsvd_batched_set_variant(h, v)
            assert lib.rsvd_batched_get_variant(h) == v
            assert lib.batched_run(plan, 1e-6, seed=3, flags=lib.RSVD_FLAG_SYNC) == lib.RSVD_OK
            outs.append([t.clone() for t in (plan.U, plan.D, plan.V, plan.rank, plan.err, plan.status)])
        for o in outs[1:]:
            for a, b in zip(outs[0], o):
                assert torch.equal(a, b)
        var, ms = lib.batched_autotune(plan, 1e-6, seed=3)
        assert 0 <= var < nv and len(ms) == nv and all(x > 0 for x in ms) and ms[var] == min(ms)
        assert lib.rsvd_batched_get_variant(h) == var
        for a, b in zip(outs[0], (plan.U, plan.D, plan.V, plan.rank, plan.err, plan.status)):
            assert torch.equal(a, b)
    finally:
        lib.rsvd_batched_set_variant(h, -1)
    _check_problem(blocks[0], plan, 0, 1e-6, 3)
