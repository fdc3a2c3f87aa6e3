"""Seeded synthetic inputs for the randomized-SVD workloads.

This module is shared by the tests, the oracle side and the GPU side.  It only
*synthesizes matrices*; it holds none of the method's arithmetic (no sketch, no
orthonormalization of samples, no SVD of B).  Haar-random orthonormal factors
are made the textbook way: QR of a Gaussian matrix with the diagonal of R made
positive (Mezzadri, "How to generate random matrices from the classical compact
groups", Notices AMS 2007).

Workload families (sizes are parameters; the defaults are the full sizes):

* ``exp_decay_matrix``   A = U diag(sigma) V^T, sigma_j = exp(-j/10),
                         2000 x 1000, float64.
* ``poly_decay_matrix``  A = U diag(sigma) V^T, Haar U, V, sigma_j = j^-1.5,
                         32768 x 32768, float32.
* ``pca_matrix``         rank-64 signal (orthonormalized Gaussian factors,
                         singular values linear 100 -> 1) + iid N(0, 1e-6) noise,
                         column-centred, 1,048,576 x 4096, float32.
* ``kernel_blocks``      4096 blocks 1/|x_i - y_j| between point clouds in unit
                         cubes whose centres are 3 apart, m, n ~ U{64..1024}.
* ``controller_matrix``  the learned-controller stream: square n x n, n
                         log-uniform, spectra exp(-j/r), j^-alpha or a step,
                         with permuted, signed DCT-II factors.

Numpy generators (``numpy.random.default_rng(seed)``) are used for anything the
CPU oracle must reproduce; the full-size float32 matrices are synthesized with
torch on the device (seeded torch generator), because their QR factors are
out of reach of a CPU.
"""
import math
import numpy as np


# ---------------------------------------------------------------- spectra ---
def exp_spectrum(r, rate=10.0):
    j = np.arange(1, r + 1, dtype=np.float64)
    return np.exp(-j / rate)


def poly_spectrum(r, alpha=1.5):
    j = np.arange(1, r + 1, dtype=np.float64)
    return j ** (-alpha)


def step_spectrum(r, rank, floor=1e-6):
    s = np.full(r, floor, dtype=np.float64)
    s[:rank] = 1.0
    return s


# ------------------------------------------------------- numpy factors ------
def haar_np(rng, m, r):
    """m x r matrix with orthonormal columns, Haar-distributed (Mezzadri)."""
    G = rng.standard_normal((m, r))
    Q, R = np.linalg.qr(G, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def lowrank_np(m, n, sigma, seed):
    """A = U diag(sigma) V^T (float64) with Haar U (m x r), V (n x r), r = len(sigma)."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    U = haar_np(rng, m, r)
    V = haar_np(rng, n, r)
    return (U * np.asarray(sigma)[None, :]) @ V.T


def exp_decay_matrix(m=2000, n=1000, seed=1001):
    """A = U diag(exp(-j/10)) V^T, U, V from QR of seeded Gaussians; float64."""
    return lowrank_np(m, n, exp_spectrum(min(m, n)), seed)


def poly_decay_matrix_np(m, n, seed, alpha=1.5, dtype=np.float32):
    """Small-size (CPU) instance of the polynomial-decay family."""
    return lowrank_np(m, n, poly_spectrum(min(m, n), alpha), seed).astype(dtype)


def exact_rank_matrix(m, n, rank, seed, cond=10.0):
    """Exactly rank-`rank` matrix with singular values spread over [1/cond, 1]."""
    s = np.geomspace(1.0, 1.0 / cond, rank) if rank > 0 else np.zeros(0)
    return lowrank_np(m, n, s, seed)


def spd_matrix_np(n, seed, alpha=1.5, dtype=np.float64):
    """Symmetric positive definite A = V diag(j^-alpha) V^T, V Haar (numpy)."""
    rng = np.random.default_rng(seed)
    V = haar_np(rng, n, n)
    lam = np.arange(1, n + 1, dtype=np.float64) ** (-alpha)
    A = (V * lam[None, :]) @ V.T
    return (0.5 * (A + A.T)).astype(dtype)


def pca_matrix_np(m, n, seed, rank=64, noise=1e-3, dtype=np.float32):
    """Small-size (CPU) instance of the PCA family, column-centred in float64."""
    rng = np.random.default_rng(seed)
    U = haar_np(rng, m, rank)
    V = haar_np(rng, n, rank)
    s = np.linspace(100.0, 1.0, rank)
    A = (U * s[None, :]) @ V.T + noise * rng.standard_normal((m, n))
    A -= A.mean(axis=0, keepdims=True)
    return A.astype(dtype)


# ------------------------------------------------------ torch (device) ------
def _torch():
    import torch
    return torch


def haar_torch(m, r, gen, device, dtype):
    torch = _torch()
    G = torch.randn(m, r, generator=gen, device=device, dtype=dtype)
    Q, R = torch.linalg.qr(G, mode="reduced")
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1
    del G, R
    return Q * d[None, :]


def poly_decay_matrix(m=32768, n=32768, seed=2001, alpha=1.5, device="cuda"):
    """Full-size polynomial-decay matrix, float32, synthesized on `device`.

    A = U diag(j^-alpha) V^T with Haar U (m x r), V (n x r), r = min(m, n); the
    product is taken in float32 without TF32.
    """
    torch = _torch()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    r = min(m, n)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        U = haar_torch(m, r, gen, device, torch.float32)
        s = torch.arange(1, r + 1, device=device, dtype=torch.float64).pow(-alpha).to(torch.float32)
        U.mul_(s[None, :])
        V = haar_torch(n, r, gen, device, torch.float32)
        A = U @ V.T
        del U, V
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return A.contiguous()


def exp_decay_matrix_torch(m, n, seed, rate=20.0, device="cuda"):
    """A = U diag(exp(-j / rate)) V^T, float32, Haar U, V (QR of seeded torch
    Gaussians, sign-fixed), synthesized on `device` without TF32."""
    torch = _torch()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    r = min(m, n)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        U = haar_torch(m, r, gen, device, torch.float32)
        s = torch.exp(-torch.arange(1, r + 1, device=device, dtype=torch.float64) / rate).to(torch.float32)
        U.mul_(s[None, :])
        V = haar_torch(n, r, gen, device, torch.float32)
        A = U @ V.T
        del U, V
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return A.contiguous()


def spd_matrix(n=16384, seed=5001, alpha=1.5, device="cuda"):
    """Symmetric positive definite A = V diag(j^-alpha) V^T, float32, Haar V,
    synthesized on `device` (products in float32 without TF32), then made
    exactly symmetric."""
    torch = _torch()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        V = haar_torch(n, n, gen, device, torch.float32)
        lam = torch.arange(1, n + 1, device=device, dtype=torch.float64).pow(-alpha).to(torch.float32)
        A = (V * lam[None, :]) @ V.T
        del V
        A = 0.5 * (A + A.T)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return A.contiguous()


def pca_matrix(m=1 << 20, n=4096, seed=3001, rank=64, noise=1e-3, device="cuda"):
    """Full-size PCA matrix, float32, synthesized on `device`, column-centred
    with float64 column means."""
    torch = _torch()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    U = haar_torch(m, rank, gen, device, torch.float32)
    V = haar_torch(n, rank, gen, device, torch.float32)
    s = torch.linspace(100.0, 1.0, rank, device=device, dtype=torch.float32)
    A = torch.randn(m, n, generator=gen, device=device, dtype=torch.float32)
    A.mul_(noise)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        A.addmm_(U * s[None, :], V.T)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    mean = A.sum(dim=0, dtype=torch.float64) / m
    A.sub_(mean.to(torch.float32)[None, :])
    return A


def column_offsets(n, seed, scale, device="cuda"):
    """Seeded column offsets mu_j ~ N(0, scale^2) (float32, length n) to add to
    a centred matrix, so that a solver's implicit centring has means to
    remove (PCA data is not centred when it arrives)."""
    torch = _torch()
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    return scale * torch.randn(n, generator=gen, device=device, dtype=torch.float32)


# ------------------------------------------------------- kernel blocks ------
def block_seed(seed, b):
    """Per-block seed: SplitMix64 of (seed, block id)."""
    z = (int(seed) * 0x9E3779B97F4A7C15 + (b + 1) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def kernel_block_points(b, seed=4001, lo=64, hi=1024):
    """Point clouds of block b: x_i ~ U([0,1]^3) (m points) and
    y_j ~ U([0,1]^3) + (3, 0, 0) (n points), m, n ~ U{lo..hi}."""
    rng = np.random.default_rng(block_seed(seed, b))
    m = int(rng.integers(lo, hi + 1))
    n = int(rng.integers(lo, hi + 1))
    x = rng.random((m, 3))
    y = rng.random((n, 3)) + np.array([3.0, 0.0, 0.0])
    return x, y


def kernel_block(b, seed=4001, lo=64, hi=1024, dtype=np.float32):
    """Block b of the batched workload: A_ij = 1 / |x_i - y_j| (binary64, then
    rounded to dtype) for the point clouds of kernel_block_points."""
    x, y = kernel_block_points(b, seed, lo, hi)
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt((d[:, :, 0] * d[:, :, 0] + d[:, :, 1] * d[:, :, 1]) + d[:, :, 2] * d[:, :, 2])
    return (1.0 / r).astype(dtype)


def kernel_block_torch(b, out, seed=4001, lo=64, hi=1024):
    """kernel_block(b) formed on out's device into the float32 tensor `out`
    (m x n), with the same binary64 operations in the same order."""
    torch = _torch()
    x, y = kernel_block_points(b, seed, lo, hi)
    xt = torch.from_numpy(x).to(out.device)
    yt = torch.from_numpy(y).to(out.device)
    d = xt[:, None, :] - yt[None, :, :]
    r = torch.sqrt((d[:, :, 0] * d[:, :, 0] + d[:, :, 1] * d[:, :, 1]) + d[:, :, 2] * d[:, :, 2])
    out.copy_((1.0 / r).to(torch.float32))
    return out


def kernel_blocks(count=4096, seed=4001, lo=64, hi=1024, dtype=np.float32):
    return [kernel_block(b, seed, lo, hi, dtype) for b in range(count)]


def kernel_block_shapes(count=4096, seed=4001, lo=64, hi=1024):
    out = []
    for b in range(count):
        rng = np.random.default_rng(block_seed(seed, b))
        out.append((int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))))
    return out


# ------------------------------------------------- controller stream -------
CONTROLLER_KINDS = ("exp", "poly", "step")


def controller_case(seed, lo=512, hi=16384):
    """One matrix of the controller stream: size n log-uniform in [lo, hi]
    (square), spectrum drawn uniformly among exp(-j/r) (r ~ U{16..256}),
    j^-alpha (alpha ~ U[0.5, 2]) and a step at rank r ~ U{16..256} followed
    by 1e-6.  Returns (n, sigma (length n), kind, parameter)."""
    rng = np.random.default_rng(int(seed))
    n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    n = max(lo, min(hi, n))
    kind = CONTROLLER_KINDS[int(rng.integers(0, 3))]
    j = np.arange(1, n + 1, dtype=np.float64)
    if kind == "exp":
        r = int(rng.integers(16, 257))
        return n, np.exp(-j / r), kind, float(r)
    if kind == "poly":
        alpha = float(rng.uniform(0.5, 2.0))
        return n, j ** (-alpha), kind, alpha
    r = int(rng.integers(16, 257))
    s = np.full(n, 1e-6)
    s[:min(r, n)] = 1.0
    return n, s, kind, float(r)


def dct_factor_np(rng, n):
    """Orthonormal n x n factor: the orthonormal DCT-II matrix with its rows
    randomly permuted and signed (a cheap dense stand-in for a Haar factor;
    the randomized range finder's error law under a Gaussian test matrix
    depends only on the singular values)."""
    k = np.arange(n, dtype=np.float64)[:, None]
    i = np.arange(n, dtype=np.float64)[None, :]
    C = np.sqrt(2.0 / n) * np.cos(np.pi * (2.0 * i + 1.0) * k / (2.0 * n))
    C[0, :] *= 1.0 / np.sqrt(2.0)
    perm = rng.permutation(n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return C.T[perm, :] * sign[:, None]


def controller_matrix_np(seed, lo=512, hi=16384, dtype=np.float32):
    """Dense A = U diag(sigma) V^T of controller_case(seed), U and V from
    dct_factor_np, formed in float64 and rounded to dtype."""
    n, sig, kind, par = controller_case(seed, lo, hi)
    rng = np.random.default_rng(int(seed) + 7919)
    U = dct_factor_np(rng, n)
    V = dct_factor_np(rng, n)
    return ((U * sig[None, :]) @ V.T).astype(dtype), (n, kind, par)


def controller_matrix(seed, lo=512, hi=16384, device="cuda"):
    """controller_matrix_np(seed) synthesized on `device` as float32: the
    same factors, formed with torch in float64 up to n = 4096 and in float32
    (without TF32) above."""
    torch = _torch()
    n, sig, kind, par = controller_case(seed, lo, hi)
    rng = np.random.default_rng(int(seed) + 7919)
    perm_u = rng.permutation(n)
    sign_u = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    perm_v = rng.permutation(n)
    sign_v = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    k = torch.arange(n, dtype=torch.float64, device=device)[:, None]
    i = torch.arange(n, dtype=torch.float64, device=device)[None, :]
    C = math.sqrt(2.0 / n) * torch.cos(math.pi * (2.0 * i + 1.0) * k / (2.0 * n))
    C[0, :] *= 1.0 / math.sqrt(2.0)
    Ct = C.T.contiguous()
    del C
    U = Ct[torch.from_numpy(perm_u).to(device), :] * torch.from_numpy(sign_u).to(device)[:, None]
    V = Ct[torch.from_numpy(perm_v).to(device), :] * torch.from_numpy(sign_v).to(device)[:, None]
    del Ct
    U.mul_(torch.from_numpy(sig).to(device)[None, :])
    if n > 4096:
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            A = U.to(torch.float32) @ V.to(torch.float32).T
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
    else:
        A = (U @ V.T).to(torch.float32)
    del U, V
    return A, (n, kind, par)


def mlp_init(seed, d_in=17, hid=128, n_out=20):
    """Initial controller parameters (He-normal weights, zero biases) as one
    flat float64 array in the order W1, b1, W2, b2, W3, b3."""
    rng = np.random.default_rng(int(seed))
    W1 = rng.standard_normal((hid, d_in)) * math.sqrt(2.0 / d_in)
    W2 = rng.standard_normal((hid, hid)) * math.sqrt(2.0 / hid)
    W3 = rng.standard_normal((n_out, hid)) * math.sqrt(1.0 / hid)
    return np.concatenate([W1.ravel(), np.zeros(hid), W2.ravel(), np.zeros(hid), W3.ravel(), np.zeros(n_out)])
