"""The dense workloads at full size, through the calls the benchmark times
(rsvd_fixed_rank, rsvd_nystrom; the same sizes, precisions and launch
configuration), checked by properties that hold at any size because the
float64 oracle cannot run there:

* 32768 x 32768 polynomial decay (sigma_j = j^-1.5, Haar U and V), bf16
  tensor-core sketches, k = 200, p = 56, q = 2;
* 2^20 x 4096 PCA matrix (rank-64 signal 100 -> 1 plus N(0, 1e-6) noise,
  column-centred), e4m3 sketches, k = 64, p = 64, q = 1;
* 16384 x 16384 SPD matrix V diag(j^-1.5) V^T, Nystrom, binary32 (its own
  test states its properties).

What is checked, and why it must hold:
* d_i <= sigma_i (1 + 1e-4): the computed values are the singular values of
  Q^T A, a compression of A, so they cannot exceed A's (up to the split-bf16
  projection's rounding, ~1e-8 here);
* d_i >= sigma_i (1 - 3%) for the poly matrix: the method's approximation
  error at l = 256, q = 2 (Sec. 8.1; 0.8% measured);
* Eckart-Young: the Frobenius residual is at least the optimum over all
  rank-k matrices, and the method stays within 1% of it;
* ||(A - U D V^T) v_i|| / ||v_i|| is at most the spectral residual, about
  sigma_{k+1} here (checked at 2 sigma_{k+1} on sampled right singular
  vectors; for orthonormal V the vector is A v_i - d_i u_i);
* U^T U = V^T V = I to binary32 accuracy (the lift is a binary32 product);
* PCA: against the exact singular values of the generated matrix (float64
  A^T A and its eigenvalues), for the e4m3, bf16 and binary32 paths alike;
  its own docstring states the bounds.
"""
import pytest

pytestmark = pytest.mark.gpu


def _fro_residual(A, U, D, V, rows=4096):
    """||A - U diag(D) V^T||_F and ||A||_F, blockwise in float64 on the device."""
    f2, a2 = 0.0, 0.0
    Ud = U.double() * D[None, :]
    Vd = V.double()
    for r0 in range(0, A.shape[0], rows):
        Ab = A[r0:r0 + rows].double()
        R = Ab - Ud[r0:r0 + rows] @ Vd.T
        f2 += float((R * R).sum())
        a2 += float((Ab * Ab).sum())
        del Ab, R
    return f2 ** 0.5, a2 ** 0.5


def _orth_err(X):
    """max |X^T X - I| in float64."""
    import torch
    Xd = X.double()
    G = Xd.T @ Xd
    return float((G - torch.eye(G.shape[0], dtype=G.dtype, device=G.device)).abs().max())


def test_poly_decay_32768_bf16_full_size(lib):
    import torch
    from workloads import poly_decay_matrix
    m = n = 32768
    k, p, q = 200, 56, 2
    A = poly_decay_matrix(m, n, seed=2001, device="cuda")
    U, D, V = lib.fixed_rank(A, k, p, q, seed=2101, prec=lib.RSVD_MIXED_BF16)
    torch.cuda.synchronize()
    sig = torch.arange(1, min(m, n) + 1, dtype=torch.float64, device="cuda").pow(-1.5)
    d = D.double()
    assert bool((d[:-1] >= d[1:]).all())
    assert bool((d <= sig[:k] * (1 + 1e-4)).all()), float((d / sig[:k]).max())
    assert bool((d >= sig[:k] * (1 - 0.03)).all()), float((1 - d / sig[:k]).max())
    assert _orth_err(U) < 1e-4 and _orth_err(V) < 1e-4
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        idx = torch.tensor([0, 1, 49, 99, 150, 199], device="cuda")
        Vs = V[:, idx]
        R = A @ Vs - U @ (D.float()[:, None] * (V.T @ Vs))     # (A - U D V^T) v_i
        r = R.double().norm(dim=0) / Vs.double().norm(dim=0)
        assert float(r.max()) <= 2 * float(sig[k]), float(r.max() / sig[k])
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    res, fro_a = _fro_residual(A, U, D, V)
    opt = float(sig[k:].pow(2).sum().sqrt())
    # ||A||_F of the binary32 matrix agrees with the construction's to rounding
    assert abs(fro_a - float(sig.pow(2).sum().sqrt())) < 1e-4 * fro_a
    assert opt * (1 - 1e-4) <= res <= 1.01 * opt, (res, opt)
    del A, U, D, V, R
    torch.cuda.empty_cache()


def _exact_sigma(A, rows=65536):
    """Singular values of A (float32 on the device) from A^T A formed in
    float64 blockwise and eigvalsh, descending: exact to about 1e-16 ||A||^2
    in the squares, far below every tolerance checked here."""
    import torch
    n = A.shape[1]
    G = torch.zeros(n, n, dtype=torch.float64, device=A.device)
    for r0 in range(0, A.shape[0], rows):
        Ab = A[r0:r0 + rows].double()
        G.addmm_(Ab.T, Ab)
        del Ab
    lam = torch.linalg.eigvalsh(G).flip(0).clamp_min(0)
    del G
    return lam.sqrt(), lam


def test_pca_2p20x4096_e4m3_full_size(lib):
    """The PCA workload through the benchmark's call, e4m3 sketches, with the
    bf16 and binary32 paths on the same matrix beside it, against the exact
    singular values of the generated A (not its construction values: the noise
    moves those by about eta^2 (m + n) / (2 sigma)).

    * d_i <= sigma_i (interlacing: the d_i are the singular values of Q^T A,
      Sec. 3 Remark 3.2), up to the projection's rounding;
    * for the 48 strongest directions the method's own error is second order
      in the angle between the signal direction and range(Q), sin^2 theta <=
      (1.09 / 26)^(2 (2q + 1)) < 1e-8 (the noise's singular values end at
      eta (sqrt m + sqrt n) = 1.09, the 48th signal value is 26), so what
      remains is rounding: on the binary32 path |d_i - sigma_i| <= 1e-5
      sigma_i (the tolerance stated for that path; 7.7e-6 measured); on the
      mixed paths the split-bf16 projection perturbs B = Q^T A by about 2^-16
      of ||A||_2 (pair representation 2^-17 per operand, the dropped Al^T Ql
      term 2^-18, the tensor core's truncating accumulation bounded by
      1024-element segments), so |d_i - sigma_i| <= 5e-5 sigma_1 (1.5e-5
      sigma_1 measured);
    * Eckart-Young: the Frobenius residual is at least the optimum
      sqrt(sum_{i > k} lambda_i) over rank-k matrices and within 0.5% of it
      (the weakest signal directions, sigma ~ 1.4 .. 5.8, lie at the noise
      edge, which q = 1 separates only partly);
    * U^T U = V^T V = I to binary32 accuracy.
    """
    import torch
    from workloads import pca_matrix
    m, n = 1 << 20, 4096
    k, p, q = 64, 64, 1
    A = pca_matrix(m, n, seed=3001, device="cuda")
    sig, lam = _exact_sigma(A)
    opt = float(lam[k:].sum().sqrt())
    for prec in (lib.RSVD_MIXED_FP8, lib.RSVD_MIXED_BF16, lib.RSVD_F32):
        U, D, V = lib.fixed_rank(A, k, p, q, seed=3101, prec=prec)
        torch.cuda.synchronize()
        d = D.double()
        assert bool((d[:-1] >= d[1:]).all())
        assert bool((d <= sig[:k] * (1 + 1e-5)).all()), (prec, float((d / sig[:k]).max()))
        err = (d[:48] - sig[:48]).abs()
        if prec == lib.RSVD_F32:
            assert float((err / sig[:48]).max()) <= 1e-5, (prec, float((err / sig[:48]).max()))
        else:
            assert float(err.max()) <= 5e-5 * float(sig[0]), (prec, float(err.max() / sig[0]))
        assert _orth_err(U) < 1e-4 and _orth_err(V) < 1e-4, prec
        res, _ = _fro_residual(A, U, D, V, rows=65536)
        assert opt * (1 - 1e-6) <= res <= 1.005 * opt, (prec, res / opt)
        del U, D, V
        torch.cuda.empty_cache()
    del A
    torch.cuda.empty_cache()


def test_nystrom_16384_f32_full_size(lib):
    """Fig. nystrom on the 16384^2 SPD workload (A = V diag(j^-1.5) V^T, Haar
    V), binary32, k = 200, p = 56, the benchmark's call.  The Nystrom
    approximation F F* lies below A in the Loewner order, so (i) each
    lambda_hat_i <= lambda_i and (ii) each Rayleigh quotient u_i^T A u_i >=
    lambda_hat_i, both up to binary32 rounding (1e-6 and 2e-5 of lambda_1
    allowed; the same steps in binary32 on the CPU at 4096^2 give -4e-9 for
    the second); without a power step the 200th value is 16% low (0.83 of
    lambda_200 from the float64 oracle at 4096^2), so 0.7 lambda_i is the
    lower bound; the residual on sampled u_i is at most the spectral residual
    (1.27 lambda_{k+1} from the oracle, 1.29 measured here)."""
    import torch
    from workloads import spd_matrix
    n, k, p = 16384, 200, 56
    A = spd_matrix(n, seed=5001, device="cuda")
    U, L = lib.nystrom(A, k, p, seed=5101, prec=lib.RSVD_F32)
    torch.cuda.synchronize()
    lam = torch.arange(1, n + 1, dtype=torch.float64, device="cuda").pow(-1.5)
    assert bool((L[:-1] >= L[1:]).all()) and bool((L > 0).all())
    assert bool((L <= lam[:k] * (1 + 1e-3) + 1e-6).all()), float((L / lam[:k]).max())
    assert bool((L >= 0.7 * lam[:k]).all()), float((L / lam[:k]).min())
    assert _orth_err(U) < 1e-4
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        AU = (A @ U).double()
        rho = (U.double() * AU).sum(dim=0)
        assert float((rho - L).min()) >= -2e-5, float((rho - L).min())
        idx = torch.tensor([0, 1, 49, 99, 150, 199], device="cuda")
        Ud = U.double()
        R = AU[:, idx] - Ud @ (L[:, None] * (Ud.T @ Ud[:, idx]))    # (A - U Lam U^T) u_i
        r = R.norm(dim=0) / Ud[:, idx].norm(dim=0)
        assert float(r.max()) <= 2 * float(lam[k]), float(r.max() / lam[k])
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del A, U, L, AU, R
    torch.cuda.empty_cache()
