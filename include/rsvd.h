/*
 * rsvd.h -- C ABI of the GB300 (sm_103a) randomized-SVD library.
 *
 * The library computes a rank-k approximate SVD  A ~= U diag(D) V^T  of a dense
 * m x n matrix by the randomized range finder with power iteration and
 * re-orthonormalization between products (Martinsson, "Randomized methods for
 * matrix computations", Sec. 8.1, Fig. "Accuracy enhanced randomized SVD (with
 * orthonormalization)"), followed by the Stage-B factorization of Sec. 3:
 *
 *   G = randn(n, l);  Q = orth(A G);
 *   repeat q times:  W = orth(A^T Q);  Q = orth(A W);
 *   B = Q^T A;  [Uhat, D, V] = svd(B);  U = Q Uhat;   keep the k leading triplets
 *
 * with l = k + p (Sec. 4, Remark "How many basis vectors").  The tolerance form
 * of the problem (Sec. 1.1: find k with ||A - U D V^T||_Fro <= eps) is solved by
 * the blocked greedy range finder of Sec. 12.3 (Fig. "greedy_blocked").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All matrices are ROW-MAJOR with a leading dimension (row stride, in
 *    elements) >= the number of columns.  A column-major caller passes A^T and
 *    swaps the roles of U and V.
 *  - Every pointer to matrix data is a DEVICE pointer on the handle's device,
 *    unless the parameter says "host".  All device buffers (inputs, outputs,
 *    workspace) are owned by the caller; A is never written.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL means
 *    the legacy default stream).  Calls return as soon as the work is enqueued
 *    unless RSVD_FLAG_SYNC is set.  Nothing allocates device memory on the
 *    solve path: all scratch comes from the caller's workspace, sized by
 *    rsvd_workspace_size().
 *  - Errors: invalid arguments are reported synchronously (RSVD_E_INVALID) and
 *    nothing is enqueued.  Numerical failures found on the device (Cholesky
 *    breakdown, non-finite values, non-convergence) are written to a status
 *    word inside the workspace; the first failure wins.  They are returned by
 *    the call itself when RSVD_FLAG_SYNC is set, or later by
 *    rsvd_query_status().  No call aborts or throws.
 *  - Not thread-safe per handle: one handle per host thread, or serialize.
 */
#ifndef RSVD_H
#define RSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsvd_handle_s* rsvd_handle_t;
typedef void* rsvd_stream_t; /* a cudaStream_t */

typedef enum {
  RSVD_OK = 0,
  RSVD_E_INVALID = 1,       /* bad argument; nothing was enqueued */
  RSVD_E_NOMEM = 2,         /* workspace too small, or host allocation failed */
  RSVD_E_CUDA = 3,          /* a CUDA runtime call failed (see rsvd_last_error_detail) */
  RSVD_E_BREAKDOWN = 4,     /* Cholesky pivot non-positive even after the shifted retries */
  RSVD_E_NOT_CONVERGED = 5, /* adaptive rank reached max_rank / min(m, n) above tolerance */
  RSVD_E_NONFINITE = 6,     /* NaN or Inf met in a Gram diagonal or a pivot */
  RSVD_E_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  RSVD_E_UNSUPPORTED = 8    /* valid request this build does not implement */
} rsvd_status;

/* Arithmetic of the solve (what A, U and V hold, and how the sketch products
 * are taken).  D is always double. */
typedef enum {
  RSVD_F64 = 0,        /* A, U, V double; every product in binary64 */
  RSVD_F32 = 1,        /* A, U, V float; plain binary32 SIMT products */
  RSVD_MIXED_BF16 = 2, /* A, U, V float; A*Omega, A^T Q, A W on tcgen05 tensor
                          cores with bf16 operands and fp32 accumulation; the
                          final B = Q^T A as a three-term split-bf16 product;
                          Gram matrices accumulated in binary64 */
  RSVD_MIXED_FP8 = 3,  /* A, U, V float; A*Omega, A^T Q, A W on tcgen05 tensor
                          cores with e4m3 operands (A scaled per row, the thin
                          operand per column; scales applied in the epilogue)
                          and fp32 accumulation; B = Q^T A as in
                          RSVD_MIXED_BF16 (three-term split bf16) */
  RSVD_MIXED_FP8_B128 = 4 /* as RSVD_MIXED_FP8 with one scale per block of 128
                          rows of A: r_b = 448 / max |A| over the block's rows
                          (binary32), found by one more read of A before the
                          conversion pass */
} rsvd_precision;

/* Element types for the stage entry points. */
typedef enum { RSVD_DT_F64 = 0, RSVD_DT_F32 = 1, RSVD_DT_BF16 = 2 } rsvd_dtype;

enum {
  RSVD_FLAG_RETURN_FULL_L = 1, /* return all l = k + p triplets instead of k */
  RSVD_FLAG_SYNC = 2,          /* block until the work ends; return the device status */
  RSVD_FLAG_CERTIFY = 4,       /* reserved; the a-posteriori certificate is rsvd_certify */
  RSVD_FLAG_USE_CONTROLLER = 8, /* rsvd_adaptive_tol: learned (l, q) controller */
  RSVD_FLAG_SPECTRAL = 16,      /* rsvd_adaptive_tol: spectral-norm stopping test (Sec. 13) */
  RSVD_FLAG_CENTER = 32,        /* rsvd_fixed_rank: factor the column-centred A - 1 mu^T (PCA) */
  RSVD_FLAG_KRYLOV = 64,        /* rsvd_fixed_rank: block Krylov basis, q counts blocks */
  RSVD_FLAG_SINGLE_PASS = 128,  /* rsvd_fixed_rank: single-pass SVD (sketches only, fitted core) */
  RSVD_FLAG_SYMMETRIC = 256,    /* with RSVD_FLAG_SINGLE_PASS: single-pass EVD of a symmetric A */
  RSVD_FLAG_SRFT = 512          /* rsvd_fixed_rank: SRFT test matrix; U, V complex */
};

typedef struct {
  int k;          /* target rank (fixed-rank solve), >= 1 */
  int p;          /* oversampling, >= 0; l = k + p <= min(m, n) and l <= 256 */
  int q;          /* power steps, >= 0 */
  int block;      /* adaptive block size b (0 -> 16) */
  int max_rank;   /* adaptive cap on the rank (0 -> min(m, n)) */
  int probe_cols; /* reserved (controller probe width) */
  double tol;     /* adaptive: relative Frobenius tolerance, eps = tol ||A||_Fro
                     (RSVD_FLAG_SPECTRAL: the absolute spectral tolerance eps) */
  uint64_t seed;  /* key of the Philox4x32-10 Gaussian stream */
  int prec;       /* rsvd_precision */
  int flags;      /* RSVD_FLAG_* */
} rsvd_params;

/* Handle: the device ordinal, its SM count and the library's small persistent
 * host state.  rsvd_create makes `device` current on the calling thread. */
rsvd_status rsvd_create(rsvd_handle_t* handle, int device);
rsvd_status rsvd_destroy(rsvd_handle_t handle);

/* Number of workspace bytes a solve of this shape and these parameters needs
 * (rsvd_fixed_rank when params->tol == 0, else rsvd_adaptive_tol).  The
 * workspace must be 256-byte aligned device memory. */
rsvd_status rsvd_workspace_size(rsvd_handle_t handle, int m, int n, const rsvd_params* params,
                                size_t* bytes);

/* Fixed-rank randomized SVD (Sec. 8.1, Fig. RSVDP_stabilized, + Sec. 3 Stage B).
 *   A, U, D, V may be device memory or host memory the device can access:
 *   pinned host memory (cudaHostAlloc / cudaHostRegister, mapped at the same
 *   address under unified addressing), or any host memory on devices with
 *   pageable-memory access; anything else is RSVD_E_INVALID.  The mixed
 *   paths (RSVD_MIXED_BF16, RSVD_MIXED_FP8) read A exactly once, in the
 *   conversion pass, so a host A costs one pass at the host link's bandwidth
 *   and no device copy; the binary32/64 paths read A 2q + 2 times.
 *   A  : m x n, lda >= n, double (RSVD_F64) or float (others).
 *   U  : m x kk output, ldu >= kk, same type as A;  kk = k, or l with
 *        RSVD_FLAG_RETURN_FULL_L.
 *   D  : kk doubles, descending.
 *   V  : n x kk output, ldv >= kk, same type as A.
 *   Each pair (u_i, v_i) is signed so that the largest-magnitude entry of v_i
 *   is positive (lowest index on ties).
 * The random test matrix is the Philox4x32-10 stream keyed by params->seed:
 * G(i, j) comes from counter (i / 4, j, 0, 0) through a 24-bit Box-Muller map
 * (see rsvd_gaussian).
 * RSVD_FLAG_CENTER (PCA, Sec. 1): factor the column-centred Abar = A - 1 mu^T,
 * mu = A^T 1 / m, without forming it: mu is one more read of A (binary64
 * sums), and every product carries its rank-one correction, Abar X = A X -
 * 1 (mu^T X) and Abar^T Y = A^T Y - mu (1^T Y).  Workspace grows by a few
 * vectors (rsvd_workspace_size with the flag set).
 * RSVD_FLAG_KRYLOV (Sec. "Extended sampling matrix"): params->q >= 1 counts
 * blocks; Q spans [A G, (A A^T) A G, ..., (A A^T)^(q-1) A G], w = q (k + p)
 * columns (w <= 256, 128 for RSVD_F64), Stage B on the w x n matrix B = Q^T A
 * (RSVD_FLAG_RETURN_FULL_L returns all w triplets).  Each block is formed
 * from the previous block's orthonormal basis and projected against the
 * blocks before it, which spans the same space in exact arithmetic.  Passes
 * over A: 2q.  Precisions RSVD_F64, RSVD_F32 and RSVD_MIXED_BF16 (k + p a
 * multiple of 8); not combined with RSVD_FLAG_CENTER.
 * RSVD_FLAG_SINGLE_PASS (Sec. "Single pass algorithms", Fig. singlepass_gen):
 * the sketches Yc = A Gc and Yr = A^T Gr (Gc the Omega stream, Gr Philox
 * stream 5) are the only products with A; Qc, Qr = the k dominant left
 * singular vectors of Yc, Yr; the k x k core C minimizes ||P C - R1||_F^2 +
 * ||C M - R2||_F^2 (P = Gr^T Qc, R1 = Yr^T Qr, M = Qr^T Gc, R2 = Qc^T Yc),
 * solved in binary64 as the Sylvester equation of its normal equations;
 * U = Qc Uhat, V = Qr Vhat from C = Uhat D Vhat^T.  q must be 0, k <= 128,
 * outputs k triplets.  The two sketches are separate launches (A is read
 * twice; nothing depends on a basis).  With RSVD_FLAG_SYMMETRIC (Fig.
 * singlepass_herm; A symmetric, m = n): Y = A G only, the symmetric core
 * minimizing ||C (Q^T G) - Q^T Y||_F (a Lyapunov equation), D receives the k
 * eigenvalues ordered by decreasing magnitude (signed), U the eigenvectors
 * (largest-magnitude entry positive) and V a copy of U.  Precisions RSVD_F64,
 * RSVD_F32, RSVD_MIXED_BF16 (bf16 tensor-core sketches, the rest binary32
 * and binary64).
 * RSVD_FLAG_SRFT (Sec. 6, eq. SRFT): Fig. RSVD (q must be 0) with Omega =
 * D F S instead of a Gaussian: D = diag(e^{i theta_j}), theta_j = 2 pi
 * (w >> 8) 2^-24 from word j mod 4 of Philox counter (j / 4, 0, 6, 0); F the
 * unitary n-point DFT; S the l columns with the smallest 64-bit keys
 * (w0 << 32 | w1 of counter (j, 0, 7, 0)), in key order.  For a real A the
 * factors are complex: U (m x kk) and V (n x kk) are COMPLEX outputs, pairs
 * (re, im) of A's element type, ldu and ldv counted in complex entries; D is
 * real; each pair is phased so that the largest-magnitude entry of v_i is
 * real and positive.  The complex steps run on the realification, so
 * 2 (k + p) <= 256 (128 for RSVD_F64).  Precisions RSVD_F64, RSVD_F32,
 * RSVD_MIXED_BF16. */
rsvd_status rsvd_fixed_rank(rsvd_handle_t handle, int m, int n, const void* A, int lda,
                            const rsvd_params* params, void* U, int ldu, double* D, void* V,
                            int ldv, void* workspace, size_t ws_bytes, rsvd_stream_t stream);

/* Eigenvalue decomposition of a symmetric positive semi-definite matrix by the
 * Nystrom method (Fig. nystrom): G = randn(n, l) (the Omega stream of
 * rsvd_fixed_rank), Y = A G, Q = orth(Y) (CholeskyQR2), B1 = A Q,
 * B2 = Q^T B1 (symmetrized), B2 = C^T C (Cholesky), F = B1 C^-1,
 * [U, Sigma, ~] = svd(F), Lambda = Sigma^2; A ~ U diag(Lambda) U^T =
 * (A Q)(Q^T A Q)^-1 (A Q)^T.  Two passes over A, like the basic RSVD, with
 * the accuracy of one more power step.  If Q^T A Q is singular to working
 * precision (rank(A) < l) the Cholesky fails after its shifted restarts and
 * the call reports RSVD_E_BREAKDOWN.
 *   A   : n x n, lda >= n, symmetric (both triangles are read); double
 *         (RSVD_F64) or float (RSVD_F32); device or device-accessible host memory.
 *   params: k, p (l = k + p <= n), seed; q must be 0; prec RSVD_F32 or
 *         RSVD_F64; flags RSVD_FLAG_RETURN_FULL_L (all l pairs), RSVD_FLAG_SYNC.
 *   U   : n x kk output, ldu >= kk, same type as A; the largest-magnitude entry
 *         of each u_i is positive.
 *   Lam : kk doubles, descending.
 * workspace: rsvd_workspace_size(handle, n, n, params) bytes, 256-byte aligned. */
rsvd_status rsvd_nystrom(rsvd_handle_t handle, int n, const void* A, int lda, const rsvd_params* params,
                         void* U, int ldu, double* Lam, void* workspace, size_t ws_bytes,
                         rsvd_stream_t stream);

/* Tolerance-driven randomized SVD (Sec. 12.3, Fig. greedy_blocked; stopping on
 * the Frobenius norm of the explicitly updated remainder, Sec. 12.4):
 * blocks of b Gaussian columns (Philox stream 1, block t = columns t*b ..)
 * are drawn until ||A - Q B||_Fro <= tol ||A||_Fro, then Stage B runs on B.
 * params->q in [0, 8] power steps per block (the power variant in the
 * caption of Fig. greedy_blocked: Y = (A_j A_j^T)^q A_j G, with orth between
 * products).
 * With RSVD_FLAG_USE_CONTROLLER (prec RSVD_F32 or RSVD_MIXED_BF16; m, n >= 16;
 * parameters attached by rsvd_controller_attach): a 16-column probe and the
 * network choose (l, q); rsvd_fixed_rank runs with k = l, p = 0 in `prec`;
 * the residual is estimated with 16 columns of Philox stream 2 (Sec. 14); if
 * the estimate meets the tolerance the result is truncated to the smallest
 * rank whose estimated error still meets it, otherwise (and if l < max_rank)
 * the plain binary32 adaptive range finder (q = 0) recomputes the result.
 * That path synchronizes the stream twice (to read the choice and the judge's
 * verdict).
 *   U, V : capacity max_rank columns (ldu, ldv >= max_rank).
 * With RSVD_FLAG_SPECTRAL (Sec. 13: the stopping test of Fig. adaptive2 and
 * Lemma thm:aposteriori with alpha = 1/10; q must be 0): tol is an ABSOLUTE
 * spectral-norm tolerance eps > 0.  Before block t is appended, its fresh
 * samples A_j G_t = (I - Q Q^T) A G_t are the b probes; if each has norm at
 * most eps / (10 sqrt(2/pi)), the loop stops without appending them, and then
 * ||A - Q B||_2 <= eps with probability at least 1 - 10^-b.  Otherwise the
 * block is appended exactly as in the Frobenius mode.
 *   rank_out : DEVICE int, receives the rank r (a multiple of b, or max_rank).
 *   err_out  : DEVICE double, receives ||A - Q B||_Fro / ||A||_Fro; in the
 *              spectral mode an absolute bound on ||A - Q B||_2 instead: the
 *              probe bound 10 sqrt(2/pi) max_i ||A_j g_i|| of the block that
 *              stopped the loop, or ||A - Q B||_Fro if the cap came first.
 * Entries of D, U, V beyond r are set to zero.  If the cap is hit first the
 * status is RSVD_E_NOT_CONVERGED and the outputs hold the rank-max_rank
 * factorization. */
rsvd_status rsvd_adaptive_tol(rsvd_handle_t handle, int m, int n, const void* A, int lda,
                              const rsvd_params* params, void* U, int ldu, double* D, void* V,
                              int ldv, int* rank_out, double* err_out, void* workspace,
                              size_t ws_bytes, rsvd_stream_t stream);

/* Batched tolerance-driven randomized SVD: `count` independent binary32
 * problems, each solved exactly as rsvd_adaptive_tol solves it (Sec. 12.3,
 * Fig. greedy_blocked, then Stage B of Sec. 3), all in ONE persistent kernel
 * launch: every CTA of the grid (one per SM) takes the next problem, largest
 * m n first, from a device-side queue.  The call enqueues one memset and two
 * kernels and never synchronizes (unless RSVD_FLAG_SYNC), so it can be
 * captured into a CUDA graph.
 *   count  : number of problems, 0 <= count <= 65536 (0 enqueues nothing).
 *   m, n, lda : DEVICE int arrays [count]; 1 <= m, n <= 1024, lda >= n.
 *   A      : DEVICE array [count] of device pointers to float m x n (row-major).
 *   U, V   : DEVICE arrays [count] of device pointers to float outputs of
 *            m x R and n x R, row-major with leading dimension exactly R.
 *   D      : DEVICE array [count] of device pointers to R doubles.
 *   rank_out, status_out : DEVICE int arrays [count] (may be NULL).
 *   err_out: DEVICE double array [count], ||A - Q B||_Fro / ||A||_Fro (may be NULL).
 * params: prec must be RSVD_F32, q must be 0, tol in (0, 1), block b in
 * [1, 16] (0 -> 16), max_rank R in [1, 64] (0 -> 64); problem p caps its rank
 * at min(R, m_p, n_p) and draws its Gaussian blocks from the Philox stream
 * keyed by params->seed + p.  Entries of D, U, V beyond the rank are zero.
 * Per-problem failures (sizes out of range, NULL pointers: RSVD_E_INVALID;
 * breakdown, non-finite values, rank cap reached) go to status_out[p] and the
 * first of them to the workspace status word. */
rsvd_status rsvd_batched_workspace_size(rsvd_handle_t handle, int count, const rsvd_params* params,
                                        size_t* bytes);
rsvd_status rsvd_batched(rsvd_handle_t handle, int count, const int* m, const int* n,
                         const void* const* A, const int* lda, const rsvd_params* params,
                         void* const* U, double* const* D, void* const* V, int* rank_out,
                         double* err_out, int* status_out, void* workspace, size_t ws_bytes,
                         rsvd_stream_t stream);

/* Launch variants of rsvd_batched and their autotuner.  A variant fixes how
 * many loads each thread keeps in flight in the passes over a problem's
 * matrix (rows ahead in the column-owned passes, columns ahead in the row-
 * owned ones); the arithmetic and its order are the same in every variant,
 * so all variants produce bit-identical outputs and the choice affects only
 * time.  rsvd_batched uses the handle's variant (the library default until
 * one is set).
 *   rsvd_batched_variants: *count = number of variants.
 *   rsvd_batched_variant_info: rows and columns ahead of variant v.
 *   rsvd_batched_set_variant: v in [0, count) or -1 (library default).
 *   rsvd_batched_get_variant: the variant rsvd_batched will launch.
 *   rsvd_batched_autotune: same arguments as rsvd_batched; runs the batch
 *     twice per variant on `stream` (the second run timed with CUDA events),
 *     stores the fastest variant in the handle, writes it to *variant_out
 *     (host, may be NULL) and each variant's time in ms to ms_out (host
 *     array of `count` variants, may be NULL).  It synchronizes, so it must
 *     not be called while `stream` is being captured.  The outputs hold the
 *     batch's result afterwards; a per-problem failure is returned as for
 *     rsvd_batched with RSVD_FLAG_SYNC. */
rsvd_status rsvd_batched_variants(int* count);
rsvd_status rsvd_batched_variant_info(int variant, int* rows_ahead, int* cols_ahead);
rsvd_status rsvd_batched_set_variant(rsvd_handle_t handle, int variant);
rsvd_status rsvd_batched_get_variant(rsvd_handle_t handle, int* variant);
rsvd_status rsvd_batched_autotune(rsvd_handle_t handle, int count, const int* m, const int* n,
                                  const void* const* A, const int* lda, const rsvd_params* params,
                                  void* const* U, double* const* D, void* const* V, int* rank_out,
                                  double* err_out, int* status_out, void* workspace, size_t ws_bytes,
                                  rsvd_stream_t stream, float* ms_out, int* variant_out);

/* Reads the device status word of the last solve that used `workspace`
 * (synchronizes `stream` first).  *status receives an rsvd_status value. */
rsvd_status rsvd_query_status(rsvd_handle_t handle, const void* workspace, int* status,
                              rsvd_stream_t stream);

/* Copies a human-readable description of the last synchronous error on this
 * handle into buf (always NUL-terminated when len > 0). */
rsvd_status rsvd_last_error_detail(rsvd_handle_t handle, char* buf, size_t len);

/* ---------------------------------------------------------------------------
 * Stage entry points: single steps of the path, for composition and testing.
 * ------------------------------------------------------------------------- */

/* Raw Philox4x32-10 words (Salmon et al., SC'11) behind the Gaussian stream:
 * out[(j * n_groups + g) * 4 + w] = word w of counter (g, col0 + j, stream_id, 0)
 * under key (seed mod 2^32, seed div 2^32), for g < n_groups, j < l. */
rsvd_status rsvd_philox_words(rsvd_handle_t handle, int n_groups, int l, uint64_t seed,
                              uint32_t stream_id, int col0, uint32_t* out, rsvd_stream_t stream);

/* Gaussian test matrix (the paper's randn that draws G in Fig. RSVD): out is n x l,
 * row-major with leading dimension ldo >= l, element type `dtype`.
 * Entry (i, j) uses counter (i / 4, col0 + j, stream_id, 0); its words
 * (w0, w1) serve rows 4g, 4g+1 and (w2, w3) rows 4g+2, 4g+3 through
 * v = w >> 8, u1 = (v_a + 1) 2^-24, u2 = v_b 2^-24,
 * z = sqrt(-2 ln u1) * (cos | sin)(2 pi u2).  binary32/bf16 outputs are
 * computed in binary32, binary64 outputs in binary64. */
rsvd_status rsvd_gaussian(rsvd_handle_t handle, int n, int l, uint64_t seed, uint32_t stream_id,
                          int col0, int dtype, void* out, int ldo, rsvd_stream_t stream);

/* One sketch product (A G, A^T Q, A W of Fig. RSVDP_stabilized):
 *   trans = 0:  Y (m x l) = A (m x n) X (n x l)
 *   trans = 1:  Y (n x l) = A^T (n x m) X (m x l)
 * A row-major m x n (lda).  prec RSVD_F64: A, X, Y double; RSVD_F32: float
 * (SIMT fp32); RSVD_MIXED_BF16: A and X bf16 (raw 16-bit storage), Y float,
 * tcgen05 tensor-core product with fp32 accumulation; RSVD_MIXED_FP8: A, X, Y
 * float, the library converts A to e4m3 per row (r_i = 448 / max_j |A_ij|
 * in binary32, A8 = e4m3(A_ij r_i) rounded to nearest, saturating) and the
 * thin operand per column the same way, after scaling its rows by 1 / r_i
 * when trans = 1 (A^T Q = A8^T (S Q)); the e4m3 product (tcgen05
 * kind::f8f6f4, fp32 accumulation) is then rescaled.  Needs workspace
 * (rsvd_sketch_workspace_size) for split-K partial sums and the 8-bit copies. */
rsvd_status rsvd_sketch_workspace_size(rsvd_handle_t handle, int prec, int trans, int m, int n,
                                       int l, size_t* bytes);
rsvd_status rsvd_sketch(rsvd_handle_t handle, int prec, int trans, int m, int n, int l,
                        const void* A, int lda, const void* X, int ldx, void* Y, int ldy,
                        void* workspace, size_t ws_bytes, rsvd_stream_t stream);

/* Projection B = Q^T A of Stage B (Sec. 3; Fig. RSVDP_stabilized),
 * returned transposed:  Bt (n x l, row-major, ldb) = A^T Q  for A m x n (lda)
 * and Q m x l (ldq).  RSVD_F64: double; RSVD_F32: float, SIMT; RSVD_MIXED_BF16:
 * A and Q float, each split into a bf16 pair (x = hi + lo) and
 * Bt = Ah^T Qh + Ah^T Ql + Al^T Qh on tcgen05 tensor cores (relative error
 * about 2^-16 instead of bf16's 2^-8). */
rsvd_status rsvd_project_workspace_size(rsvd_handle_t handle, int prec, int m, int n, int l, size_t* bytes);
rsvd_status rsvd_project(rsvd_handle_t handle, int prec, int m, int n, int l, const void* A, int lda,
                         const void* Q, int ldq, void* Bt, int ldb, void* workspace, size_t ws_bytes,
                         rsvd_stream_t stream);

/* Diagnostics.  rsvd_kernel_launches: number of kernels this library has
 * enqueued (through any handle) since it was loaded.  rsvd_profile: while
 * enabled (on != 0) every tensor-core sketch product (kind 0) and
 * split-bf16 projection (kind 1) enqueued through `handle` is bracketed by a
 * pair of CUDA events on its stream; rsvd_profile_read waits for the recorded
 * events, returns the summed device time in milliseconds and the number of
 * launches of that kind, and clears them. */
rsvd_status rsvd_kernel_launches(rsvd_handle_t handle, long long* count);
rsvd_status rsvd_profile(rsvd_handle_t handle, int on);
rsvd_status rsvd_profile_read(rsvd_handle_t handle, int kind, double* total_ms, long long* launches);

/* ---------------------------------------------------------------------------
 * Learned (l, q) controller (the paper has no learned component; the probe is
 * Fig. RSVD of Sec. 4 with l = 16, the labels come from the tolerance-driven
 * range finder of Sec. 12.3, Fig. greedy_blocked, and the judge is the
 * a-posteriori estimate of Sec. 13-14, eq. (infomm) and Lemma
 * thm:aposteriori).
 *
 * Network: x (17 floats) -> h1 = relu(W1 x + b1) (128) -> h2 = relu(W2 h1 + b2)
 * (128) -> z = W3 h2 + b3 (20).  z[0..15] are the logits of l = 16 (c + 1),
 * c = 0..15; z[16..19] the logits of q = 0..3.  The parameters are one
 * DEVICE array of RSVD_CTRL_PARAMS floats: W1 (128 x 17, row-major
 * [out][in]), b1 (128), W2 (128 x 128), b2 (128), W3 (20 x 128), b3 (20).
 * The caller owns it (the handle only keeps the pointer).
 * Features x: log10(sigma_i / sigma_1) of the probe Y = A G (G = the first 16
 * columns of the Omega stream of rsvd_fixed_rank), i = 2..16, clipped below at
 * -3, then log2(m) / 16 and log2(n) / 16.
 * ------------------------------------------------------------------------- */
#define RSVD_CTRL_D_IN 17
#define RSVD_CTRL_HIDDEN 128
#define RSVD_CTRL_OUT 20
#define RSVD_CTRL_PARAMS 21396

/* Probe features of a float m x n matrix A (lda), m, n >= 16:
 *   feat : DEVICE float[17] (the network input above);
 *   fro2 : DEVICE double, ||A||_F^2 (may be NULL).
 * One pass over A (the 16-column sketch and the squares are fused). */
rsvd_status rsvd_probe_workspace_size(rsvd_handle_t handle, int m, int n, size_t* bytes);
rsvd_status rsvd_probe_features(rsvd_handle_t handle, int m, int n, const float* A, int lda, uint64_t seed,
                                float* feat, double* fro2, void* workspace, size_t ws_bytes, rsvd_stream_t stream);

/* Network evaluation and training on the GPU.  X: DEVICE batch x 17 floats;
 * yl: DEVICE int[batch], l classes in [0, 15]; yq: DEVICE int[batch], q in
 * [0, 3] (labels outside these ranges are clamped into them); lam >= 0: weight of the penalty on the probability of a too small l.
 * Loss (mean over the batch):
 *   -log p_l[yl] - log p_q[yq] + lam * sum_{c < yl} p_l[c],  p = softmax per head.
 *   rsvd_mlp_forward   : logits (DEVICE batch x 20); needs no workspace.
 *   rsvd_mlp_grad      : grad (DEVICE RSVD_CTRL_PARAMS floats) of the loss,
 *                        loss (DEVICE double).
 *   rsvd_mlp_train_step: one Adam step (Kingma and Ba 2015; beta1 0.9, beta2
 *                        0.999, eps 1e-8, step >= 1) on theta with moments m1,
 *                        m2 (DEVICE, RSVD_CTRL_PARAMS floats each, zero before
 *                        step 1); loss (DEVICE double, may be NULL) receives
 *                        the loss before the step.
 * Gradients are summed over CTAs in a fixed order: results are reproducible. */
rsvd_status rsvd_mlp_workspace_size(rsvd_handle_t handle, int batch, size_t* bytes);
rsvd_status rsvd_mlp_forward(rsvd_handle_t handle, int batch, const float* X, const float* theta, float* logits,
                             rsvd_stream_t stream);
rsvd_status rsvd_mlp_grad(rsvd_handle_t handle, int batch, const float* X, const int* yl, const int* yq, float lam,
                          const float* theta, float* grad, double* loss, void* workspace, size_t ws_bytes,
                          rsvd_stream_t stream);
rsvd_status rsvd_mlp_train_step(rsvd_handle_t handle, int batch, const float* X, const int* yl, const int* yq,
                                float lam, float* theta, float* m1, float* m2, int step, float lr, double* loss,
                                void* workspace, size_t ws_bytes, rsvd_stream_t stream);

/* Attaches trained parameters (DEVICE, caller-owned, kept alive by the caller
 * while attached; NULL detaches) to the handle for rsvd_adaptive_tol with
 * RSVD_FLAG_USE_CONTROLLER.  quantile in (0, 1]: l is the smallest class whose
 * cumulative probability reaches it (larger = more conservative); safety in
 * (0, 1]: a prediction is accepted when the residual estimate is at most
 * safety * tol * ||A||_F. */
rsvd_status rsvd_controller_attach(rsvd_handle_t handle, const float* theta, double quantile, double safety);

/* What a controlled solve does when the judge rejects the network's (l, q):
 * mode 0 (default): the blocked adaptive range finder (Sec. 12.3) recomputes
 * the result from scratch; mode 1: the fixed-rank solve is repeated once at
 * the largest rank allowed (max_rank) with q = max(q, 2) and judged again
 * (NOT_CONVERGED if that also misses the tolerance). */
rsvd_status rsvd_controller_fallback(rsvd_handle_t handle, int mode);

/* Host-side record of the last controlled solve on this handle:
 * info[0] = l, info[1] = q of the last fixed-rank solve (the network's choice,
 * or the escalated one when info[3] = 2), info[2] = accepted by the judge,
 * info[3] = 0 no fallback, 1 fell back to the adaptive range finder, 2
 * escalated to the largest rank, info[4] = output rank;
 * est[0] = Frobenius residual estimate / ||A||_F, est[1] = spectral bound /
 * ||A||_F (Lemma thm:aposteriori).  info: 5 ints, est: 2 doubles (host). */
rsvd_status rsvd_controller_last(rsvd_handle_t handle, int* info, double* est);

/* A-posteriori certificate (Sec. 14: eq. infomm and Lemma thm:aposteriori)
 * for any rank-r factorization A ~= U diag(D) V^T in binary32: with G = 16
 * columns of the Philox stream 2 under `seed` (rsvd_gaussian stream_id 2),
 * E = A G - U (D (V^T G)) and
 *   out[0] = sqrt(mean_i ||E(:, i)||^2), an unbiased estimate of ||A - U D V^T||_F^2
 *            under the square root (E ||E g||^2 = ||A - U D V^T||_F^2),
 *   out[1] = 10 sqrt(2/pi) max_i ||E(:, i)||, a bound on ||A - U D V^T||_2 that
 *            holds with probability at least 1 - 10^-16,
 *   out[2] = ||A||_F  (out: 3 doubles, host).
 * A m x n (lda >= n), U m x r (ldu >= r), D r doubles, V n x r (ldv >= r),
 * device memory or device-accessible host memory; 0 <= r <= 1024 (r = 0
 * certifies the zero approximation).  Reads A once.  Synchronizes `stream`.
 * Workspace: rsvd_certify_workspace_size bytes, 256-byte aligned. */
rsvd_status rsvd_certify_workspace_size(rsvd_handle_t handle, int m, int n, int r, size_t* bytes);
rsvd_status rsvd_certify(rsvd_handle_t handle, int m, int n, const float* A, int lda, int r, const float* U,
                         int ldu, const double* D, const float* V, int ldv, uint64_t seed, double* out,
                         void* workspace, size_t ws_bytes, rsvd_stream_t stream);

/* Allocation-free variant of rsvd_sketch for RSVD_MIXED_BF16 (the paper has
 * no counterpart: this is a deployment convenience).  For callers that may
 * not allocate device memory at all -- code running inside another
 * framework's memory pool, an allocation-free real-time loop, a plugin that is
 * handed only its input and output buffers -- and so cannot provide the
 * workspace rsvd_sketch needs.  Same product, same arguments as rsvd_sketch
 * minus the workspace: Y (fp32) = A X (trans = 0) or A^T X (trans = 1), A and X
 * bf16 with leading dimensions that are multiples of 8 elements and 16-byte
 * aligned rows.
 * Scratch: a fixed 20 MiB array inside the library's device image (partial
 * sums for at most 160 CTAs of 128 x 128 fp32 tiles, plus a status word);
 * every GPU that loads the library keeps it until the process exits.
 * Limits: l <= 128; larger l returns RSVD_E_INVALID ("l exceeds the fixed
 * scratch limit").  No cudaMalloc, cudaFree or other allocating call is made.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before capturing a stream.
 * The current device must be the handle's device (RSVD_E_INVALID otherwise).
 * status_out (optional, may be NULL): an int in device memory or mapped host
 * memory owned by the caller; it receives the device status word of this
 * call (RSVD_OK, or RSVD_E_TIMEOUT if a bounded wait in the kernel gave up
 * and Y is incomplete), copied in stream order after the product.
 * Every call reuses the same array, status word included: calls that overlap
 * on the GPU (other streams, other host threads) race on it and must be
 * serialized. */
rsvd_status rsvd_sketch_noalloc(rsvd_handle_t handle, int trans, int m, int n, int l, const void* A, int lda,
                                const void* X, int ldx, float* Y, int ldy, int* status_out,
                                rsvd_stream_t stream);

/* Orthonormalization (Sec. 2.3, "orth", unpivoted): Q = Y R^-1 with R upper
 * triangular, diag(R) > 0, by CholeskyQR2 (a shifted first pass is added when
 * the Gram matrix is too ill-conditioned, Fukaya et al., SISC 2020).  Y is
 * rows x l row-major (ldy), double for RSVD_F64 else float, overwritten by Q.
 * R (optional, may be NULL): l x l row-major doubles, receives R.
 * Gram matrices are accumulated in binary64. */
rsvd_status rsvd_orth_workspace_size(rsvd_handle_t handle, int prec, int rows, int l,
                                     size_t* bytes);
rsvd_status rsvd_orth(rsvd_handle_t handle, int prec, int rows, int l, void* Y, int ldy, double* R,
                      void* workspace, size_t ws_bytes, rsvd_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* RSVD_H */
