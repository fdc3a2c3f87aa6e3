// Launch wrappers shared between the library's translation units.
#pragma once

#include "common.cuh"

namespace rsvd {

// k_gauss.cu
void launch_philox_words(int n_groups, int l, uint64_t seed, uint32_t stream_id, int col0, uint32_t* out,
                         cudaStream_t s);
void launch_gaussian(int n, int l, uint64_t seed, uint32_t stream_id, int col0, int dtype, void* out, int ldo,
                     cudaStream_t s);

// k_gemm.cu
int simt_splits(int M, int N, int K, int sms);
size_t simt_gemm_workspace(int M, int N, int K, int sms, size_t elem);
template <typename T>
void launch_gemm_simt(bool trans, int M, int N, int K, const T* A, int lda, const T* X, int ldx, T* Y, int ldy,
                      T* partial, int sms, cudaStream_t s);

// k_orth.cu
int gram_splits(int rows, int l, int sms, size_t tsize);
template <typename T>
void launch_gram(int rows, int l, const T* Y, int ldy, double* P, double* G, float* Gf, int sms, const int* gate,
                 cudaStream_t s, const int* skip = nullptr, __nv_bfloat16* Yh = nullptr, __nv_bfloat16* Yl = nullptr,
                 int lb = 0);
size_t chol_smem_bytes(int l, size_t csize);
size_t orth_workspace_bytes(int rows, int l, int sms, size_t csize);
template <typename T, typename C>
// skip (optional): every kernel returns at once while *skip != 0 (device-side loop control)
void run_orth(int rows, int l, T* Y, int ldy, double* Rout, __nv_bfloat16* Ybf, int lb, void* ws, DevStatus* st,
              int sms, cudaStream_t s, const int* skip = nullptr);
template <typename T>
void launch_copy_bf16(int rows, int l, const T* Y, int ldy, __nv_bfloat16* Yb, int lb, cudaStream_t s);
// Nystrom factor: B = C^T C (Cholesky of the symmetrized l x l B), Y <- Y C^-1 (run_orth's workspace)
template <typename T, typename C>
void run_chol_solve(int rows, int l, const T* B, int ldb, T* Y, int ldy, void* ws, DevStatus* st, int sms,
                    cudaStream_t s);
// CholeskyQR2 with the apply Q = Y R^-1 on tensor cores (three-term split bf16); binary32 data
size_t orth_tc_workspace_bytes(int rows, int l, int sms);
// intermediate: Y is a power-iteration basis whose span alone is used next;
// the second pass is skipped when the first already gives a basis with
// ||Q^T Q - I||_2 <= 1/2 (checked on the second pass's Gram), and no third
// pass runs.
void run_orth_tc(int rows, int l, float* Y, int ldy, double* Rout, __nv_bfloat16* Ybf, int lb, void* ws,
                 DevStatus* st, int sms, cudaStream_t s, bool intermediate = false);
void launch_triu_mm(int l, const double* A, const double* B, double* Cm, const int* gate, int copy_if_gated,
                    cudaStream_t s, const int* skip = nullptr);

// k_svd.cu
int jacobi_cluster_size(int l);
size_t jacobi_smem_bytes(int l, size_t csize);
template <typename C>
cudaError_t launch_jacobi(int l, const double* Rb, C* Wt, C* Jt, double* sigma, DevStatus* st, cudaStream_t s);
template <typename C>
void launch_sort_gather(int l, int kk, const double* sigma, const C* Wt, const C* Jt, double* D, C* Wsel, C* Jsel,
                        cudaStream_t s);
size_t sign_workspace_bytes(int n, int kk);
template <typename T, typename C>
void launch_sign_fix(int n, int kk, int l, T* V, int ldv, C* Wsel, void* ws, cudaStream_t s);

// k_tc.cu
size_t tc_gemm_workspace(int M, int N, int K, int sms);
bool tc_supported(int N);
int tc_rows_per_tile(int M, bool split3);
// bm: rows per tile (128 or 256); 0 lets the launcher choose (tc_rows_per_tile).
cudaError_t launch_tc_gemm(bool trans, bool split3, int M, int N, int K, const __nv_bfloat16* A, int lda,
                           const __nv_bfloat16* A2, const __nv_bfloat16* X, int ldx, const __nv_bfloat16* X2, float* Y,
                           int ldy, float* part, int sms, DevStatus* st, cudaStream_t s, int bm = 0,
                           const int* gate = nullptr);
void launch_split_bf16(int rows, int cols, const float* A, int lda, __nv_bfloat16* Ah, __nv_bfloat16* Al, int ldb,
                       int sms, cudaStream_t s);
// Y (M x N fp32) = diag(rs) (A8 X8t^T) diag(cs): A8 M x K, X8t N x K, e4m3
// bytes row-major (ld in bytes, multiples of 16); rs may be null.
size_t tc_gemm_e4m3_workspace(int M, int N, int K, int sms);
cudaError_t launch_tc_gemm_e4m3(int M, int N, int K, const uint8_t* A8, int lda, const uint8_t* X8t, int ldx,
                                const float* rs, const float* cs, float* Y, int ldy, float* part, int sms,
                                DevStatus* st, cudaStream_t s);

// k_fp8.cu
// Rows of A (fp32) scaled to e4m3: A8 (rows x cols, ld8 bytes), s[i] = max_j |A_ij| / 448;
// optionally the bf16 pair Ah + Al of A (ldb elements).
void launch_fp8_rows(int rows, int cols, const float* A, int lda, uint8_t* A8, int ld8, float* s,
                     __nv_bfloat16* Ah, __nv_bfloat16* Al, int ldb, int sms, cudaStream_t st,
                     const float* amax = nullptr);  // amax: a given maximum per row (block scaling)
// amax[i] = max |A| over i's block of `block` rows (the per-block scale of the
// e4m3 copy, RSVD_MIXED_FP8_B128)
void launch_fp8_block_max(int rows, int cols, const float* A, int lda, int block, float* amax, cudaStream_t st);
// B (cols x rows bytes, ldt) = A^T for e4m3 bytes A (rows x cols, lda).
void launch_u8_transpose(int rows, int cols, const uint8_t* A, int lda, uint8_t* B, int ldt, cudaStream_t st);
// X (rows x cols fp32, ldx), optionally with row scales rsc: X' = diag(rsc) X in binary32;
// X8t (cols x rows e4m3 bytes, ldt) = e4m3(X'^T diag(448 / amax_j)), c[j] = amax_j / 448 (column amax of X').
size_t fp8_cols_workspace(int rows, int cols);
void launch_fp8_cols(int rows, int cols, const float* X, int ldx, const float* rsc, uint8_t* X8t, int ldt, float* c,
                     void* ws, cudaStream_t st);

// k_adapt.cu
size_t adapt_workspace_bytes(int m, int n, int R, int b, int sms, size_t es);
template <typename T, typename C>
void run_adaptive(int m, int n, const T* A, int lda, double tol, int R, int b, int q, uint64_t seed, void* ws,
                  void* orthws, DevStatus* st, int sms, cudaStream_t s, T** Qout, T** Btout,
                  double spectral_eps = 0.0);  // > 0: spectral-norm stopping test with this absolute eps

// k_centre.cu (implicit column centring, RSVD_FLAG_CENTER)
struct CentreBufs {
  double* mu;    // n column means
  double* vec;   // l: mu^T X or 1^T Q
  double* part;  // per-slice partial sums
};
size_t centre_workspace_bytes(int m, int n, int l, int sms);
CentreBufs centre_carve(void* ws, int m, int n, int l, int sms);
template <typename T>
void centre_means(int m, int n, const T* A, int lda, const CentreBufs& B, int sms, cudaStream_t s);
template <typename T, typename X>
void centre_forward(int m, int n, int l, const X* Xop, int ldx, T* Y, int ldy, const CentreBufs& B, int sms,
                    cudaStream_t s);
template <typename T, typename Q>
void centre_adjoint(int m, int n, int l, const Q* Qm, int ldq, T* Z, int ldz, const CentreBufs& B, int sms,
                    cudaStream_t s);

// singlepass.cu (Figs. singlepass_gen, singlepass_herm)
struct SinglePassLayout {
  DevStatus* st;
  void *Gc, *Gr, *Yc, *Yr, *orthws;
  double *Rc, *Rr;
  void *Wt, *Jt;
  double *sig, *sigs;
  void *Wsel, *Jc, *Jr, *Qc, *Qr, *Pt, *Mt, *part;
  double *Jd, *Rd, *P, *MT, *X1, *X2;
  double* K[6];
  double *s1, *s2;
  void* orth64;
  double *Rb64, *Wt64, *Jt64, *sig64, *part64;
  void *Uh, *Vh;
  __nv_bfloat16 *Ah, *Gcb, *Grb;
  float* tcpart;
  size_t bytes;
};
SinglePassLayout single_pass_layout(void* ws, int m, int n, int k, int l, size_t es, int sms, bool mixed);
template <typename T>
void run_single_pass_svd(int m, int n, const T* A, int lda, int k, int p, uint64_t seed, T* U, int ldu, double* D,
                         T* V, int ldv, const SinglePassLayout& L, int sms, bool mixed, cudaStream_t s);
template <typename T>
void run_single_pass_evd(int n, const T* A, int lda, int k, int p, uint64_t seed, T* U, int ldu, double* D, T* V,
                         int ldv, const SinglePassLayout& L, int sms, bool mixed, cudaStream_t s);

// srft.cu (eq. SRFT: Fig. RSVD with Omega = D F S, on the realification)
struct SrftLayout {
  DevStatus* st;
  unsigned long long* key;
  int* S;
  void *Om, *Y2, *Yh, *Z, *orthws;
  double* Rb;
  void *Wt, *Jt;
  double *sig, *Dall;
  void *Wsel, *Jsel, *W2, *J2, *Uh, *Vh, *Xi, *part;
  __nv_bfloat16 *Ah, *Al, *Omb, *Qh, *Ql;
  float* tcpart;
  size_t bytes;
};
SrftLayout srft_layout(void* ws, int m, int n, int l, int kk, size_t es, int sms, bool mixed);
// U, V: complex outputs, interleaved (re, im), leading dimensions in complex entries
template <typename T>
cudaError_t run_srft(int m, int n, const T* A, int lda, int k, int p, int kk, uint64_t seed, T* U, int ldu, double* D,
                     T* V, int ldv, const SrftLayout& L, int sms, bool mixed, cudaStream_t s);

// k_batched.cu
int batched_max_rank();
int batched_max_dim();
int batched_max_block();
size_t batched_workspace_bytes(int count, int ctas);
int batched_variants();
int batched_default_variant();
void batched_variant_info(int v, int* pf, int* pd);
cudaError_t launch_batched(int count, const int* m, const int* n, const int* lda, const float* const* A,
                           float* const* U, double* const* D, float* const* V, int R, int b, uint64_t seed,
                           double tol, int* rank_out, double* err_out, int* status_out, void* ws, int ctas,
                           cudaStream_t s, int variant);

// k_ctrl.cu
int thin_splits(int m, int n, int sms);
int launch_thin_sketch(int m, int n, const float* A, int lda, const float* G, float* Yp, float* Y, double* fro2p,
                       int sms, cudaStream_t s);
void launch_ctrl_features(int m, int n, const double* Gram, int nfro, const double* fro2p, RsvdCtrlBlock* blk,
                          cudaStream_t s);
void launch_ctrl_decide(RsvdCtrlBlock* blk, float quantile, int lmax, cudaStream_t s);
void launch_fro2_reduce(int nfro, const double* fro2p, RsvdCtrlBlock* blk, cudaStream_t s);
size_t mlp_workspace_bytes(int batch);
// mode -1: logits only (no workspace); 0: gradient into grad; 1: Adam step on th
cudaError_t launch_mlp(int mode, int batch, const float* X, const int* yl, const int* yq, float lam,
                       const float* th, float* logits, float* grad, float* m1, float* m2, int t, float lr,
                       double* loss_out, void* ws, cudaStream_t s);
int resid_blocks(int m, int sms);
void launch_judge(int m, int l, const float* Yc, const float* U, int ldu, const double* D, const float* T,
                  double* part, double tol, double safety, RsvdCtrlBlock* blk, int sms, cudaStream_t s);

}  // namespace rsvd
