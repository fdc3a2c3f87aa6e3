// Single-pass randomized SVD and EVD (Sec. "Single pass algorithms", Figs.
// singlepass_gen and singlepass_herm).  Every product with A is a sketch
// taken before any basis exists; the small core C is fitted to the sketches
// by least squares instead of being formed as Q^T A Q.
//
// General A (m x n), l = k + p:
//   Gc = randn(n, l) (stream 0), Gr = randn(m, l) (stream 5)
//   Yc = A Gc, Yr = A^T Gr
//   Qc, Qr = the k dominant left singular vectors of Yc, Yr
//   C = argmin ||P C - R1||^2 + ||C M - R2||^2,  P = Gr^T Qc, R1 = Yr^T Qr,
//                                                M = Qr^T Gc, R2 = Qc^T Yc
//   C = Uhat D Vhat^T,  U = Qc Uhat,  V = Qr Vhat
// Symmetric A (n x n):
//   Y = A G,  Q = the k dominant left singular vectors of Y
//   C = argmin over symmetric C of ||C M - N||,  M = Q^T G, N = Q^T Y
//   C = Uhat Lambda Uhat^T (pairs ordered by |lambda|),  U = Q Uhat
//
// The fits are solved from their normal equations, which are Sylvester
// equations with symmetric positive definite coefficients:
//   general:   S1 C + C S2 = F,   S1 = P^T P, S2 = M M^T, F = P^T R1 + R2 M^T
//   symmetric: S C + C S = F,     S = M M^T,             F = N M^T + M N^T
// With S1 = E1 L1 E1^T and S2 = E2 L2 E2^T (squared singular values and right
// singular vectors of P and M^T), C = E1 [(E1^T F E2) ./ (L1_i + L2_j)] E2^T.
// The fit runs in binary64 (k <= 128).  The dominant singular vectors come
// from the CholeskyQR of the sketch, Y = Q R, and the Jacobi SVD of R: with
// R = J Sigma W^T, the left singular vectors of Y are Q J, and Q^T Y = R, so
// R2 = Qc^T Yc = J_k^T R needs no second read of the sketch.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

namespace {

template <typename T>
__global__ void to_double_kernel(int rows, int cols, const T* __restrict__ X, int ldx, double* __restrict__ Y,
                                 int ldy) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int i = idx / cols, j = idx % cols;
  Y[(size_t)i * ldy + j] = (double)X[(size_t)i * ldx + j];
}

template <typename T>
__global__ void from_double_kernel(int rows, int cols, const double* __restrict__ X, int ldx, T* __restrict__ Y,
                                   int ldy) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int i = idx / cols, j = idx % cols;
  Y[(size_t)i * ldy + j] = (T)X[(size_t)i * ldx + j];
}

// F = X1^T + X2 (k x k), or F = X2 + X2^T when X1 == null
__global__ void sum_t_kernel(int k, const double* __restrict__ X1, const double* __restrict__ X2,
                             double* __restrict__ F) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * k) return;
  const int i = idx / k, j = idx % k;
  const double a = X1 ? X1[(size_t)j * k + i] : X2[(size_t)j * k + i];
  F[idx] = a + X2[idx];
}

// H(i, j) = G(i, j) / (s1_i^2 + s2_j^2)   (s: singular values of P, M^T)
__global__ void sylvester_scale_kernel(int k, const double* __restrict__ s1, const double* __restrict__ s2,
                                       double* __restrict__ G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * k) return;
  const int i = idx / k, j = idx % k;
  const double d = s1[i] * s1[i] + s2[j] * s2[j];
  G[idx] = d > 0.0 ? G[idx] / d : 0.0;
}

// B = A^T (k x k)
__global__ void transpose_kernel(int k, const double* __restrict__ A, double* __restrict__ B) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * k) return;
  const int i = idx / k, j = idx % k;
  B[(size_t)j * k + i] = A[idx];
}

// Symmetric C = (Q_C J) Sigma W^T: lambda_i = sigma_i sign(<(Q_C J)_i, W_i>).
__global__ void eig_sign_kernel(int k, const double* __restrict__ Uc, const double* __restrict__ W,
                                double* __restrict__ D) {
  const int c = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += 32) s += Uc[(size_t)i * k + c] * W[(size_t)i * k + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0 && s < 0.0) D[c] = -D[c];
}

int grid_for(int total) { return ceil_div(total > 0 ? total : 1, 256); }

}  // namespace

// ------------------------------------------------------------------ layout --
SinglePassLayout single_pass_layout(void* ws, int m, int n, int k, int l, size_t es, int sms, bool mixed) {
  Carver c(ws);
  SinglePassLayout L;
  const int big = m > n ? m : n;
  L.st = c.take<DevStatus>(1);
  L.Gc = c.take<unsigned char>((size_t)n * l * es);
  L.Gr = c.take<unsigned char>((size_t)m * l * es);
  L.Yc = c.take<unsigned char>((size_t)m * l * es);
  L.Yr = c.take<unsigned char>((size_t)n * l * es);
  L.orthws = c.take<unsigned char>(mixed ? orth_tc_workspace_bytes(big, l, sms) : orth_workspace_bytes(big, l, sms, es));
  L.Rc = c.take<double>((size_t)l * l);
  L.Rr = c.take<double>((size_t)l * l);
  L.Wt = c.take<unsigned char>((size_t)l * l * es);
  L.Jt = c.take<unsigned char>((size_t)l * l * es);
  L.sig = c.take<double>((size_t)l);
  L.sigs = c.take<double>((size_t)l);
  L.Wsel = c.take<unsigned char>((size_t)l * l * es);
  L.Jc = c.take<unsigned char>((size_t)l * l * es);
  L.Jr = c.take<unsigned char>((size_t)l * l * es);
  L.Qc = c.take<unsigned char>((size_t)m * k * es);
  L.Qr = c.take<unsigned char>((size_t)n * k * es);
  L.Pt = c.take<unsigned char>((size_t)l * k * es);
  L.Mt = c.take<unsigned char>((size_t)l * k * es);
  size_t pw = simt_gemm_workspace(l, k, big, sms, es);
  const size_t pw2 = simt_gemm_workspace(big, k, l, sms, es);
  if (pw2 > pw) pw = pw2;
  if (sign_workspace_bytes(big, k) > pw) pw = sign_workspace_bytes(big, k);
  L.part = c.take<unsigned char>(pw + 256);
  // binary64 fit
  L.Jd = c.take<double>((size_t)l * l);
  L.Rd = c.take<double>((size_t)l * l);
  L.P = c.take<double>((size_t)l * k);
  L.MT = c.take<double>((size_t)l * k);
  L.X1 = c.take<double>((size_t)k * l);
  L.X2 = c.take<double>((size_t)k * l);
  for (int i = 0; i < 6; ++i) L.K[i] = c.take<double>((size_t)k * k);
  L.s1 = c.take<double>((size_t)k);
  L.s2 = c.take<double>((size_t)k);
  L.orth64 = c.take<unsigned char>(orth_workspace_bytes(l, k, sms, 8));
  L.Rb64 = c.take<double>((size_t)k * k);
  L.Wt64 = c.take<double>((size_t)k * k);
  L.Jt64 = c.take<double>((size_t)k * k);
  L.sig64 = c.take<double>((size_t)k);
  L.part64 = c.take<double>(simt_gemm_workspace(k, k, l, sms, 8) / 8 + 64);
  L.Uh = c.take<unsigned char>((size_t)k * k * es);
  L.Vh = c.take<unsigned char>((size_t)k * k * es);
  if (mixed) {
    const int n8 = (n + 7) / 8 * 8, l8 = (l + 7) / 8 * 8;
    L.Ah = c.take<__nv_bfloat16>((size_t)m * n8);
    L.Gcb = c.take<__nv_bfloat16>((size_t)n * l8);
    L.Grb = c.take<__nv_bfloat16>((size_t)m * l8);
    size_t tw = tc_gemm_workspace(m, l, n, sms);
    if (tc_gemm_workspace(n, l, m, sms) > tw) tw = tc_gemm_workspace(n, l, m, sms);
    L.tcpart = c.take<float>(tw / sizeof(float) + 1);
  } else {
    L.Ah = nullptr;
    L.Gcb = L.Grb = nullptr;
    L.tcpart = nullptr;
  }
  L.bytes = c.size();
  return L;
}

// ---------------------------------------------------------------- helpers --
// The k dominant left singular vectors of Y (rows x l, overwritten by its Q):
// Y = Q R (R into Rb), R^T J = W Sigma, Qk = Q J_k.  Jsel (l x l, sorted) is kept.
template <typename T>
static void dominant_left(int rows, int l, int k, T* Y, double* Rb, T* Qk, T* Jsel, const SinglePassLayout& L,
                          int sms, bool mixed, cudaStream_t s) {
  if (mixed && sizeof(T) == 4)
    run_orth_tc(rows, l, (float*)Y, l, Rb, nullptr, 0, L.orthws, L.st, sms, s);
  else
    run_orth<T, T>(rows, l, Y, l, Rb, nullptr, 0, L.orthws, L.st, sms, s);
  launch_jacobi<T>(l, Rb, (T*)L.Wt, (T*)L.Jt, L.sig, L.st, s);
  launch_sort_gather<T>(l, l, L.sig, (const T*)L.Wt, (const T*)L.Jt, L.sigs, (T*)L.Wsel, Jsel, s);
  launch_gemm_simt<T>(false, rows, k, l, Y, l, Jsel, l, Qk, k, nullptr, sms, s);
}

// SVD of X (rows x k binary64, overwritten): right singular vectors into Wsel
// (k x k, descending), singular values into sig; Q_X J into QJ if given.
static void small_svd64(int rows, int k, double* X, double* sig, double* Wsel, double* QJ, const SinglePassLayout& L,
                        int sms, cudaStream_t s) {
  run_orth<double, double>(rows, k, X, k, L.Rb64, nullptr, 0, L.orth64, L.st, sms, s);
  launch_jacobi<double>(k, L.Rb64, L.Wt64, L.Jt64, L.sig64, L.st, s);
  double* Jsel = L.K[5];
  launch_sort_gather<double>(k, k, L.sig64, L.Wt64, L.Jt64, sig, Wsel, Jsel, s);
  if (QJ) launch_gemm_simt<double>(false, rows, k, k, X, k, Jsel, k, QJ, k, nullptr, sms, s);
}

// C = E1 [(E1^T F E2) ./ (s1_i^2 + s2_j^2)] E2^T; F is overwritten.
static void sylvester(int k, const double* E1, const double* s1, const double* E2, const double* s2, double* F,
                      double* C, double* tmp, double* tmp2, int sms, cudaStream_t s) {
  launch_gemm_simt<double>(true, k, k, k, E1, k, F, k, tmp, k, nullptr, sms, s);      // E1^T F
  launch_gemm_simt<double>(false, k, k, k, tmp, k, E2, k, F, k, nullptr, sms, s);     // (E1^T F) E2
  sylvester_scale_kernel<<<grid_for(k * k), 256, 0, s>>>(k, s1, s2, F);
  note_launch();
  launch_gemm_simt<double>(false, k, k, k, E1, k, F, k, tmp, k, nullptr, sms, s);     // E1 H
  transpose_kernel<<<grid_for(k * k), 256, 0, s>>>(k, E2, tmp2);                       // E2^T
  note_launch();
  launch_gemm_simt<double>(false, k, k, k, tmp, k, tmp2, k, C, k, nullptr, sms, s);   // (E1 H) E2^T
}

// ------------------------------------------------------------------ solves --
template <typename T>
void run_single_pass_svd(int m, int n, const T* A, int lda, int k, int p, uint64_t seed, T* U, int ldu, double* D,
                         T* V, int ldv, const SinglePassLayout& L, int sms, bool mixed, cudaStream_t s) {
  const int l = k + p;
  const int dt = sizeof(T) == 8 ? RSVD_DT_F64 : RSVD_DT_F32;
  T* Gc = (T*)L.Gc;
  T* Gr = (T*)L.Gr;
  T* Yc = (T*)L.Yc;
  T* Yr = (T*)L.Yr;
  T* part = (T*)L.part;
  launch_gaussian(n, l, seed, 0u, 0, dt, Gc, l, s);
  launch_gaussian(m, l, seed, 5u, 0, dt, Gr, l, s);
  // the two sketches
  if (mixed && sizeof(T) == 4) {
    const int n8 = (n + 7) / 8 * 8, l8 = (l + 7) / 8 * 8;
    launch_split_bf16(m, n, (const float*)A, lda, L.Ah, nullptr, n8, sms, s);
    launch_split_bf16(n, l, (const float*)Gc, l, L.Gcb, nullptr, l8, sms, s);
    launch_split_bf16(m, l, (const float*)Gr, l, L.Grb, nullptr, l8, sms, s);
    launch_tc_gemm(false, false, m, l, n, L.Ah, n8, nullptr, L.Gcb, l8, nullptr, (float*)Yc, l, L.tcpart, sms, L.st, s);
    launch_tc_gemm(true, false, n, l, m, L.Ah, n8, nullptr, L.Grb, l8, nullptr, (float*)Yr, l, L.tcpart, sms, L.st, s);
  } else {
    launch_gemm_simt<T>(false, m, l, n, A, lda, Gc, l, Yc, l, part, sms, s);
    launch_gemm_simt<T>(true, n, l, m, A, lda, Gr, l, Yr, l, part, sms, s);
  }
  // Qc, Qr and their J (Yc, Yr now hold the Q factors)
  dominant_left<T>(m, l, k, Yc, L.Rc, (T*)L.Qc, (T*)L.Jc, L, sms, mixed, s);
  dominant_left<T>(n, l, k, Yr, L.Rr, (T*)L.Qr, (T*)L.Jr, L, sms, mixed, s);
  // P = Gr^T Qc, M^T = Gc^T Qr (l x k), in binary64
  launch_gemm_simt<T>(true, l, k, m, Gr, l, (const T*)L.Qc, k, (T*)L.Pt, k, part, sms, s);
  launch_gemm_simt<T>(true, l, k, n, Gc, l, (const T*)L.Qr, k, (T*)L.Mt, k, part, sms, s);
  to_double_kernel<T><<<grid_for(l * k), 256, 0, s>>>(l, k, (const T*)L.Pt, k, L.P, k);
  to_double_kernel<T><<<grid_for(l * k), 256, 0, s>>>(l, k, (const T*)L.Mt, k, L.MT, k);
  note_launch();
  note_launch();
  // X1 = R1^T = J_r,k^T R_r and R2 = J_c,k^T R_c (k x l)
  to_double_kernel<T><<<grid_for(l * l), 256, 0, s>>>(l, l, (const T*)L.Jr, l, L.Jd, l);
  note_launch();
  launch_gemm_simt<double>(true, k, l, l, L.Jd, l, L.Rr, l, L.X1, l, nullptr, sms, s);
  to_double_kernel<T><<<grid_for(l * l), 256, 0, s>>>(l, l, (const T*)L.Jc, l, L.Jd, l);
  note_launch();
  launch_gemm_simt<double>(true, k, l, l, L.Jd, l, L.Rc, l, L.X2, l, nullptr, sms, s);
  // F = P^T R1 + R2 M^T = (X1 P)^T + R2 M^T
  double *K0 = L.K[0], *K1 = L.K[1], *K2 = L.K[2], *K3 = L.K[3], *K4 = L.K[4];
  launch_gemm_simt<double>(false, k, k, l, L.X1, l, L.P, k, K0, k, L.part64, sms, s);
  launch_gemm_simt<double>(false, k, k, l, L.X2, l, L.MT, k, K1, k, L.part64, sms, s);
  sum_t_kernel<<<grid_for(k * k), 256, 0, s>>>(k, K0, K1, K2);  // F
  note_launch();
  // S1 = P^T P = E1 diag(s1^2) E1^T, S2 = M M^T = E2 diag(s2^2) E2^T
  small_svd64(l, k, L.P, L.s1, K0, nullptr, L, sms, s);   // E1 -> K0
  small_svd64(l, k, L.MT, L.s2, K1, nullptr, L, sms, s);  // E2 -> K1
  sylvester(k, K0, L.s1, K1, L.s2, K2, K3, K4, L.X1, sms, s);  // C -> K3
  // C = (Q_C J) Sigma W^T: Uhat = Q_C J (K2), Vhat = W (K0), D = sigma
  small_svd64(k, k, K3, D, K0, K2, L, sms, s);
  from_double_kernel<T><<<grid_for(k * k), 256, 0, s>>>(k, k, K2, k, (T*)L.Uh, k);
  from_double_kernel<T><<<grid_for(k * k), 256, 0, s>>>(k, k, K0, k, (T*)L.Vh, k);
  note_launch();
  note_launch();
  // V = Qr Vhat; the sign convention on V, carried to Uhat; U = Qc Uhat
  launch_gemm_simt<T>(false, n, k, k, (const T*)L.Qr, k, (const T*)L.Vh, k, V, ldv, nullptr, sms, s);
  launch_sign_fix<T, T>(n, k, k, V, ldv, (T*)L.Uh, L.part, s);
  launch_gemm_simt<T>(false, m, k, k, (const T*)L.Qc, k, (const T*)L.Uh, k, U, ldu, nullptr, sms, s);
}

template <typename T>
void run_single_pass_evd(int n, const T* A, int lda, int k, int p, uint64_t seed, T* U, int ldu, double* D, T* V,
                         int ldv, const SinglePassLayout& L, int sms, bool mixed, cudaStream_t s) {
  const int l = k + p;
  const int dt = sizeof(T) == 8 ? RSVD_DT_F64 : RSVD_DT_F32;
  T* G = (T*)L.Gc;
  T* Y = (T*)L.Yc;
  T* part = (T*)L.part;
  launch_gaussian(n, l, seed, 0u, 0, dt, G, l, s);
  if (mixed && sizeof(T) == 4) {
    const int n8 = (n + 7) / 8 * 8, l8 = (l + 7) / 8 * 8;
    launch_split_bf16(n, n, (const float*)A, lda, L.Ah, nullptr, n8, sms, s);
    launch_split_bf16(n, l, (const float*)G, l, L.Gcb, nullptr, l8, sms, s);
    launch_tc_gemm(false, false, n, l, n, L.Ah, n8, nullptr, L.Gcb, l8, nullptr, (float*)Y, l, L.tcpart, sms, L.st, s);
  } else {
    launch_gemm_simt<T>(false, n, l, n, A, lda, G, l, Y, l, part, sms, s);
  }
  dominant_left<T>(n, l, k, Y, L.Rc, (T*)L.Qc, (T*)L.Jc, L, sms, mixed, s);
  // M^T = G^T Q (l x k); N = Q^T Y = J_k^T R (k x l)
  launch_gemm_simt<T>(true, l, k, n, G, l, (const T*)L.Qc, k, (T*)L.Mt, k, part, sms, s);
  to_double_kernel<T><<<grid_for(l * k), 256, 0, s>>>(l, k, (const T*)L.Mt, k, L.MT, k);
  to_double_kernel<T><<<grid_for(l * l), 256, 0, s>>>(l, l, (const T*)L.Jc, l, L.Jd, l);
  note_launch();
  note_launch();
  launch_gemm_simt<double>(true, k, l, l, L.Jd, l, L.Rc, l, L.X2, l, nullptr, sms, s);
  // F = N M^T + M N^T
  double *K0 = L.K[0], *K1 = L.K[1], *K2 = L.K[2], *K3 = L.K[3], *K4 = L.K[4];
  launch_gemm_simt<double>(false, k, k, l, L.X2, l, L.MT, k, K1, k, L.part64, sms, s);
  sum_t_kernel<<<grid_for(k * k), 256, 0, s>>>(k, nullptr, K1, K2);
  note_launch();
  // S = M M^T = E diag(s^2) E^T; Lyapunov solve S C + C S = F
  small_svd64(l, k, L.MT, L.s1, K0, nullptr, L, sms, s);
  sylvester(k, K0, L.s1, K0, L.s1, K2, K3, K4, L.X1, sms, s);  // C -> K3 (symmetric)
  // EVD of the symmetric C through its SVD: C = (Q_C J) Sigma W^T,
  // eigenvectors W, eigenvalues sigma_i sign(<(Q_C J)_i, W_i>)
  small_svd64(k, k, K3, D, K0, K2, L, sms, s);
  eig_sign_kernel<<<k, 32, 0, s>>>(k, K2, K0, D);
  note_launch();
  from_double_kernel<T><<<grid_for(k * k), 256, 0, s>>>(k, k, K0, k, (T*)L.Uh, k);
  note_launch();
  launch_gemm_simt<T>(false, n, k, k, (const T*)L.Qc, k, (const T*)L.Uh, k, U, ldu, nullptr, sms, s);
  // the sign convention: the largest-magnitude entry of each u_i positive
  launch_sign_fix<T, T>(n, k, k, U, ldu, (T*)L.Vh, L.part, s);
  cudaMemcpy2DAsync(V, (size_t)ldv * sizeof(T), U, (size_t)ldu * sizeof(T), (size_t)k * sizeof(T), n,
                    cudaMemcpyDeviceToDevice, s);
}

template void run_single_pass_svd<float>(int, int, const float*, int, int, int, uint64_t, float*, int, double*,
                                         float*, int, const SinglePassLayout&, int, bool, cudaStream_t);
template void run_single_pass_svd<double>(int, int, const double*, int, int, int, uint64_t, double*, int, double*,
                                          double*, int, const SinglePassLayout&, int, bool, cudaStream_t);
template void run_single_pass_evd<float>(int, const float*, int, int, int, uint64_t, float*, int, double*, float*,
                                         int, const SinglePassLayout&, int, bool, cudaStream_t);
template void run_single_pass_evd<double>(int, const double*, int, int, int, uint64_t, double*, int, double*,
                                          double*, int, const SinglePassLayout&, int, bool, cudaStream_t);

}  // namespace rsvd
