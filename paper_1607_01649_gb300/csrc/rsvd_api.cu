// C ABI of the randomized-SVD library: argument checks, workspace layout and
// the order of kernel launches on the caller's stream.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

struct rsvd_handle_s {
  int device;
  int sms;
  char err[512];
  // profiling: event pairs bracketing tensor-core products, per kind
  bool profile;
  std::vector<cudaEvent_t> pool;                     // free events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> rec[2];
  // learned controller: caller-owned parameters and the last decision
  const float* ctrl_theta;
  double ctrl_quantile, ctrl_safety;
  int ctrl_fallback;  // 0: adaptive range finder, 1: fixed rank at the largest rank
  int ctrl_info[5];
  double ctrl_est[2];
  // rsvd_batched launch variant (-1: the library default), set by the autotuner
  int batched_variant;
};

namespace rsvd {
namespace {

rsvd_status fail(rsvd_handle_t h, rsvd_status code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

rsvd_status check_launch(rsvd_handle_t h, const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
  return RSVD_OK;
}

int max_l_for(int prec) { return prec == RSVD_F64 ? 128 : 256; }

inline bool is_fp8(int prec) { return prec == RSVD_MIXED_FP8 || prec == RSVD_MIXED_FP8_B128; }

size_t elem_size(int prec) { return prec == RSVD_F64 ? sizeof(double) : sizeof(float); }

// ------------------------------------------------------ fixed-rank layout --
struct FixedLayout {
  DevStatus* st;
  void* Om;      // n x l
  void* Ybuf;    // m x l  (Y, then Q)
  void* Zbuf;    // n x l  (Z, W, B^T, Q_B)
  void* part;    // split-K partials
  void* orthws;  // orth scratch
  double* Rb;    // l x l
  void* Wt;      // l x l
  void* Jt;      // l x l
  double* sigma; // l
  void* Wsel;    // l x kk
  void* Jsel;    // l x kk
  size_t bytes;
};

FixedLayout fixed_layout(void* ws, int m, int n, int l, int kk, int prec, int sms) {
  const size_t es = elem_size(prec);
  Carver c(ws);
  FixedLayout L;
  L.st = c.take<DevStatus>(1);
  L.Om = c.take<unsigned char>((size_t)n * l * es);
  L.Ybuf = c.take<unsigned char>((size_t)m * l * es);
  L.Zbuf = c.take<unsigned char>((size_t)n * l * es);
  size_t pw = simt_gemm_workspace(m, l, n, sms, es);
  const size_t pw2 = simt_gemm_workspace(n, l, m, sms, es);
  if (pw2 > pw) pw = pw2;
  // the l x l product Q^T B1 of the Nystrom path (m = n), split over K = n
  const size_t pw3 = simt_gemm_workspace(l, l, n, sms, es);
  if (pw3 > pw) pw = pw3;
  if (sign_workspace_bytes(n, kk) > pw) pw = sign_workspace_bytes(n, kk);
  L.part = c.take<unsigned char>(pw);
  size_t ow = orth_workspace_bytes(m, l, sms, es);
  const size_t ow2 = orth_workspace_bytes(n, l, sms, es);
  if (ow2 > ow) ow = ow2;
  L.orthws = c.take<unsigned char>(ow);
  L.Rb = c.take<double>((size_t)l * l);
  L.Wt = c.take<unsigned char>((size_t)l * l * es);
  L.Jt = c.take<unsigned char>((size_t)l * l * es);
  L.sigma = c.take<double>((size_t)l);
  L.Wsel = c.take<unsigned char>((size_t)l * kk * es);
  L.Jsel = c.take<unsigned char>((size_t)l * kk * es);
  L.bytes = c.size();
  return L;
}

// Whether the handle's device can read and write p directly: device or
// managed memory; host memory registered with (or allocated by) the CUDA
// runtime and mapped at the same address; or pageable host memory on a
// device with pageable-memory access (address translation services).
bool device_accessible(rsvd_handle_t h, const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == h->device;
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer == p;
  int pageable = 0;
  if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, h->device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return pageable != 0;
}

rsvd_status validate_fixed(rsvd_handle_t h, int m, int n, const void* A, int lda, const rsvd_params* p,
                           const void* U, int ldu, const void* D, const void* V, int ldv, int* kk_out) {
  if (!h) return RSVD_E_INVALID;
  if (!p) return fail(h, RSVD_E_INVALID, "params is NULL");
  if (m < 0 || n < 0) return fail(h, RSVD_E_INVALID, "negative size m=%d n=%d", m, n);
  if (p->k < 0 || p->p < 0 || p->q < 0) return fail(h, RSVD_E_INVALID, "k, p, q must be >= 0");
  if (p->prec != RSVD_F64 && p->prec != RSVD_F32 && p->prec != RSVD_MIXED_BF16 && !is_fp8(p->prec))
    return fail(h, RSVD_E_UNSUPPORTED, "precision %d is not implemented", p->prec);
  const int l0 = p->k + p->p;
  const bool krylov = (p->flags & RSVD_FLAG_KRYLOV) != 0;
  if (krylov && p->q < 1) return fail(h, RSVD_E_INVALID, "block Krylov: q (the number of blocks) must be >= 1");
  const int l = krylov ? l0 * p->q : l0;  // the basis width
  const int kk = (p->flags & RSVD_FLAG_RETURN_FULL_L) ? l : p->k;
  *kk_out = kk;
  if (p->k == 0) return RSVD_OK;
  const int mn = m < n ? m : n;
  if (l > mn) return fail(h, RSVD_E_INVALID, "basis width %d exceeds min(m, n) = %d", l, mn);
  if (l > max_l_for(p->prec))
    return fail(h, RSVD_E_UNSUPPORTED, "basis width %d exceeds the supported maximum %d", l, max_l_for(p->prec));
  if (p->flags & RSVD_FLAG_SINGLE_PASS) {
    if (p->q != 0) return fail(h, RSVD_E_INVALID, "single pass: q must be 0 (A is read once per sketch)");
    if (p->k > 128) return fail(h, RSVD_E_UNSUPPORTED, "single pass: k must be <= 128 (binary64 fit)");
    if (is_fp8(p->prec))
      return fail(h, RSVD_E_UNSUPPORTED, "single pass runs in RSVD_F64, RSVD_F32 and RSVD_MIXED_BF16");
    if (p->flags & (RSVD_FLAG_KRYLOV | RSVD_FLAG_CENTER | RSVD_FLAG_RETURN_FULL_L))
      return fail(h, RSVD_E_INVALID, "single pass takes neither Krylov blocks, centring nor RETURN_FULL_L");
    if ((p->flags & RSVD_FLAG_SYMMETRIC) && m != n)
      return fail(h, RSVD_E_INVALID, "single-pass EVD: A must be square (m = %d, n = %d)", m, n);
  }
  if (p->flags & RSVD_FLAG_SRFT) {
    if (p->q != 0) return fail(h, RSVD_E_INVALID, "SRFT sketch: q must be 0 (Fig. RSVD)");
    if (is_fp8(p->prec))
      return fail(h, RSVD_E_UNSUPPORTED, "SRFT runs in RSVD_F64, RSVD_F32 and RSVD_MIXED_BF16");
    if (p->flags & (RSVD_FLAG_KRYLOV | RSVD_FLAG_CENTER | RSVD_FLAG_SINGLE_PASS))
      return fail(h, RSVD_E_INVALID, "SRFT takes neither Krylov blocks, centring nor the single-pass fit");
    if (2 * l0 > max_l_for(p->prec))
      return fail(h, RSVD_E_UNSUPPORTED, "SRFT: the realified basis 2 (k + p) = %d exceeds %d", 2 * l0,
                  max_l_for(p->prec));
  }
  if (krylov && is_fp8(p->prec))
    return fail(h, RSVD_E_UNSUPPORTED, "block Krylov runs in RSVD_F64, RSVD_F32 and RSVD_MIXED_BF16");
  if (krylov && p->prec == RSVD_MIXED_BF16 && (l0 % 8) != 0)
    return fail(h, RSVD_E_INVALID, "block Krylov in RSVD_MIXED_BF16 needs k + p a multiple of 8");
  if (lda < n) return fail(h, RSVD_E_INVALID, "lda %d < n %d", lda, n);
  if (ldu < kk || ldv < kk) return fail(h, RSVD_E_INVALID, "ldu/ldv smaller than the output rank %d", kk);
  if (!A || !U || !D || !V) return fail(h, RSVD_E_INVALID, "NULL matrix pointer");
  return RSVD_OK;
}

rsvd_status check_access(rsvd_handle_t h, const void* A, const void* U, const void* D, const void* V) {
  const void* ptrs[4] = {A, U, D, V};
  const char* names[4] = {"A", "U", "D", "V"};
  for (int i = 0; i < 4; ++i)
    if (!device_accessible(h, ptrs[i]))
      return fail(h, RSVD_E_INVALID, "%s is not memory the device can access (pin host buffers)", names[i]);
  return RSVD_OK;
}

template <typename T, typename C>
rsvd_status fixed_rank_simt(rsvd_handle_t h, int m, int n, const T* A, int lda, const rsvd_params* p, T* U,
                            int ldu, double* D, T* V, int ldv, const FixedLayout& L, cudaStream_t s,
                            const CentreBufs* cb = nullptr) {
  const int l = p->k + p->p;
  const int kk = (p->flags & RSVD_FLAG_RETURN_FULL_L) ? l : p->k;
  const int sms = h->sms;
  T* Om = (T*)L.Om;
  T* Y = (T*)L.Ybuf;
  T* Z = (T*)L.Zbuf;
  T* part = (T*)L.part;
  const int dt = sizeof(T) == 8 ? RSVD_DT_F64 : RSVD_DT_F32;
  // G = randn(n, l)
  launch_gaussian(n, l, p->seed, 0u, 0, dt, Om, l, s);
  // implicit centring: column means, then a rank-one correction per product
  if (cb) centre_means<T>(m, n, A, lda, *cb, sms, s);
  // Q = orth(A G)
  launch_gemm_simt<T>(false, m, l, n, A, lda, Om, l, Y, l, part, sms, s);
  if (cb) centre_forward<T, T>(m, n, l, Om, l, Y, l, *cb, sms, s);
  run_orth<T, C>(m, l, Y, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
  // q power steps with orth after every product
  for (int j = 0; j < p->q; ++j) {
    launch_gemm_simt<T>(true, n, l, m, A, lda, Y, l, Z, l, part, sms, s);
    if (cb) centre_adjoint<T, T>(m, n, l, Y, l, Z, l, *cb, sms, s);
    run_orth<T, C>(n, l, Z, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
    launch_gemm_simt<T>(false, m, l, n, A, lda, Z, l, Y, l, part, sms, s);
    if (cb) centre_forward<T, T>(m, n, l, Z, l, Y, l, *cb, sms, s);
    run_orth<T, C>(m, l, Y, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
  }
  // B^T = A^T Q, then B^T = Q_B R_B
  launch_gemm_simt<T>(true, n, l, m, A, lda, Y, l, Z, l, part, sms, s);
  if (cb) centre_adjoint<T, T>(m, n, l, Y, l, Z, l, *cb, sms, s);
  run_orth<T, C>(n, l, Z, l, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  // SVD of R_B^T by one-sided Jacobi
  cudaError_t e = launch_jacobi<C>(l, L.Rb, (C*)L.Wt, (C*)L.Jt, L.sigma, L.st, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "jacobi launch: %s", cudaGetErrorString(e));
  launch_sort_gather<C>(l, kk, L.sigma, (const C*)L.Wt, (const C*)L.Jt, D, (C*)L.Wsel, (C*)L.Jsel, s);
  // U = Q Uhat, V = Q_B J, truncated to kk; sign convention
  launch_gemm_simt<T>(false, n, kk, l, Z, l, (const T*)L.Jsel, kk, V, ldv, nullptr, sms, s);
  launch_sign_fix<T, C>(n, kk, l, V, ldv, (C*)L.Wsel, L.part, s);
  launch_gemm_simt<T>(false, m, kk, l, Y, l, (const T*)L.Wsel, kk, U, ldu, nullptr, sms, s);
  return check_launch(h, "rsvd_fixed_rank");
}

// Lambda = Sigma^2 in place (kk values).
__global__ void square_kernel(int kk, double* __restrict__ D) {
  for (int i = threadIdx.x; i < kk; i += blockDim.x) D[i] = D[i] * D[i];
}

// Eigenvalue decomposition of a symmetric positive semi-definite A by the
// Nystrom method (Fig. nystrom), SIMT products:
//   G = randn(n, l); Y = A G; Q = orth(Y); B1 = A Q; B2 = Q^T B1;
//   B2 = C^T C; F = B1 C^-1; [U, Sigma, ~] = svd(F); Lambda = Sigma^2,
// with the SVD of F as in Stage B: F = Q_F R_F, one-sided Jacobi on R_F^T
// (R_F^T J = W), so U = Q_F J and Sigma = the column norms of W.
template <typename T, typename C>
rsvd_status nystrom_simt(rsvd_handle_t h, int n, const T* A, int lda, const rsvd_params* p, T* U, int ldu,
                         double* Lam, const FixedLayout& L, cudaStream_t s) {
  const int l = p->k + p->p;
  const int kk = (p->flags & RSVD_FLAG_RETURN_FULL_L) ? l : p->k;
  const int sms = h->sms;
  T* Om = (T*)L.Om;
  T* Y = (T*)L.Ybuf;
  T* Z = (T*)L.Zbuf;
  T* part = (T*)L.part;
  const int dt = sizeof(T) == 8 ? RSVD_DT_F64 : RSVD_DT_F32;
  launch_gaussian(n, l, p->seed, 0u, 0, dt, Om, l, s);
  // Q = orth(A G)
  launch_gemm_simt<T>(false, n, l, n, A, lda, Om, l, Y, l, part, sms, s);
  run_orth<T, C>(n, l, Y, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
  // B1 = A Q (in Z), B2 = Q^T B1 (l x l, in the n x l buffer of G)
  launch_gemm_simt<T>(false, n, l, n, A, lda, Y, l, Z, l, part, sms, s);
  launch_gemm_simt<T>(true, l, l, n, Y, l, Z, l, Om, l, part, sms, s);
  // F = B1 C^-1, B2 = C^T C
  run_chol_solve<T, C>(n, l, Om, l, Z, l, L.orthws, L.st, sms, s);
  // F = Q_F R_F, SVD of R_F^T
  run_orth<T, C>(n, l, Z, l, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  cudaError_t e = launch_jacobi<C>(l, L.Rb, (C*)L.Wt, (C*)L.Jt, L.sigma, L.st, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "jacobi launch: %s", cudaGetErrorString(e));
  launch_sort_gather<C>(l, kk, L.sigma, (const C*)L.Wt, (const C*)L.Jt, Lam, (C*)L.Wsel, (C*)L.Jsel, s);
  // U = Q_F J, truncated to kk; the largest-magnitude entry of each u_i positive
  launch_gemm_simt<T>(false, n, kk, l, Z, l, (const T*)L.Jsel, kk, U, ldu, nullptr, sms, s);
  launch_sign_fix<T, C>(n, kk, l, U, ldu, (C*)L.Wsel, L.part, s);
  square_kernel<<<1, 256, 0, s>>>(kk, Lam);
  note_launch();
  return check_launch(h, "rsvd_nystrom");
}

inline int round8(int v) { return (v + 7) / 8 * 8; }

// ------------------------------------------------------------ mixed layout --
struct MixedLayout {
  DevStatus* st;
  __nv_bfloat16* Ah;   // m x lda8: bf16(A)
  __nv_bfloat16* Al;   // m x lda8: bf16(A - Ah)
  __nv_bfloat16* Omb;  // n x l8
  float* Y;            // m x l   (Y, then Q)
  __nv_bfloat16* Yb;   // m x l8  bf16(Q)
  __nv_bfloat16* Yl;   // m x l8  bf16(Q - bf16(Q))
  float* Z;            // n x l   (Z, W, B^T, Q_B)
  __nv_bfloat16* Zb;   // n x l8  bf16(W)
  float* part;         // stream-K partials
  void* orthws;
  double* Rb;
  float* Wt;
  float* Jt;
  double* sigma;
  float* Wsel;
  float* Jsel;
  size_t bytes;
};

MixedLayout mixed_layout(void* ws, int m, int n, int l, int kk, int sms) {
  Carver c(ws);
  MixedLayout L;
  const int n8 = round8(n), l8 = round8(l);
  L.st = c.take<DevStatus>(1);
  L.Ah = c.take<__nv_bfloat16>((size_t)m * n8);
  L.Al = c.take<__nv_bfloat16>((size_t)m * n8);
  L.Omb = c.take<__nv_bfloat16>((size_t)n * l8);
  L.Y = c.take<float>((size_t)m * l);
  L.Yb = c.take<__nv_bfloat16>((size_t)m * l8);
  L.Yl = c.take<__nv_bfloat16>((size_t)m * l8);
  L.Z = c.take<float>((size_t)n * l);
  L.Zb = c.take<__nv_bfloat16>((size_t)n * l8);
  size_t pw = tc_gemm_workspace(m, l, n, sms);
  const size_t pw2 = tc_gemm_workspace(n, l, m, sms);
  if (pw2 > pw) pw = pw2;
  const size_t pw3 = simt_gemm_workspace(n, kk, l, sms, 4);
  if (pw3 > pw) pw = pw3;
  if (sign_workspace_bytes(n, kk) > pw) pw = sign_workspace_bytes(n, kk);
  L.part = c.take<float>(pw / sizeof(float) + 1);
  size_t ow = orth_tc_workspace_bytes(m, l, sms);
  const size_t ow2 = orth_tc_workspace_bytes(n, l, sms);
  if (ow2 > ow) ow = ow2;
  L.orthws = c.take<unsigned char>(ow);
  L.Rb = c.take<double>((size_t)l * l);
  L.Wt = c.take<float>((size_t)l * l);
  L.Jt = c.take<float>((size_t)l * l);
  L.sigma = c.take<double>((size_t)l);
  L.Wsel = c.take<float>((size_t)l * kk);
  L.Jsel = c.take<float>((size_t)l * kk);
  L.bytes = c.size();
  return L;
}

cudaEvent_t prof_event(rsvd_handle_t h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one tensor-core product with events when profiling is on.
struct ProfScope {
  rsvd_handle_t h;
  int kind;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  ProfScope(rsvd_handle_t h_, int kind_, cudaStream_t s_) : h(h_), kind(kind_), s(s_) {
    if (h->profile) {
      e0 = prof_event(h);
      cudaEventRecord(e0, s);
    }
  }
  ~ProfScope() {
    if (e0) {
      cudaEvent_t e1 = prof_event(h);
      cudaEventRecord(e1, s);
      h->rec[kind].push_back({e0, e1});
    }
  }
};

rsvd_status tc_call(rsvd_handle_t h, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return RSVD_OK;
}

// Mixed-precision fixed-rank path: bf16 tensor-core sketches with fp32
// accumulation, binary64-accumulated Gram matrices, three-term split-bf16
// projection B^T = A^T Q.
rsvd_status fixed_rank_mixed(rsvd_handle_t h, int m, int n, const float* A, int lda, const rsvd_params* p, float* U,
                             int ldu, double* D, float* V, int ldv, const MixedLayout& L, cudaStream_t s,
                             const CentreBufs* cb = nullptr) {
  const int l = p->k + p->p;
  const int kk = (p->flags & RSVD_FLAG_RETURN_FULL_L) ? l : p->k;
  const int sms = h->sms;
  const int n8 = round8(n), l8 = round8(l);
  rsvd_status st;
  // A = Ah + Al (bf16 pair); the sketches read Ah, the projection both
  launch_split_bf16(m, n, A, lda, L.Ah, L.Al, n8, sms, s);
  // G = randn(n, l), bf16
  launch_gaussian(n, l, p->seed, 0u, 0, RSVD_DT_BF16, L.Omb, l8, s);
  // implicit centring: column means of A, then a rank-one correction per product
  if (cb) centre_means<float>(m, n, A, lda, *cb, sms, s);
  // Q = orth(A G)
  {
    ProfScope ps(h, 0, s);
    if ((st = tc_call(h, launch_tc_gemm(false, false, m, l, n, L.Ah, n8, nullptr, L.Omb, l8, nullptr, L.Y, l, L.part,
                                        sms, L.st, s), "sketch A G")) != RSVD_OK)
      return st;
  }
  if (cb) centre_forward<float, __nv_bfloat16>(m, n, l, L.Omb, l8, L.Y, l, *cb, sms, s);
  run_orth_tc(m, l, L.Y, l, nullptr, L.Yb, l8, L.orthws, L.st, sms, s, p->q > 0);
  // power steps
  for (int j = 0; j < p->q; ++j) {
    {
      ProfScope ps(h, 0, s);
      if ((st = tc_call(h, launch_tc_gemm(true, false, n, l, m, L.Ah, n8, nullptr, L.Yb, l8, nullptr, L.Z, l,
                                          L.part, sms, L.st, s), "sketch A^T Q")) != RSVD_OK)
        return st;
    }
    if (cb) centre_adjoint<float, __nv_bfloat16>(m, n, l, L.Yb, l8, L.Z, l, *cb, sms, s);
    run_orth_tc(n, l, L.Z, l, nullptr, L.Zb, l8, L.orthws, L.st, sms, s, true);
    {
      ProfScope ps(h, 0, s);
      if ((st = tc_call(h, launch_tc_gemm(false, false, m, l, n, L.Ah, n8, nullptr, L.Zb, l8, nullptr, L.Y, l,
                                          L.part, sms, L.st, s), "sketch A W")) != RSVD_OK)
        return st;
    }
    if (cb) centre_forward<float, __nv_bfloat16>(m, n, l, L.Zb, l8, L.Y, l, *cb, sms, s);
    run_orth_tc(m, l, L.Y, l, nullptr, L.Yb, l8, L.orthws, L.st, sms, s, j + 1 < p->q);
  }
  // B^T = A^T Q as Ah^T Qh + Ah^T Ql + Al^T Qh
  launch_split_bf16(m, l, L.Y, l, L.Yb, L.Yl, l8, sms, s);
  {
    ProfScope ps(h, 1, s);
    if ((st = tc_call(h, launch_tc_gemm(true, true, n, l, m, L.Ah, n8, L.Al, L.Yb, l8, L.Yl, L.Z, l, L.part, sms,
                                        L.st, s), "projection")) != RSVD_OK)
      return st;
  }
  if (cb) centre_adjoint<float, float>(m, n, l, L.Y, l, L.Z, l, *cb, sms, s);
  run_orth_tc(n, l, L.Z, l, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  // SVD of R_B^T
  cudaError_t e = launch_jacobi<float>(l, L.Rb, L.Wt, L.Jt, L.sigma, L.st, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "jacobi launch: %s", cudaGetErrorString(e));
  launch_sort_gather<float>(l, kk, L.sigma, L.Wt, L.Jt, D, L.Wsel, L.Jsel, s);
  // U = Q Uhat, V = Q_B J
  launch_gemm_simt<float>(false, n, kk, l, L.Z, l, L.Jsel, kk, V, ldv, nullptr, sms, s);
  launch_sign_fix<float, float>(n, kk, l, V, ldv, L.Wsel, L.part, s);
  launch_gemm_simt<float>(false, m, kk, l, L.Y, l, L.Wsel, kk, U, ldu, nullptr, sms, s);
  return check_launch(h, "rsvd_fixed_rank (mixed)");
}

inline int round16(int v) { return (v + 15) / 16 * 16; }

// e4m3 path: the mixed layout plus the 8-bit copies of A and of the thin operand.
struct Fp8Extra {
  uint8_t* A8;    // m x n16
  uint8_t* A8T;   // n x m16
  float* s;       // m row scales
  float* Om;      // n x l fp32
  uint8_t* X8t;   // l x max(m16, n16)
  float* cvec;    // l column scales
  void* colws;    // fp8_cols scratch
  float* part8;   // e4m3 product partials
  float* amax;    // m: the block maxima of RSVD_MIXED_FP8_B128
  size_t bytes;
};

Fp8Extra fp8_extra(void* ws, int m, int n, int l, int sms) {
  Carver c(ws);
  Fp8Extra E;
  E.A8 = c.take<uint8_t>((size_t)m * round16(n));
  E.A8T = c.take<uint8_t>((size_t)n * round16(m));
  E.s = c.take<float>((size_t)m);
  E.Om = c.take<float>((size_t)n * l);
  const int kmax = round16(m > n ? m : n);
  E.X8t = c.take<uint8_t>((size_t)l * kmax);
  E.cvec = c.take<float>((size_t)l);
  size_t cw = fp8_cols_workspace(m, l);
  if (fp8_cols_workspace(n, l) > cw) cw = fp8_cols_workspace(n, l);
  E.colws = c.take<unsigned char>(cw);
  size_t pw = tc_gemm_e4m3_workspace(m, l, n, sms);
  if (tc_gemm_e4m3_workspace(n, l, m, sms) > pw) pw = tc_gemm_e4m3_workspace(n, l, m, sms);
  E.part8 = c.take<float>(pw / sizeof(float) + 1);
  E.amax = c.take<float>((size_t)m);
  E.bytes = c.size();
  return E;
}

// Workspace of the e4m3 stage call rsvd_sketch(prec = RSVD_MIXED_FP8).
struct SketchFp8 {
  DevStatus* st;
  uint8_t *A8, *A8T, *X8t;
  float *s, *c, *part, *amax;
  void* colws;
  size_t bytes;
};

SketchFp8 sketch_fp8_layout(void* ws, int trans, int m, int n, int l, int sms) {
  Carver c(ws);
  SketchFp8 F;
  F.st = c.take<DevStatus>(1);
  F.A8 = c.take<uint8_t>((size_t)m * round16(n));
  F.A8T = trans ? c.take<uint8_t>((size_t)n * round16(m)) : nullptr;
  F.s = c.take<float>((size_t)m);
  const int K = trans ? m : n, M = trans ? n : m;
  F.X8t = c.take<uint8_t>((size_t)l * round16(K));
  F.c = c.take<float>((size_t)l);
  F.colws = c.take<unsigned char>(fp8_cols_workspace(K, l));
  F.part = c.take<float>(tc_gemm_e4m3_workspace(M, l, K, sms) / sizeof(float) + 1);
  F.amax = c.take<float>((size_t)m);
  F.bytes = c.size();
  return F;
}

// e4m3 sketches (A G, A^T Q, A W) with per-row scales of A and per-column
// scales of the thin operand, then the same split-bf16 projection, small SVD
// and lift as the bf16 path.
rsvd_status fixed_rank_fp8(rsvd_handle_t h, int m, int n, const float* A, int lda, const rsvd_params* p, float* U,
                           int ldu, double* D, float* V, int ldv, const MixedLayout& L, const Fp8Extra& E,
                           cudaStream_t s, const CentreBufs* cb = nullptr) {
  const int l = p->k + p->p;
  const int kk = (p->flags & RSVD_FLAG_RETURN_FULL_L) ? l : p->k;
  const int sms = h->sms;
  const int n8 = round8(n), l8 = round8(l), n16 = round16(n), m16 = round16(m);
  rsvd_status st;
  // one pass over A: A8 with row scales (or, RSVD_MIXED_FP8_B128, the scale
  // of each 128-row block, found by one read of A before it), and the bf16
  // pair for the projection
  const bool b128 = p->prec == RSVD_MIXED_FP8_B128;
  if (b128) launch_fp8_block_max(m, n, A, lda, 128, E.amax, s);
  launch_fp8_rows(m, n, A, lda, E.A8, n16, E.s, L.Ah, L.Al, n8, sms, s, b128 ? E.amax : nullptr);
  launch_u8_transpose(m, n, E.A8, n16, E.A8T, m16, s);
  // G = randn(n, l); Y = A G
  launch_gaussian(n, l, p->seed, 0u, 0, RSVD_DT_F32, E.Om, l, s);
  // implicit centring: column means of A, then a rank-one correction per product
  if (cb) centre_means<float>(m, n, A, lda, *cb, sms, s);
  launch_fp8_cols(n, l, E.Om, l, nullptr, E.X8t, n16, E.cvec, E.colws, s);
  {
    ProfScope ps(h, 0, s);
    if ((st = tc_call(h, launch_tc_gemm_e4m3(m, l, n, E.A8, n16, E.X8t, n16, E.s, E.cvec, L.Y, l, E.part8, sms, L.st,
                                             s), "e4m3 sketch A G")) != RSVD_OK)
      return st;
  }
  if (cb) centre_forward<float, float>(m, n, l, E.Om, l, L.Y, l, *cb, sms, s);
  run_orth_tc(m, l, L.Y, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s, p->q > 0);
  for (int j = 0; j < p->q; ++j) {
    // Z = A^T Q = A8^T (S Q)
    launch_fp8_cols(m, l, L.Y, l, E.s, E.X8t, m16, E.cvec, E.colws, s);
    {
      ProfScope ps(h, 0, s);
      if ((st = tc_call(h, launch_tc_gemm_e4m3(n, l, m, E.A8T, m16, E.X8t, m16, nullptr, E.cvec, L.Z, l, E.part8, sms,
                                               L.st, s), "e4m3 sketch A^T Q")) != RSVD_OK)
        return st;
    }
    if (cb) centre_adjoint<float, float>(m, n, l, L.Y, l, L.Z, l, *cb, sms, s);
    run_orth_tc(n, l, L.Z, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s, true);
    launch_fp8_cols(n, l, L.Z, l, nullptr, E.X8t, n16, E.cvec, E.colws, s);
    {
      ProfScope ps(h, 0, s);
      if ((st = tc_call(h, launch_tc_gemm_e4m3(m, l, n, E.A8, n16, E.X8t, n16, E.s, E.cvec, L.Y, l, E.part8, sms,
                                               L.st, s), "e4m3 sketch A W")) != RSVD_OK)
        return st;
    }
    if (cb) centre_forward<float, float>(m, n, l, L.Z, l, L.Y, l, *cb, sms, s);
    run_orth_tc(m, l, L.Y, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s, j + 1 < p->q);
  }
  // B^T = A^T Q as Ah^T Qh + Ah^T Ql + Al^T Qh
  launch_split_bf16(m, l, L.Y, l, L.Yb, L.Yl, l8, sms, s);
  {
    ProfScope ps(h, 1, s);
    if ((st = tc_call(h, launch_tc_gemm(true, true, n, l, m, L.Ah, n8, L.Al, L.Yb, l8, L.Yl, L.Z, l, L.part, sms,
                                        L.st, s), "projection")) != RSVD_OK)
      return st;
  }
  if (cb) centre_adjoint<float, float>(m, n, l, L.Y, l, L.Z, l, *cb, sms, s);
  run_orth_tc(n, l, L.Z, l, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  cudaError_t e = launch_jacobi<float>(l, L.Rb, L.Wt, L.Jt, L.sigma, L.st, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "jacobi launch: %s", cudaGetErrorString(e));
  launch_sort_gather<float>(l, kk, L.sigma, L.Wt, L.Jt, D, L.Wsel, L.Jsel, s);
  launch_gemm_simt<float>(false, n, kk, l, L.Z, l, L.Jsel, kk, V, ldv, nullptr, sms, s);
  launch_sign_fix<float, float>(n, kk, l, V, ldv, L.Wsel, L.part, s);
  launch_gemm_simt<float>(false, m, kk, l, L.Y, l, L.Wsel, kk, U, ldu, nullptr, sms, s);
  return check_launch(h, "rsvd_fixed_rank (e4m3)");
}

// ------------------------------------------------------------ block Krylov --
// Randomized SVD on the extended sampling matrix (Sec. "Extended sampling
// matrix"): the basis spans [A G, (A A^T) A G, ..., (A A^T)^(q-1) A G], q
// blocks of l = k + p columns, w = q l in all; then Stage B on B = Q^T A.
// The section forms the blocks by plain repeated products; in binary32 their
// scales drift apart as sigma^(2j) and the last blocks lose what the first
// ones hold, so here each new block is taken from the previous block's
// orthonormal basis (Z = orth(A^T Q_(j-1)), Y_j = A Z: the same span, as in
// Fig. RSVDP_stabilized), projected twice against the blocks before it and
// orthonormalized.  In exact arithmetic Q spans the same Krylov space, so U,
// D and V are those of the section's method.
template <typename T>
__global__ void sub_inplace_kernel(int rows, int cols, T* __restrict__ Y, int ldy, const T* __restrict__ X, int ldx) {
  const long long total = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    Y[(size_t)i * ldy + j] -= X[(size_t)i * ldx + j];
  }
}

template <typename T>
void launch_sub_inplace(int rows, int cols, T* Y, int ldy, const T* X, int ldx, int sms, cudaStream_t s) {
  const long long total = (long long)rows * cols;
  if (total == 0) return;
  long long want = (total + 1023) / 1024;
  const int blocks = (int)(want < sms * 8 ? want : sms * 8);
  sub_inplace_kernel<T><<<blocks, 256, 0, s>>>(rows, cols, Y, ldy, X, ldx);
  note_launch();
}

struct KrylovExtra {
  void* C;     // w x l coefficients
  void* T;     // m x l product Q_prev C
  void* part;  // split-K partials of Q_prev^T Y_j
  size_t bytes;
};

KrylovExtra krylov_extra(void* ws, int m, int w, int l, size_t es, int sms) {
  Carver c(ws);
  KrylovExtra K;
  K.C = c.take<unsigned char>((size_t)w * l * es);
  K.T = c.take<unsigned char>((size_t)m * l * es);
  size_t pw = simt_gemm_workspace(w, l, m, sms, es);
  const size_t pw2 = simt_gemm_workspace(m, l, w, sms, es);
  if (pw2 > pw) pw = pw2;
  K.part = c.take<unsigned char>(pw + 256);
  K.bytes = c.size();
  return K;
}

// Y_j (m x l, ld w) -= Q_prev (Q_prev^T Y_j), Q_prev = the jl columns before it; twice.
template <typename T>
void krylov_project(int m, int w, int l, int j, T* Y, const KrylovExtra& K, int sms, cudaStream_t s) {
  T* Yj = Y + (size_t)j * l;
  for (int rep = 0; rep < 2; ++rep) {
    launch_gemm_simt<T>(true, j * l, l, m, Y, w, Yj, w, (T*)K.C, l, (T*)K.part, sms, s);
    launch_gemm_simt<T>(false, m, l, j * l, Y, w, (const T*)K.C, l, (T*)K.T, l, (T*)K.part, sms, s);
    launch_sub_inplace<T>(m, l, Yj, w, (const T*)K.T, l, sms, s);
  }
}

template <typename T, typename C>
rsvd_status fixed_rank_krylov_simt(rsvd_handle_t h, int m, int n, const T* A, int lda, const rsvd_params* p, T* U,
                                   int ldu, double* D, T* V, int ldv, const FixedLayout& L, const KrylovExtra& K,
                                   cudaStream_t s) {
  const int l = p->k + p->p, qb = p->q, w = l * qb;
  const int kk = (p->flags & RSVD_FLAG_RETURN_FULL_L) ? w : p->k;
  const int sms = h->sms;
  T* Om = (T*)L.Om;
  T* Y = (T*)L.Ybuf;  // m x w
  T* Z = (T*)L.Zbuf;  // n x l per block, then B^T n x w
  T* part = (T*)L.part;
  const int dt = sizeof(T) == 8 ? RSVD_DT_F64 : RSVD_DT_F32;
  launch_gaussian(n, l, p->seed, 0u, 0, dt, Om, l, s);
  launch_gemm_simt<T>(false, m, l, n, A, lda, Om, l, Y, w, part, sms, s);
  run_orth<T, C>(m, l, Y, w, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
  for (int j = 1; j < qb; ++j) {
    launch_gemm_simt<T>(true, n, l, m, A, lda, Y + (size_t)(j - 1) * l, w, Z, l, part, sms, s);
    run_orth<T, C>(n, l, Z, l, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
    launch_gemm_simt<T>(false, m, l, n, A, lda, Z, l, Y + (size_t)j * l, w, part, sms, s);
    krylov_project<T>(m, w, l, j, Y, K, sms, s);
    run_orth<T, C>(m, l, Y + (size_t)j * l, w, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
  }
  // B^T = A^T Q (n x w), B^T = Q_B R_B, SVD of R_B^T, lift
  launch_gemm_simt<T>(true, n, w, m, A, lda, Y, w, Z, w, part, sms, s);
  run_orth<T, C>(n, w, Z, w, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  cudaError_t e = launch_jacobi<C>(w, L.Rb, (C*)L.Wt, (C*)L.Jt, L.sigma, L.st, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "jacobi launch: %s", cudaGetErrorString(e));
  launch_sort_gather<C>(w, kk, L.sigma, (const C*)L.Wt, (const C*)L.Jt, D, (C*)L.Wsel, (C*)L.Jsel, s);
  launch_gemm_simt<T>(false, n, kk, w, Z, w, (const T*)L.Jsel, kk, V, ldv, nullptr, sms, s);
  launch_sign_fix<T, C>(n, kk, w, V, ldv, (C*)L.Wsel, L.part, s);
  launch_gemm_simt<T>(false, m, kk, w, Y, w, (const T*)L.Wsel, kk, U, ldu, nullptr, sms, s);
  return check_launch(h, "rsvd_fixed_rank (block Krylov)");
}

// The same on tensor cores (RSVD_MIXED_BF16): bf16 products for the blocks,
// the three-term split-bf16 projection for B^T = A^T Q (w <= 256 columns);
// the projections of the blocks against each other run in binary32.
rsvd_status fixed_rank_krylov_mixed(rsvd_handle_t h, int m, int n, const float* A, int lda, const rsvd_params* p,
                                    float* U, int ldu, double* D, float* V, int ldv, const MixedLayout& L,
                                    const KrylovExtra& K, cudaStream_t s) {
  const int l = p->k + p->p, qb = p->q, w = l * qb;
  const int kk = (p->flags & RSVD_FLAG_RETURN_FULL_L) ? w : p->k;
  const int sms = h->sms;
  const int n8 = round8(n), l8 = round8(l);  // l % 8 == 0, so w8 == w
  rsvd_status st;
  launch_split_bf16(m, n, A, lda, L.Ah, L.Al, n8, sms, s);
  launch_gaussian(n, l, p->seed, 0u, 0, RSVD_DT_BF16, L.Omb, l8, s);
  {
    ProfScope ps(h, 0, s);
    if ((st = tc_call(h, launch_tc_gemm(false, false, m, l, n, L.Ah, n8, nullptr, L.Omb, l8, nullptr, L.Y, w, L.part,
                                        sms, L.st, s), "Krylov block 0")) != RSVD_OK)
      return st;
  }
  run_orth_tc(m, l, L.Y, w, nullptr, L.Yb, w, L.orthws, L.st, sms, s);
  for (int j = 1; j < qb; ++j) {
    {
      ProfScope ps(h, 0, s);
      if ((st = tc_call(h, launch_tc_gemm(true, false, n, l, m, L.Ah, n8, nullptr, L.Yb + (size_t)(j - 1) * l, w,
                                          nullptr, L.Z, l, L.part, sms, L.st, s), "Krylov A^T Q")) != RSVD_OK)
        return st;
    }
    run_orth_tc(n, l, L.Z, l, nullptr, L.Zb, l8, L.orthws, L.st, sms, s);
    {
      ProfScope ps(h, 0, s);
      if ((st = tc_call(h, launch_tc_gemm(false, false, m, l, n, L.Ah, n8, nullptr, L.Zb, l8, nullptr,
                                          L.Y + (size_t)j * l, w, L.part, sms, L.st, s), "Krylov A W")) != RSVD_OK)
        return st;
    }
    krylov_project<float>(m, w, l, j, L.Y, K, sms, s);
    run_orth_tc(m, l, L.Y + (size_t)j * l, w, nullptr, L.Yb + (size_t)j * l, w, L.orthws, L.st, sms, s);
  }
  launch_split_bf16(m, w, L.Y, w, L.Yb, L.Yl, w, sms, s);
  {
    ProfScope ps(h, 1, s);
    if ((st = tc_call(h, launch_tc_gemm(true, true, n, w, m, L.Ah, n8, L.Al, L.Yb, w, L.Yl, L.Z, w, L.part, sms,
                                        L.st, s), "projection")) != RSVD_OK)
      return st;
  }
  run_orth_tc(n, w, L.Z, w, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  cudaError_t e = launch_jacobi<float>(w, L.Rb, L.Wt, L.Jt, L.sigma, L.st, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "jacobi launch: %s", cudaGetErrorString(e));
  launch_sort_gather<float>(w, kk, L.sigma, L.Wt, L.Jt, D, L.Wsel, L.Jsel, s);
  launch_gemm_simt<float>(false, n, kk, w, L.Z, w, L.Jsel, kk, V, ldv, nullptr, sms, s);
  launch_sign_fix<float, float>(n, kk, w, V, ldv, L.Wsel, L.part, s);
  launch_gemm_simt<float>(false, m, kk, w, L.Y, w, L.Wsel, kk, U, ldu, nullptr, sms, s);
  return check_launch(h, "rsvd_fixed_rank (block Krylov, mixed)");
}

// ---------------------------------------------------------- adaptive path --
struct AdaptParams {
  int R;  // max rank
  int b;  // block
};

AdaptParams adapt_params(int m, int n, const rsvd_params* p) {
  AdaptParams a;
  const int mn = m < n ? m : n;
  const int cap = max_l_for(p->prec);
  a.b = p->block > 0 ? p->block : 16;
  a.R = p->max_rank > 0 ? p->max_rank : (mn < cap ? mn : cap);
  return a;
}

rsvd_status validate_adaptive(rsvd_handle_t h, int m, int n, const void* A, int lda, const rsvd_params* p) {
  if (!h) return RSVD_E_INVALID;
  if (!p) return fail(h, RSVD_E_INVALID, "params is NULL");
  if (m < 1 || n < 1) return fail(h, RSVD_E_INVALID, "m and n must be >= 1");
  if (p->prec != RSVD_F64 && p->prec != RSVD_F32)
    return fail(h, RSVD_E_UNSUPPORTED, "rsvd_adaptive_tol supports RSVD_F64 and RSVD_F32");
  if (p->flags & RSVD_FLAG_SPECTRAL) {
    if (!(p->tol > 0.0) || !isfinite(p->tol))
      return fail(h, RSVD_E_INVALID, "spectral mode: tol (absolute eps) must be positive and finite");
    if (p->q != 0) return fail(h, RSVD_E_INVALID, "spectral mode takes no power steps (q must be 0)");
  } else if (!(p->tol > 0.0) || !(p->tol < 1.0)) {
    return fail(h, RSVD_E_INVALID, "tol must lie in (0, 1)");
  }
  if (p->q < 0 || p->q > 8) return fail(h, RSVD_E_INVALID, "q must lie in [0, 8]");
  const AdaptParams a = adapt_params(m, n, p);
  if (a.b < 1 || a.b > 32) return fail(h, RSVD_E_INVALID, "block must lie in [1, 32]");
  const int mn = m < n ? m : n;
  if (a.R < 1 || a.R > mn) return fail(h, RSVD_E_INVALID, "max_rank must lie in [1, min(m, n)]");
  if (a.R > max_l_for(p->prec))
    return fail(h, RSVD_E_UNSUPPORTED, "max_rank %d exceeds the supported maximum %d", a.R, max_l_for(p->prec));
  if (lda < n) return fail(h, RSVD_E_INVALID, "lda %d < n %d", lda, n);
  if (!A) return fail(h, RSVD_E_INVALID, "NULL A");
  return RSVD_OK;
}

struct AdaptLayout {
  DevStatus* st;
  void* abufs;
  void* orthws;
  void* part;
  double* Rb;
  void *Wt, *Jt, *Wsel, *Jsel;
  double* sigma;
  size_t bytes;
};

AdaptLayout adapt_layout(void* ws, int m, int n, const rsvd_params* p, int sms) {
  const AdaptParams a = adapt_params(m, n, p);
  const size_t es = elem_size(p->prec);
  Carver c(ws);
  AdaptLayout L;
  L.st = c.take<DevStatus>(1);
  L.abufs = c.take<unsigned char>(adapt_workspace_bytes(m, n, a.R, a.b, sms, es));
  size_t ow = orth_workspace_bytes(m, a.b, sms, es);
  const size_t ow2 = orth_workspace_bytes(n, a.R, sms, es);
  if (ow2 > ow) ow = ow2;
  L.orthws = c.take<unsigned char>(ow);
  size_t pw = simt_gemm_workspace(n, a.R, a.R, sms, es);
  if (sign_workspace_bytes(n, a.R) > pw) pw = sign_workspace_bytes(n, a.R);
  L.part = c.take<unsigned char>(pw + 256);
  L.Rb = c.take<double>((size_t)a.R * a.R);
  L.Wt = c.take<unsigned char>((size_t)a.R * a.R * es);
  L.Jt = c.take<unsigned char>((size_t)a.R * a.R * es);
  L.Wsel = c.take<unsigned char>((size_t)a.R * a.R * es);
  L.Jsel = c.take<unsigned char>((size_t)a.R * a.R * es);
  L.sigma = c.take<double>((size_t)a.R);
  L.bytes = c.size();
  return L;
}

// Stage B on A ~= Q B (Sec. 3): B^T = Q_B R_B, SVD of R_B^T by one-sided
// Jacobi, U = Q Uhat, V = Q_B J, sign convention; l = rank columns.
template <typename T, typename C>
rsvd_status adapt_stage_b(rsvd_handle_t h, int m, int n, int l, T* Q, int ldq, T* Bt, int ldbt, const AdaptLayout& L,
                          T* U, int ldu, double* D, T* V, int ldv, cudaStream_t s) {
  const int sms = h->sms;
  run_orth<T, C>(n, l, Bt, ldbt, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  cudaError_t e = launch_jacobi<C>(l, L.Rb, (C*)L.Wt, (C*)L.Jt, L.sigma, L.st, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "jacobi launch: %s", cudaGetErrorString(e));
  launch_sort_gather<C>(l, l, L.sigma, (const C*)L.Wt, (const C*)L.Jt, D, (C*)L.Wsel, (C*)L.Jsel, s);
  launch_gemm_simt<T>(false, n, l, l, Bt, ldbt, (const T*)L.Jsel, l, V, ldv, nullptr, sms, s);
  launch_sign_fix<T, C>(n, l, l, V, ldv, (C*)L.Wsel, L.part, s);
  launch_gemm_simt<T>(false, m, l, l, Q, ldq, (const T*)L.Wsel, l, U, ldu, nullptr, sms, s);
  return check_launch(h, "rsvd_adaptive_tol stage B");
}

template <typename T, typename C>
rsvd_status adaptive_impl(rsvd_handle_t h, int m, int n, const T* A, int lda, const rsvd_params* p, T* U, int ldu,
                          double* D, T* V, int ldv, int* rank_out, double* err_out, const AdaptLayout& L,
                          cudaStream_t s) {
  const AdaptParams a = adapt_params(m, n, p);
  T *Q = nullptr, *Bt = nullptr;
  cudaMemsetAsync(L.st, 0, sizeof(DevStatus), s);
  const bool spectral = (p->flags & RSVD_FLAG_SPECTRAL) != 0;
  run_adaptive<T, C>(m, n, A, lda, spectral ? 0.5 : p->tol, a.R, a.b, p->q, p->seed, L.abufs, L.orthws, L.st,
                     h->sms, s, &Q, &Bt, spectral ? p->tol : 0.0);
  rsvd_status st = check_launch(h, "rsvd_adaptive_tol");
  if (st != RSVD_OK) return st;
  // one synchronization: the rank sizes Stage B
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "synchronize: %s", cudaGetErrorString(e));
  DevStatus hs;
  e = cudaMemcpy(&hs, L.st, sizeof(DevStatus), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "status read: %s", cudaGetErrorString(e));
  const int rank = hs.rank;
  if (rank > 0) {
    st = adapt_stage_b<T, C>(h, m, n, rank, Q, a.R, Bt, a.R, L, U, ldu, D, V, ldv, s);
    if (st != RSVD_OK) return st;
  }
  if (rank < a.R) {  // zero the unused trailing triplets
    cudaMemsetAsync(D + rank, 0, (size_t)(a.R - rank) * sizeof(double), s);
    cudaMemset2DAsync(U + rank, (size_t)ldu * sizeof(T), 0, (size_t)(a.R - rank) * sizeof(T), m, s);
    cudaMemset2DAsync(V + rank, (size_t)ldv * sizeof(T), 0, (size_t)(a.R - rank) * sizeof(T), n, s);
  }
  double err = hs.fro2_a > 0.0 ? sqrt(hs.fro2_res > 0.0 ? hs.fro2_res / hs.fro2_a : 0.0) : 0.0;
  if (spectral) {
    // absolute bounds on ||A - Q B||_2: the probe bound of the block that
    // stopped the loop (Lemma thm:aposteriori), else ||A - Q B||_Fro
    err = hs.scratch[2] != 0.0 ? 10.0 * sqrt(2.0 / M_PI) * hs.scratch[1]
                               : sqrt(hs.fro2_res > 0.0 ? hs.fro2_res : 0.0);
  }
  if (rank_out) cudaMemcpyAsync(rank_out, &L.st->rank, sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (err_out) cudaMemcpyAsync(err_out, &err, sizeof(double), cudaMemcpyHostToDevice, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "synchronize: %s", cudaGetErrorString(e));
  int code = 0;
  cudaMemcpy(&code, &L.st->code, sizeof(int), cudaMemcpyDeviceToHost);
  if (code != 0) return fail(h, (rsvd_status)code, "device reported status %d (rank %d)", code, rank);
  return check_launch(h, "rsvd_adaptive_tol");
}

rsvd_status finish_sync(rsvd_handle_t h, const rsvd_params* p, DevStatus* st, cudaStream_t s) {
  if (!(p->flags & RSVD_FLAG_SYNC)) return RSVD_OK;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "synchronize: %s", cudaGetErrorString(e));
  int code = 0;
  e = cudaMemcpy(&code, &st->code, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "status read: %s", cudaGetErrorString(e));
  if (code != 0) return fail(h, (rsvd_status)code, "device reported status %d", code);
  return RSVD_OK;
}

// ------------------------------------------------------- controller path --
constexpr int CTRL_NC = 16;

struct CtrlLayout {
  RsvdCtrlBlock* blk;
  float* G;       // n x 16: probe, then certificate columns
  float* Yp;      // split partials of the thin sketch
  float* Y;       // m x 16
  double* fro2p;  // partial sums of squares
  double* P;      // Gram partials
  double* Gram;   // 16 x 16
  float* T;       // R x 16: V^T G
  float* Tpart;   // split partials of T
  double* rpart;  // judge partials
  void* rest;     // fixed-rank / adaptive workspace
  size_t bytes;
};

CtrlLayout ctrl_layout(void* ws, int m, int n, int R, int sms, size_t rest_bytes) {
  Carver c(ws);
  CtrlLayout L;
  L.blk = c.take<RsvdCtrlBlock>(1);
  L.G = c.take<float>((size_t)n * CTRL_NC);
  L.Yp = c.take<float>((size_t)thin_splits(m, n, sms) * m * CTRL_NC);
  L.Y = c.take<float>((size_t)m * CTRL_NC);
  L.fro2p = c.take<double>((size_t)ceil_div(m, 128) * thin_splits(m, n, sms));
  L.P = c.take<double>((size_t)gram_splits(m, CTRL_NC, sms, 4) * CTRL_NC * CTRL_NC);
  L.Gram = c.take<double>(CTRL_NC * CTRL_NC);
  L.T = c.take<float>((size_t)R * CTRL_NC);
  L.Tpart = c.take<float>(simt_gemm_workspace(R, CTRL_NC, n, sms, 4) / 4 + 1);
  L.rpart = c.take<double>((size_t)resid_blocks(m, sms) * CTRL_NC);
  L.rest = c.take<unsigned char>(rest_bytes);
  L.bytes = c.size();
  return L;
}

// Probe: G = the first 16 columns of the Omega stream; Y = A G and ||A||_F^2
// in one pass; the 16 x 16 Gram of Y in binary64; features into blk.
void run_probe(rsvd_handle_t h, int m, int n, const float* A, int lda, uint64_t seed, const CtrlLayout& L,
               cudaStream_t s) {
  launch_gaussian(n, CTRL_NC, seed, 0u, 0, RSVD_DT_F32, L.G, CTRL_NC, s);
  const int nfro = launch_thin_sketch(m, n, A, lda, L.G, L.Yp, L.Y, L.fro2p, h->sms, s);
  launch_gram<float>(m, CTRL_NC, L.Y, CTRL_NC, L.P, L.Gram, nullptr, h->sms, nullptr, s);
  launch_ctrl_features(m, n, L.Gram, nfro, L.fro2p, L.blk, s);
}

struct CtrlSizes {
  int R, b;
  size_t rest;
};

CtrlSizes ctrl_sizes(rsvd_handle_t h, int m, int n, const rsvd_params* p) {
  CtrlSizes z;
  const int mn = m < n ? m : n;
  z.R = p->max_rank > 0 ? p->max_rank : (mn < 256 ? mn : 256);
  z.b = p->block > 0 ? p->block : 16;
  size_t fx = p->prec == RSVD_MIXED_BF16 ? mixed_layout(nullptr, m, n, z.R, z.R, h->sms).bytes
                                         : fixed_layout(nullptr, m, n, z.R, z.R, RSVD_F32, h->sms).bytes;
  rsvd_params ap = *p;
  ap.prec = RSVD_F32;
  ap.q = 0;
  ap.max_rank = z.R;
  ap.block = z.b;
  const size_t ad = adapt_layout(nullptr, m, n, &ap, h->sms).bytes;
  z.rest = fx > ad ? fx : ad;
  return z;
}

rsvd_status validate_controlled(rsvd_handle_t h, int m, int n, const void* A, int lda, const rsvd_params* p,
                                bool need_theta = true) {
  if (!h) return RSVD_E_INVALID;
  if (!p) return fail(h, RSVD_E_INVALID, "params is NULL");
  if (p->prec != RSVD_F32 && p->prec != RSVD_MIXED_BF16)
    return fail(h, RSVD_E_UNSUPPORTED, "the controller runs RSVD_F32 or RSVD_MIXED_BF16");
  if (m < CTRL_NC || n < CTRL_NC) return fail(h, RSVD_E_INVALID, "the controller needs m, n >= 16");
  if (!(p->tol > 0.0) || !(p->tol < 1.0)) return fail(h, RSVD_E_INVALID, "tol must lie in (0, 1)");
  const int mn = m < n ? m : n;
  const int R = p->max_rank > 0 ? p->max_rank : (mn < 256 ? mn : 256);
  if (R < 1 || R > mn || R > 256) return fail(h, RSVD_E_INVALID, "max_rank must lie in [1, min(m, n, 256)]");
  const int b = p->block > 0 ? p->block : 16;
  if (b < 1 || b > 32) return fail(h, RSVD_E_INVALID, "block must lie in [1, 32]");
  if (lda < n) return fail(h, RSVD_E_INVALID, "lda %d < n %d", lda, n);
  if (!A) return fail(h, RSVD_E_INVALID, "NULL A");
  if (need_theta && !h->ctrl_theta)
    return fail(h, RSVD_E_INVALID, "no controller parameters attached (rsvd_controller_attach)");
  if (p->prec == RSVD_MIXED_BF16 && ((uintptr_t)A & 15) != 0)
    return fail(h, RSVD_E_INVALID, "A must be 16-byte aligned");
  return RSVD_OK;
}

void zero_tail(int m, int n, int r, int R, float* U, int ldu, double* D, float* V, int ldv, cudaStream_t s) {
  if (r >= R) return;
  cudaMemsetAsync(D + r, 0, (size_t)(R - r) * sizeof(double), s);
  cudaMemset2DAsync(U + r, (size_t)ldu * sizeof(float), 0, (size_t)(R - r) * sizeof(float), m, s);
  cudaMemset2DAsync(V + r, (size_t)ldv * sizeof(float), 0, (size_t)(R - r) * sizeof(float), n, s);
}

// Probe -> network -> (l, q) -> rsvd_fixed_rank -> residual estimate ->
// accept and truncate, or fall back to the adaptive range finder.
rsvd_status controlled_impl(rsvd_handle_t h, int m, int n, const float* A, int lda, const rsvd_params* p, float* U,
                            int ldu, double* D, float* V, int ldv, int* rank_out, double* err_out, void* ws,
                            cudaStream_t s) {
  const CtrlSizes z = ctrl_sizes(h, m, n, p);
  const CtrlLayout L = ctrl_layout(ws, m, n, z.R, h->sms, z.rest);
  const int mn = m < n ? m : n;
  const int lmax = z.R < mn ? z.R : mn;
  cudaMemsetAsync(L.blk, 0, sizeof(RsvdCtrlBlock), s);
  run_probe(h, m, n, A, lda, p->seed, L, s);
  cudaError_t e = launch_mlp(-1, 1, L.blk->feat, nullptr, nullptr, 0.f, h->ctrl_theta, L.blk->logits, nullptr,
                             nullptr, nullptr, 0, 0.f, nullptr, nullptr, s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "controller network: %s", cudaGetErrorString(e));
  launch_ctrl_decide(L.blk, (float)h->ctrl_quantile, lmax, s);
  rsvd_status st = check_launch(h, "controller probe");
  if (st != RSVD_OK) return st;
  RsvdCtrlBlock hb;
  e = cudaMemcpyAsync(&hb, L.blk, sizeof(hb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "controller read: %s", cudaGetErrorString(e));
  int l = hb.l_hat < 1 ? 1 : (hb.l_hat > lmax ? lmax : hb.l_hat);
  int q = hb.q_hat;
  h->ctrl_info[0] = l;
  h->ctrl_info[1] = q;
  h->ctrl_info[3] = 0;
  // one fixed-rank solve with (l, q), all l triplets returned, and the judge:
  // E = A Gc - U (D (V^T Gc)), Gc = 16 columns of Philox stream 2
  int fcode = 0;
  auto solve_and_judge = [&](int ll, int qq) -> rsvd_status {
    rsvd_params fp = *p;
    fp.k = ll;
    fp.p = 0;
    fp.q = qq;
    fp.flags = RSVD_FLAG_RETURN_FULL_L;
    DevStatus* fst;
    rsvd_status r2;
    if (p->prec == RSVD_MIXED_BF16) {
      const MixedLayout M = mixed_layout(L.rest, m, n, ll, ll, h->sms);
      fst = M.st;
      cudaMemsetAsync(M.st, 0, sizeof(DevStatus), s);
      r2 = fixed_rank_mixed(h, m, n, A, lda, &fp, U, ldu, D, V, ldv, M, s);
    } else {
      const FixedLayout F = fixed_layout(L.rest, m, n, ll, ll, RSVD_F32, h->sms);
      fst = F.st;
      cudaMemsetAsync(F.st, 0, sizeof(DevStatus), s);
      r2 = fixed_rank_simt<float, float>(h, m, n, A, lda, &fp, U, ldu, D, V, ldv, F, s);
    }
    if (r2 != RSVD_OK) return r2;
    launch_gaussian(n, CTRL_NC, p->seed, 2u, 0, RSVD_DT_F32, L.G, CTRL_NC, s);
    launch_thin_sketch(m, n, A, lda, L.G, L.Yp, L.Y, nullptr, h->sms, s);
    launch_gemm_simt<float>(true, ll, CTRL_NC, n, V, ldv, L.G, CTRL_NC, L.T, CTRL_NC, L.Tpart, h->sms, s);
    launch_judge(m, ll, L.Y, U, ldu, D, L.T, L.rpart, p->tol, h->ctrl_safety, L.blk, h->sms, s);
    r2 = check_launch(h, "controller judge");
    if (r2 != RSVD_OK) return r2;
    cudaError_t e2 = cudaMemcpyAsync(&hb, L.blk, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&fcode, &fst->code, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
    if (e2 != cudaSuccess) return fail(h, RSVD_E_CUDA, "judge read: %s", cudaGetErrorString(e2));
    const double fro = sqrt(hb.fro2 > 0.0 ? hb.fro2 : 0.0);
    h->ctrl_info[2] = (hb.accepted && fcode == 0) ? 1 : 0;
    h->ctrl_est[0] = fro > 0.0 ? sqrt(hb.est2) / fro : 0.0;
    h->ctrl_est[1] = fro > 0.0 ? hb.spec_bound / fro : 0.0;
    return RSVD_OK;
  };
  auto accept = [&]() -> rsvd_status {
    const int r = hb.rank;
    zero_tail(m, n, r, z.R, U, ldu, D, V, ldv, s);
    const double err = h->ctrl_est[0];
    if (rank_out) cudaMemcpyAsync(rank_out, &r, sizeof(int), cudaMemcpyHostToDevice, s);
    if (err_out) cudaMemcpyAsync(err_out, &err, sizeof(double), cudaMemcpyHostToDevice, s);
    h->ctrl_info[4] = r;
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e2 != cudaSuccess) return fail(h, RSVD_E_CUDA, "synchronize: %s", cudaGetErrorString(e2));
    return check_launch(h, "rsvd_adaptive_tol (controller)");
  };
  if ((st = solve_and_judge(l, q)) != RSVD_OK) return st;
  if (h->ctrl_info[2]) return accept();
  if (l < lmax && h->ctrl_fallback == 1) {
    // escalate: the largest rank allowed, at least two power steps
    l = lmax;
    q = q > 2 ? q : 2;
    h->ctrl_info[0] = l;
    h->ctrl_info[1] = q;
    h->ctrl_info[3] = 2;
    if ((st = solve_and_judge(l, q)) != RSVD_OK) return st;
    if (h->ctrl_info[2]) return accept();
  } else if (l < z.R) {
    // fall back: the blocked adaptive range finder in binary32, q = 0
    rsvd_params ap = *p;
    ap.prec = RSVD_F32;
    ap.q = 0;
    ap.max_rank = z.R;
    ap.block = z.b;
    ap.flags = 0;
    const AdaptLayout AL = adapt_layout(L.rest, m, n, &ap, h->sms);
    h->ctrl_info[3] = 1;
    st = adaptive_impl<float, float>(h, m, n, A, lda, &ap, U, ldu, D, V, ldv, rank_out, err_out, AL, s);
    int r = 0;
    cudaMemcpy(&r, &AL.st->rank, sizeof(int), cudaMemcpyDeviceToHost);
    h->ctrl_info[4] = r;
    return st;
  }
  // the largest rank allowed already misses the tolerance
  zero_tail(m, n, l, z.R, U, ldu, D, V, ldv, s);
  const double err = h->ctrl_est[0];
  if (rank_out) cudaMemcpyAsync(rank_out, &l, sizeof(int), cudaMemcpyHostToDevice, s);
  if (err_out) cudaMemcpyAsync(err_out, &err, sizeof(double), cudaMemcpyHostToDevice, s);
  h->ctrl_info[4] = l;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, RSVD_E_CUDA, "synchronize: %s", cudaGetErrorString(e));
  if (fcode != 0) return fail(h, (rsvd_status)fcode, "fixed-rank solve reported status %d", fcode);
  return fail(h, RSVD_E_NOT_CONVERGED, "estimated residual %.3e above tol %.3e at the largest rank %d", err, p->tol,
              l);
}

}  // namespace

// Accessors for translation units that only see the opaque handle.
int handle_device(rsvd_handle_t h) { return h->device; }
int handle_sms(rsvd_handle_t h) { return h->sms; }
rsvd_status handle_fail(rsvd_handle_t h, rsvd_status code, const char* msg) { return fail(h, code, "%s", msg); }

}  // namespace rsvd

using namespace rsvd;

extern "C" {

rsvd_status rsvd_create(rsvd_handle_t* handle, int device) {
  if (!handle) return RSVD_E_INVALID;
  *handle = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return RSVD_E_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return RSVD_E_CUDA;
  rsvd_handle_s* h = new (std::nothrow) rsvd_handle_s();
  if (!h) return RSVD_E_NOMEM;
  h->device = device;
  h->err[0] = 0;
  h->profile = false;
  h->ctrl_theta = nullptr;
  h->ctrl_quantile = 0.9;
  h->ctrl_safety = 0.8;
  h->ctrl_fallback = 0;
  h->batched_variant = -1;
  if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete h;
    return RSVD_E_CUDA;
  }
  *handle = h;
  return RSVD_OK;
}

rsvd_status rsvd_destroy(rsvd_handle_t handle) {
  if (!handle) return RSVD_OK;
  for (auto e : handle->pool) cudaEventDestroy(e);
  for (auto& r : handle->rec)
    for (auto& pr : r) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  delete handle;
  return RSVD_OK;
}

rsvd_status rsvd_kernel_launches(rsvd_handle_t handle, long long* count) {
  if (!handle || !count) return RSVD_E_INVALID;
  *count = launch_counter().load();
  return RSVD_OK;
}

rsvd_status rsvd_profile(rsvd_handle_t handle, int on) {
  if (!handle) return RSVD_E_INVALID;
  handle->profile = on != 0;
  return RSVD_OK;
}

rsvd_status rsvd_profile_read(rsvd_handle_t handle, int kind, double* total_ms, long long* launches) {
  if (!handle || kind < 0 || kind > 1 || !total_ms || !launches) return RSVD_E_INVALID;
  double tot = 0.0;
  long long cnt = 0;
  for (auto& pr : handle->rec[kind]) {
    if (cudaEventSynchronize(pr.second) != cudaSuccess) return fail(handle, RSVD_E_CUDA, "profile event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pr.first, pr.second);
    tot += ms;
    ++cnt;
    handle->pool.push_back(pr.first);
    handle->pool.push_back(pr.second);
  }
  handle->rec[kind].clear();
  *total_ms = tot;
  *launches = cnt;
  return RSVD_OK;
}

rsvd_status rsvd_last_error_detail(rsvd_handle_t handle, char* buf, size_t len) {
  if (!handle || !buf || len == 0) return RSVD_E_INVALID;
  strncpy(buf, handle->err, len - 1);
  buf[len - 1] = 0;
  return RSVD_OK;
}

rsvd_status rsvd_workspace_size(rsvd_handle_t handle, int m, int n, const rsvd_params* params, size_t* bytes) {
  if (!handle || !params || !bytes) return RSVD_E_INVALID;
  if (params->tol > 0.0 && (params->flags & RSVD_FLAG_USE_CONTROLLER)) {
    rsvd_status st = validate_controlled(handle, m, n, (const void*)16, n, params, false);
    if (st != RSVD_OK) return st;
    const CtrlSizes z = ctrl_sizes(handle, m, n, params);
    *bytes = ctrl_layout(nullptr, m, n, z.R, handle->sms, z.rest).bytes;
    return RSVD_OK;
  }
  if (params->tol > 0.0) {
    rsvd_status st = validate_adaptive(handle, m, n, (const void*)1, n, params);
    if (st != RSVD_OK) return st;
    *bytes = adapt_layout(nullptr, m, n, params, handle->sms).bytes;
    return RSVD_OK;
  }
  int kk = 0;
  rsvd_status st = validate_fixed(handle, m, n, (const void*)1, n, params, (const void*)1, 1 << 30,
                                  (const void*)1, (const void*)1, 1 << 30, &kk);
  if (st != RSVD_OK) return st;
  int l = params->k + params->p;
  if (params->flags & RSVD_FLAG_SRFT) {
    const size_t es = params->prec == RSVD_F64 ? 8 : 4;
    *bytes = srft_layout(nullptr, m, n, l, kk, es, handle->sms, params->prec == RSVD_MIXED_BF16).bytes;
    return RSVD_OK;
  }
  if (params->flags & RSVD_FLAG_SINGLE_PASS) {
    const size_t es = params->prec == RSVD_F64 ? 8 : 4;
    *bytes = single_pass_layout(nullptr, m, n, params->k, l, es, handle->sms, params->prec == RSVD_MIXED_BF16).bytes;
    return RSVD_OK;
  }
  if (params->flags & RSVD_FLAG_KRYLOV) {
    const int l0 = l;
    l *= params->q;
    const size_t es = params->prec == RSVD_F64 ? 8 : 4;
    const size_t base = params->prec == RSVD_MIXED_BF16 ? mixed_layout(nullptr, m, n, l, kk, handle->sms).bytes
                                                        : fixed_layout(nullptr, m, n, l, kk, params->prec, handle->sms).bytes;
    *bytes = base + krylov_extra(nullptr, m, l, l0, es, handle->sms).bytes;
    if (params->flags & RSVD_FLAG_CENTER) return fail(handle, RSVD_E_UNSUPPORTED, "block Krylov does not centre");
    return RSVD_OK;
  }
  if (params->prec == RSVD_MIXED_BF16)
    *bytes = mixed_layout(nullptr, m, n, l, kk, handle->sms).bytes;
  else if (is_fp8(params->prec))
    *bytes = mixed_layout(nullptr, m, n, l, kk, handle->sms).bytes + fp8_extra(nullptr, m, n, l, handle->sms).bytes;
  else
    *bytes = fixed_layout(nullptr, m, n, l, kk, params->prec, handle->sms).bytes;
  if (params->flags & RSVD_FLAG_CENTER) *bytes += centre_workspace_bytes(m, n, l, handle->sms);
  return RSVD_OK;
}

rsvd_status rsvd_fixed_rank(rsvd_handle_t handle, int m, int n, const void* A, int lda, const rsvd_params* params,
                            void* U, int ldu, double* D, void* V, int ldv, void* workspace, size_t ws_bytes,
                            rsvd_stream_t stream) {
  int kk = 0;
  rsvd_status st = validate_fixed(handle, m, n, A, lda, params, U, ldu, D, V, ldv, &kk);
  if (st != RSVD_OK) return st;
  if (params->k == 0) return RSVD_OK;
  if ((st = check_access(handle, A, U, D, V)) != RSVD_OK) return st;
  const int l = params->k + params->p;
  cudaStream_t s = (cudaStream_t)stream;
  size_t need = 0;
  st = rsvd_workspace_size(handle, m, n, params, &need);
  if (st != RSVD_OK) return st;
  if (!workspace || ws_bytes < need)
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
  if (params->flags & RSVD_FLAG_SRFT) {
    const bool mixed = params->prec == RSVD_MIXED_BF16;
    const size_t es = params->prec == RSVD_F64 ? 8 : 4;
    if (mixed && ((uintptr_t)A & 15) != 0) return fail(handle, RSVD_E_INVALID, "A must be 16-byte aligned");
    const SrftLayout L = srft_layout(workspace, m, n, l, kk, es, handle->sms, mixed);
    cudaMemsetAsync(L.st, 0, sizeof(DevStatus), s);
    cudaError_t e;
    if (params->prec == RSVD_F64)
      e = run_srft<double>(m, n, (const double*)A, lda, params->k, params->p, kk, params->seed, (double*)U, ldu, D,
                           (double*)V, ldv, L, handle->sms, false, s);
    else
      e = run_srft<float>(m, n, (const float*)A, lda, params->k, params->p, kk, params->seed, (float*)U, ldu, D,
                          (float*)V, ldv, L, handle->sms, mixed, s);
    if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "SRFT solve: %s", cudaGetErrorString(e));
    st = check_launch(handle, "rsvd_fixed_rank (SRFT)");
    if (st != RSVD_OK) return st;
    return finish_sync(handle, params, L.st, s);
  }
  if (params->flags & RSVD_FLAG_SINGLE_PASS) {
    const bool mixed = params->prec == RSVD_MIXED_BF16;
    const size_t es = params->prec == RSVD_F64 ? 8 : 4;
    if (mixed && ((uintptr_t)A & 15) != 0) return fail(handle, RSVD_E_INVALID, "A must be 16-byte aligned");
    const SinglePassLayout L = single_pass_layout(workspace, m, n, params->k, l, es, handle->sms, mixed);
    cudaMemsetAsync(L.st, 0, sizeof(DevStatus), s);
    const bool sym = (params->flags & RSVD_FLAG_SYMMETRIC) != 0;
    if (params->prec == RSVD_F64) {
      if (sym)
        run_single_pass_evd<double>(n, (const double*)A, lda, params->k, params->p, params->seed, (double*)U, ldu, D,
                                    (double*)V, ldv, L, handle->sms, false, s);
      else
        run_single_pass_svd<double>(m, n, (const double*)A, lda, params->k, params->p, params->seed, (double*)U, ldu,
                                    D, (double*)V, ldv, L, handle->sms, false, s);
    } else {
      if (sym)
        run_single_pass_evd<float>(n, (const float*)A, lda, params->k, params->p, params->seed, (float*)U, ldu, D,
                                   (float*)V, ldv, L, handle->sms, mixed, s);
      else
        run_single_pass_svd<float>(m, n, (const float*)A, lda, params->k, params->p, params->seed, (float*)U, ldu, D,
                                   (float*)V, ldv, L, handle->sms, mixed, s);
    }
    st = check_launch(handle, "rsvd_fixed_rank (single pass)");
    if (st != RSVD_OK) return st;
    return finish_sync(handle, params, L.st, s);
  }
  if (params->flags & RSVD_FLAG_KRYLOV) {
    const int w = l * params->q;
    const size_t es = params->prec == RSVD_F64 ? 8 : 4;
    if (params->prec == RSVD_MIXED_BF16) {
      if (((uintptr_t)A & 15) != 0) return fail(handle, RSVD_E_INVALID, "A must be 16-byte aligned");
      const MixedLayout M = mixed_layout(workspace, m, n, w, kk, handle->sms);
      const KrylovExtra K = krylov_extra((char*)workspace + M.bytes, m, w, l, es, handle->sms);
      cudaMemsetAsync(M.st, 0, sizeof(DevStatus), s);
      st = fixed_rank_krylov_mixed(handle, m, n, (const float*)A, lda, params, (float*)U, ldu, D, (float*)V, ldv, M,
                                   K, s);
      if (st != RSVD_OK) return st;
      return finish_sync(handle, params, M.st, s);
    }
    const FixedLayout L = fixed_layout(workspace, m, n, w, kk, params->prec, handle->sms);
    const KrylovExtra K = krylov_extra((char*)workspace + L.bytes, m, w, l, es, handle->sms);
    cudaMemsetAsync(L.st, 0, sizeof(DevStatus), s);
    if (params->prec == RSVD_F64)
      st = fixed_rank_krylov_simt<double, double>(handle, m, n, (const double*)A, lda, params, (double*)U, ldu, D,
                                                  (double*)V, ldv, L, K, s);
    else
      st = fixed_rank_krylov_simt<float, float>(handle, m, n, (const float*)A, lda, params, (float*)U, ldu, D,
                                                (float*)V, ldv, L, K, s);
    if (st != RSVD_OK) return st;
    return finish_sync(handle, params, L.st, s);
  }
  // implicit centring buffers sit after the path's own layout
  const bool centre = (params->flags & RSVD_FLAG_CENTER) != 0;
  CentreBufs cbuf;
  const CentreBufs* cb = nullptr;
  auto carve_centre = [&](size_t off) {
    if (!centre) return;
    cbuf = centre_carve((char*)workspace + off, m, n, l, handle->sms);
    cb = &cbuf;
  };
  if (params->prec == RSVD_MIXED_BF16) {
    if (((uintptr_t)A & 15) != 0) return fail(handle, RSVD_E_INVALID, "A must be 16-byte aligned");
    const MixedLayout M = mixed_layout(workspace, m, n, l, kk, handle->sms);
    carve_centre(M.bytes);
    cudaMemsetAsync(M.st, 0, sizeof(DevStatus), s);
    st = fixed_rank_mixed(handle, m, n, (const float*)A, lda, params, (float*)U, ldu, D, (float*)V, ldv, M, s, cb);
    if (st != RSVD_OK) return st;
    return finish_sync(handle, params, M.st, s);
  }
  if (is_fp8(params->prec)) {
    if (((uintptr_t)A & 15) != 0) return fail(handle, RSVD_E_INVALID, "A must be 16-byte aligned");
    const MixedLayout M = mixed_layout(workspace, m, n, l, kk, handle->sms);
    const Fp8Extra E = fp8_extra((char*)workspace + M.bytes, m, n, l, handle->sms);
    carve_centre(M.bytes + E.bytes);
    cudaMemsetAsync(M.st, 0, sizeof(DevStatus), s);
    st = fixed_rank_fp8(handle, m, n, (const float*)A, lda, params, (float*)U, ldu, D, (float*)V, ldv, M, E, s, cb);
    if (st != RSVD_OK) return st;
    return finish_sync(handle, params, M.st, s);
  }
  const FixedLayout L = fixed_layout(workspace, m, n, l, kk, params->prec, handle->sms);
  carve_centre(L.bytes);
  cudaMemsetAsync(L.st, 0, sizeof(DevStatus), s);
  if (params->prec == RSVD_F64)
    st = fixed_rank_simt<double, double>(handle, m, n, (const double*)A, lda, params, (double*)U, ldu, D,
                                         (double*)V, ldv, L, s, cb);
  else
    st = fixed_rank_simt<float, float>(handle, m, n, (const float*)A, lda, params, (float*)U, ldu, D, (float*)V,
                                       ldv, L, s, cb);
  if (st != RSVD_OK) return st;
  return finish_sync(handle, params, L.st, s);
}

rsvd_status rsvd_nystrom(rsvd_handle_t handle, int n, const void* A, int lda, const rsvd_params* params, void* U,
                         int ldu, double* Lam, void* workspace, size_t ws_bytes, rsvd_stream_t stream) {
  int kk = 0;
  rsvd_status st = validate_fixed(handle, n, n, A, lda, params, U, ldu, Lam, U, ldu, &kk);
  if (st != RSVD_OK) return st;
  if (params->prec != RSVD_F32 && params->prec != RSVD_F64)
    return fail(handle, RSVD_E_UNSUPPORTED, "rsvd_nystrom supports RSVD_F32 and RSVD_F64");
  if (params->q != 0) return fail(handle, RSVD_E_UNSUPPORTED, "rsvd_nystrom has no power steps (q must be 0)");
  if (params->k == 0) return RSVD_OK;
  if ((st = check_access(handle, A, U, Lam, U)) != RSVD_OK) return st;
  size_t need = 0;
  st = rsvd_workspace_size(handle, n, n, params, &need);
  if (st != RSVD_OK) return st;
  if (!workspace || ws_bytes < need)
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
  const int l = params->k + params->p;
  cudaStream_t s = (cudaStream_t)stream;
  const FixedLayout L = fixed_layout(workspace, n, n, l, kk, params->prec, handle->sms);
  cudaMemsetAsync(L.st, 0, sizeof(DevStatus), s);
  if (params->prec == RSVD_F64)
    st = nystrom_simt<double, double>(handle, n, (const double*)A, lda, params, (double*)U, ldu, Lam, L, s);
  else
    st = nystrom_simt<float, float>(handle, n, (const float*)A, lda, params, (float*)U, ldu, Lam, L, s);
  if (st != RSVD_OK) return st;
  return finish_sync(handle, params, L.st, s);
}

rsvd_status rsvd_adaptive_tol(rsvd_handle_t handle, int m, int n, const void* A, int lda, const rsvd_params* params,
                              void* U, int ldu, double* D, void* V, int ldv, int* rank_out, double* err_out,
                              void* workspace, size_t ws_bytes, rsvd_stream_t stream) {
  if (params && (params->flags & RSVD_FLAG_USE_CONTROLLER)) {
    rsvd_status st = validate_controlled(handle, m, n, A, lda, params);
    if (st != RSVD_OK) return st;
    const CtrlSizes z = ctrl_sizes(handle, m, n, params);
    if (ldu < z.R || ldv < z.R) return fail(handle, RSVD_E_INVALID, "ldu/ldv smaller than max_rank %d", z.R);
    if (!U || !D || !V) return fail(handle, RSVD_E_INVALID, "NULL output pointer");
    const size_t need = ctrl_layout(nullptr, m, n, z.R, handle->sms, z.rest).bytes;
    if (!workspace || ws_bytes < need)
      return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
    if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
    return controlled_impl(handle, m, n, (const float*)A, lda, params, (float*)U, ldu, D, (float*)V, ldv, rank_out,
                           err_out, workspace, (cudaStream_t)stream);
  }
  rsvd_status st = validate_adaptive(handle, m, n, A, lda, params);
  if (st != RSVD_OK) return st;
  const AdaptParams a = adapt_params(m, n, params);
  if (ldu < a.R || ldv < a.R) return fail(handle, RSVD_E_INVALID, "ldu/ldv smaller than max_rank %d", a.R);
  if (!U || !D || !V) return fail(handle, RSVD_E_INVALID, "NULL output pointer");
  const AdaptLayout need = adapt_layout(nullptr, m, n, params, handle->sms);
  if (!workspace || ws_bytes < need.bytes)
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need.bytes);
  if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
  const AdaptLayout L = adapt_layout(workspace, m, n, params, handle->sms);
  cudaStream_t s = (cudaStream_t)stream;
  if (params->prec == RSVD_F64)
    return adaptive_impl<double, double>(handle, m, n, (const double*)A, lda, params, (double*)U, ldu, D, (double*)V,
                                         ldv, rank_out, err_out, L, s);
  return adaptive_impl<float, float>(handle, m, n, (const float*)A, lda, params, (float*)U, ldu, D, (float*)V, ldv,
                                     rank_out, err_out, L, s);
}

namespace {

constexpr int BATCHED_MAX_COUNT = 65536;

rsvd_status validate_batched(rsvd_handle_t h, int count, const rsvd_params* p, int* R, int* b) {
  if (!h) return RSVD_E_INVALID;
  if (!p) return fail(h, RSVD_E_INVALID, "params is NULL");
  if (count < 0 || count > BATCHED_MAX_COUNT)
    return fail(h, RSVD_E_INVALID, "count %d outside [0, %d]", count, BATCHED_MAX_COUNT);
  if (p->prec != RSVD_F32) return fail(h, RSVD_E_UNSUPPORTED, "rsvd_batched supports RSVD_F32");
  if (p->q != 0) return fail(h, RSVD_E_UNSUPPORTED, "rsvd_batched has no power steps (q must be 0)");
  if (!(p->tol > 0.0) || !(p->tol < 1.0)) return fail(h, RSVD_E_INVALID, "tol must lie in (0, 1)");
  if (p->q < 0 || p->q > 8) return fail(h, RSVD_E_INVALID, "q must lie in [0, 8]");
  *b = p->block > 0 ? p->block : batched_max_block();
  if (*b < 1 || *b > batched_max_block())
    return fail(h, RSVD_E_INVALID, "block must lie in [1, %d]", batched_max_block());
  *R = p->max_rank > 0 ? p->max_rank : batched_max_rank();
  if (*R < 1 || *R > batched_max_rank())
    return fail(h, RSVD_E_INVALID, "max_rank must lie in [1, %d]", batched_max_rank());
  return RSVD_OK;
}

}  // namespace

rsvd_status rsvd_batched_workspace_size(rsvd_handle_t handle, int count, const rsvd_params* params, size_t* bytes) {
  int R = 0, b = 0;
  if (!bytes) return RSVD_E_INVALID;
  rsvd_status st = validate_batched(handle, count, params, &R, &b);
  if (st != RSVD_OK) return st;
  *bytes = batched_workspace_bytes(count, handle->sms);
  return RSVD_OK;
}

rsvd_status rsvd_batched(rsvd_handle_t handle, int count, const int* m, const int* n, const void* const* A,
                         const int* lda, const rsvd_params* params, void* const* U, double* const* D, void* const* V,
                         int* rank_out, double* err_out, int* status_out, void* workspace, size_t ws_bytes,
                         rsvd_stream_t stream) {
  int R = 0, b = 0;
  rsvd_status st = validate_batched(handle, count, params, &R, &b);
  if (st != RSVD_OK) return st;
  if (count == 0) return RSVD_OK;
  if (!m || !n || !A || !lda || !U || !D || !V) return fail(handle, RSVD_E_INVALID, "NULL array argument");
  const size_t need = batched_workspace_bytes(count, handle->sms);
  if (!workspace || ws_bytes < need)
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e =
      launch_batched(count, m, n, lda, (const float* const*)A, (float* const*)U, D, (float* const*)V, R, b,
                     params->seed, params->tol, rank_out, err_out, status_out, workspace, handle->sms, s,
                     handle->batched_variant);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_batched launch: %s", cudaGetErrorString(e));
  return finish_sync(handle, params, (DevStatus*)workspace, s);
}

rsvd_status rsvd_batched_variants(int* count) {
  if (!count) return RSVD_E_INVALID;
  *count = batched_variants();
  return RSVD_OK;
}

rsvd_status rsvd_batched_variant_info(int variant, int* rows_ahead, int* cols_ahead) {
  if (variant < 0 || variant >= batched_variants() || !rows_ahead || !cols_ahead) return RSVD_E_INVALID;
  batched_variant_info(variant, rows_ahead, cols_ahead);
  return RSVD_OK;
}

rsvd_status rsvd_batched_set_variant(rsvd_handle_t handle, int variant) {
  if (!handle) return RSVD_E_INVALID;
  if (variant < -1 || variant >= batched_variants())
    return fail(handle, RSVD_E_INVALID, "variant must lie in [-1, %d]", batched_variants() - 1);
  handle->batched_variant = variant;
  return RSVD_OK;
}

rsvd_status rsvd_batched_get_variant(rsvd_handle_t handle, int* variant) {
  if (!handle || !variant) return RSVD_E_INVALID;
  *variant = handle->batched_variant < 0 ? batched_default_variant() : handle->batched_variant;
  return RSVD_OK;
}

rsvd_status rsvd_batched_autotune(rsvd_handle_t handle, int count, const int* m, const int* n, const void* const* A,
                                  const int* lda, const rsvd_params* params, void* const* U, double* const* D,
                                  void* const* V, int* rank_out, double* err_out, int* status_out, void* workspace,
                                  size_t ws_bytes, rsvd_stream_t stream, float* ms_out, int* variant_out) {
  int R = 0, b = 0;
  rsvd_status st = validate_batched(handle, count, params, &R, &b);
  if (st != RSVD_OK) return st;
  if (!m || !n || !A || !lda || !U || !D || !V) return fail(handle, RSVD_E_INVALID, "NULL array argument");
  const size_t need = batched_workspace_bytes(count, handle->sms);
  if (!workspace || ws_bytes < need)
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const int nv = batched_variants();
  int best = batched_default_variant();
  float best_ms = 0.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(handle, RSVD_E_CUDA, "event create failed");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(handle, RSVD_E_CUDA, "event create failed");
  }
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < nv && e == cudaSuccess && count > 0; ++v) {
    // one untimed run (first launch of the variant), then one timed run
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      if (rep == 1) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess)
        e = launch_batched(count, m, n, lda, (const float* const*)A, (float* const*)U, D, (float* const*)V, R, b,
                           params->seed, params->tol, rank_out, err_out, status_out, workspace, handle->sms, s, v);
      if (rep == 1 && e == cudaSuccess) e = cudaEventRecord(e1, s);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
      if (ms_out) ms_out[v] = ms;
      if (v == 0 || ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_batched_autotune: %s", cudaGetErrorString(e));
  handle->batched_variant = best;
  if (variant_out) *variant_out = best;
  int code = 0;
  e = cudaMemcpy(&code, &((const DevStatus*)workspace)->code, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "status read: %s", cudaGetErrorString(e));
  if (code != RSVD_OK) return fail(handle, (rsvd_status)code, "a problem of the batch reported status %d", code);
  return RSVD_OK;
}

rsvd_status rsvd_query_status(rsvd_handle_t handle, const void* workspace, int* status, rsvd_stream_t stream) {
  if (!handle || !workspace || !status) return RSVD_E_INVALID;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "synchronize: %s", cudaGetErrorString(e));
  e = cudaMemcpy(status, &((const DevStatus*)workspace)->code, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "status read: %s", cudaGetErrorString(e));
  return RSVD_OK;
}

rsvd_status rsvd_philox_words(rsvd_handle_t handle, int n_groups, int l, uint64_t seed, uint32_t stream_id, int col0,
                              uint32_t* out, rsvd_stream_t stream) {
  if (!handle) return RSVD_E_INVALID;
  if (n_groups < 0 || l < 0 || col0 < 0) return fail(handle, RSVD_E_INVALID, "negative size");
  if ((long long)n_groups * l > 0 && !out) return fail(handle, RSVD_E_INVALID, "NULL output");
  launch_philox_words(n_groups, l, seed, stream_id, col0, out, (cudaStream_t)stream);
  return check_launch(handle, "rsvd_philox_words");
}

rsvd_status rsvd_gaussian(rsvd_handle_t handle, int n, int l, uint64_t seed, uint32_t stream_id, int col0, int dtype,
                          void* out, int ldo, rsvd_stream_t stream) {
  if (!handle) return RSVD_E_INVALID;
  if (n < 0 || l < 0 || col0 < 0) return fail(handle, RSVD_E_INVALID, "negative size");
  if (dtype != RSVD_DT_F64 && dtype != RSVD_DT_F32 && dtype != RSVD_DT_BF16)
    return fail(handle, RSVD_E_INVALID, "unknown dtype %d", dtype);
  if (ldo < l) return fail(handle, RSVD_E_INVALID, "ldo %d < l %d", ldo, l);
  if ((long long)n * l > 0 && !out) return fail(handle, RSVD_E_INVALID, "NULL output");
  launch_gaussian(n, l, seed, stream_id, col0, dtype, out, ldo, (cudaStream_t)stream);
  return check_launch(handle, "rsvd_gaussian");
}

rsvd_status rsvd_sketch_workspace_size(rsvd_handle_t handle, int prec, int trans, int m, int n, int l, size_t* bytes) {
  if (!handle || !bytes || m < 0 || n < 0 || l < 0) return RSVD_E_INVALID;
  const int M = trans ? n : m, K = trans ? m : n;
  if (prec == RSVD_F64 || prec == RSVD_F32)
    *bytes = simt_gemm_workspace(M, l, K, handle->sms, elem_size(prec)) + 512;
  else if (prec == RSVD_MIXED_BF16)
    *bytes = tc_gemm_workspace(M, l, K, handle->sms) + 512;
  else if (is_fp8(prec))
    *bytes = sketch_fp8_layout(nullptr, trans, m, n, l, handle->sms).bytes;
  else
    return fail(handle, RSVD_E_UNSUPPORTED, "precision %d is not built yet", prec);
  return RSVD_OK;
}

rsvd_status rsvd_sketch(rsvd_handle_t handle, int prec, int trans, int m, int n, int l, const void* A, int lda,
                        const void* X, int ldx, void* Y, int ldy, void* workspace, size_t ws_bytes,
                        rsvd_stream_t stream) {
  if (!handle) return RSVD_E_INVALID;
  if (m < 0 || n < 0 || l < 0) return fail(handle, RSVD_E_INVALID, "negative size");
  const int M = trans ? n : m, K = trans ? m : n;
  if (lda < n || ldx < l || ldy < l) return fail(handle, RSVD_E_INVALID, "leading dimension too small");
  if ((long long)M * l == 0) return RSVD_OK;
  if (!A || !X || !Y) return fail(handle, RSVD_E_INVALID, "NULL matrix pointer");
  size_t need = 0;
  rsvd_status st = rsvd_sketch_workspace_size(handle, prec, trans, m, n, l, &need);
  if (st != RSVD_OK) return st;
  if (need > 512 && (!workspace || ws_bytes < need))
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  if (is_fp8(prec)) {
    if (l > 256) return fail(handle, RSVD_E_UNSUPPORTED, "l = %d > 256", l);
    const SketchFp8 F = sketch_fp8_layout(workspace, trans, m, n, l, handle->sms);
    cudaMemsetAsync(F.st, 0, sizeof(DevStatus), s);
    if (prec == RSVD_MIXED_FP8_B128) launch_fp8_block_max(m, n, (const float*)A, lda, 128, F.amax, s);
    launch_fp8_rows(m, n, (const float*)A, lda, F.A8, round16(n), F.s, nullptr, nullptr, 0, handle->sms, s,
                    prec == RSVD_MIXED_FP8_B128 ? F.amax : nullptr);
    cudaError_t e;
    if (!trans) {
      launch_fp8_cols(n, l, (const float*)X, ldx, nullptr, F.X8t, round16(n), F.c, F.colws, s);
      e = launch_tc_gemm_e4m3(m, l, n, F.A8, round16(n), F.X8t, round16(n), F.s, F.c, (float*)Y, ldy, F.part,
                              handle->sms, F.st, s);
    } else {
      launch_u8_transpose(m, n, F.A8, round16(n), F.A8T, round16(m), s);
      launch_fp8_cols(m, l, (const float*)X, ldx, F.s, F.X8t, round16(m), F.c, F.colws, s);
      e = launch_tc_gemm_e4m3(n, l, m, F.A8T, round16(m), F.X8t, round16(m), nullptr, F.c, (float*)Y, ldy, F.part,
                              handle->sms, F.st, s);
    }
    if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_sketch (e4m3): %s", cudaGetErrorString(e));
    return check_launch(handle, "rsvd_sketch (e4m3)");
  }
  if (prec == RSVD_MIXED_BF16) {
    if (l > 256) return fail(handle, RSVD_E_UNSUPPORTED, "l = %d > 256", l);
    if ((lda % 8) || (ldx % 8) || (((uintptr_t)A | (uintptr_t)X) & 15))
      return fail(handle, RSVD_E_INVALID, "bf16 operands need 16-byte aligned rows (lda, ldx multiples of 8)");
    Carver c(workspace);
    DevStatus* dst = c.take<DevStatus>(1);
    float* part = c.take<float>(tc_gemm_workspace(M, l, K, handle->sms) / sizeof(float) + 1);
    cudaMemsetAsync(dst, 0, sizeof(DevStatus), s);
    cudaError_t e = launch_tc_gemm(trans != 0, false, M, l, K, (const __nv_bfloat16*)A, lda, nullptr,
                                   (const __nv_bfloat16*)X, ldx, nullptr, (float*)Y, ldy, part, handle->sms, dst, s);
    if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_sketch: %s", cudaGetErrorString(e));
    return check_launch(handle, "rsvd_sketch");
  }
  if (prec == RSVD_F64)
    launch_gemm_simt<double>(trans != 0, M, l, K, (const double*)A, lda, (const double*)X, ldx, (double*)Y, ldy,
                             (double*)workspace, handle->sms, s);
  else
    launch_gemm_simt<float>(trans != 0, M, l, K, (const float*)A, lda, (const float*)X, ldx, (float*)Y, ldy,
                            (float*)workspace, handle->sms, s);
  return check_launch(handle, "rsvd_sketch");
}

rsvd_status rsvd_project_workspace_size(rsvd_handle_t handle, int prec, int m, int n, int l, size_t* bytes) {
  if (!handle || !bytes || m < 0 || n < 0 || l < 0) return RSVD_E_INVALID;
  Carver c(nullptr);
  c.take<DevStatus>(1);
  if (prec == RSVD_MIXED_BF16) {
    c.take<__nv_bfloat16>((size_t)2 * m * round8(n));
    c.take<__nv_bfloat16>((size_t)2 * m * round8(l));
    c.take<unsigned char>(tc_gemm_workspace(n, l, m, handle->sms));
  } else if (prec == RSVD_F64 || prec == RSVD_F32) {
    c.take<unsigned char>(simt_gemm_workspace(n, l, m, handle->sms, elem_size(prec)));
  } else {
    return fail(handle, RSVD_E_UNSUPPORTED, "precision %d", prec);
  }
  *bytes = c.size();
  return RSVD_OK;
}

rsvd_status rsvd_project(rsvd_handle_t handle, int prec, int m, int n, int l, const void* A, int lda, const void* Q,
                         int ldq, void* Bt, int ldb, void* workspace, size_t ws_bytes, rsvd_stream_t stream) {
  if (!handle) return RSVD_E_INVALID;
  if (m < 0 || n < 0 || l < 0) return fail(handle, RSVD_E_INVALID, "negative size");
  if (lda < n || ldq < l || ldb < l) return fail(handle, RSVD_E_INVALID, "leading dimension too small");
  if ((long long)n * l == 0) return RSVD_OK;
  if (!A || !Q || !Bt) return fail(handle, RSVD_E_INVALID, "NULL matrix pointer");
  size_t need = 0;
  rsvd_status st = rsvd_project_workspace_size(handle, prec, m, n, l, &need);
  if (st != RSVD_OK) return st;
  if (!workspace || ws_bytes < need) return fail(handle, RSVD_E_NOMEM, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  Carver c(workspace);
  DevStatus* dst = c.take<DevStatus>(1);
  cudaMemsetAsync(dst, 0, sizeof(DevStatus), s);
  if (prec == RSVD_MIXED_BF16) {
    if (l > 256) return fail(handle, RSVD_E_UNSUPPORTED, "l = %d > 256", l);
    const int n8 = round8(n), l8 = round8(l);
    __nv_bfloat16* Ah = c.take<__nv_bfloat16>((size_t)m * n8);
    __nv_bfloat16* Al = c.take<__nv_bfloat16>((size_t)m * n8);
    __nv_bfloat16* Qh = c.take<__nv_bfloat16>((size_t)m * l8);
    __nv_bfloat16* Ql = c.take<__nv_bfloat16>((size_t)m * l8);
    float* part = c.take<float>(tc_gemm_workspace(n, l, m, handle->sms) / sizeof(float) + 1);
    launch_split_bf16(m, n, (const float*)A, lda, Ah, Al, n8, handle->sms, s);
    launch_split_bf16(m, l, (const float*)Q, ldq, Qh, Ql, l8, handle->sms, s);
    cudaError_t e = launch_tc_gemm(true, true, n, l, m, Ah, n8, Al, Qh, l8, Ql, (float*)Bt, ldb, part, handle->sms,
                                   dst, s);
    if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_project: %s", cudaGetErrorString(e));
  } else if (prec == RSVD_F64) {
    launch_gemm_simt<double>(true, n, l, m, (const double*)A, lda, (const double*)Q, ldq, (double*)Bt, ldb,
                             c.take<double>(simt_gemm_workspace(n, l, m, handle->sms, 8) / 8 + 1), handle->sms, s);
  } else {
    launch_gemm_simt<float>(true, n, l, m, (const float*)A, lda, (const float*)Q, ldq, (float*)Bt, ldb,
                            c.take<float>(simt_gemm_workspace(n, l, m, handle->sms, 4) / 4 + 1), handle->sms, s);
  }
  return check_launch(handle, "rsvd_project");
}

rsvd_status rsvd_orth_workspace_size(rsvd_handle_t handle, int prec, int rows, int l, size_t* bytes) {
  if (!handle || !bytes || rows < 0 || l < 0) return RSVD_E_INVALID;
  if (prec != RSVD_F64 && prec != RSVD_F32) return fail(handle, RSVD_E_UNSUPPORTED, "precision %d", prec);
  Carver c(nullptr);
  c.take<DevStatus>(1);
  c.take<unsigned char>(orth_workspace_bytes(rows, l, handle->sms, elem_size(prec)));
  *bytes = c.size();
  return RSVD_OK;
}

rsvd_status rsvd_orth(rsvd_handle_t handle, int prec, int rows, int l, void* Y, int ldy, double* R, void* workspace,
                      size_t ws_bytes, rsvd_stream_t stream) {
  if (!handle) return RSVD_E_INVALID;
  if (rows < 0 || l < 0) return fail(handle, RSVD_E_INVALID, "negative size");
  if (l == 0) return RSVD_OK;
  if (l > rows) return fail(handle, RSVD_E_INVALID, "l = %d exceeds rows = %d", l, rows);
  if (l > max_l_for(prec)) return fail(handle, RSVD_E_UNSUPPORTED, "l = %d too large", l);
  if (ldy < l) return fail(handle, RSVD_E_INVALID, "ldy %d < l %d", ldy, l);
  if (!Y) return fail(handle, RSVD_E_INVALID, "NULL Y");
  size_t need = 0;
  rsvd_status st = rsvd_orth_workspace_size(handle, prec, rows, l, &need);
  if (st != RSVD_OK) return st;
  if (!workspace || ws_bytes < need) return fail(handle, RSVD_E_NOMEM, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  Carver c(workspace);
  DevStatus* dst = c.take<DevStatus>(1);
  void* ows = c.take<unsigned char>(orth_workspace_bytes(rows, l, handle->sms, elem_size(prec)));
  cudaMemsetAsync(dst, 0, sizeof(DevStatus), s);
  if (prec == RSVD_F64)
    run_orth<double, double>(rows, l, (double*)Y, ldy, R, nullptr, 0, ows, dst, handle->sms, s);
  else
    run_orth<float, float>(rows, l, (float*)Y, ldy, R, nullptr, 0, ows, dst, handle->sms, s);
  return check_launch(handle, "rsvd_orth");
}

rsvd_status rsvd_probe_workspace_size(rsvd_handle_t handle, int m, int n, size_t* bytes) {
  if (!handle || !bytes) return RSVD_E_INVALID;
  if (m < 16 || n < 16) return fail(handle, RSVD_E_INVALID, "the probe needs m, n >= 16");
  *bytes = ctrl_layout(nullptr, m, n, 16, handle->sms, 0).bytes;
  return RSVD_OK;
}

rsvd_status rsvd_probe_features(rsvd_handle_t handle, int m, int n, const float* A, int lda, uint64_t seed,
                                float* feat, double* fro2, void* workspace, size_t ws_bytes, rsvd_stream_t stream) {
  size_t need = 0;
  rsvd_status st = rsvd_probe_workspace_size(handle, m, n, &need);
  if (st != RSVD_OK) return st;
  if (lda < n) return fail(handle, RSVD_E_INVALID, "lda %d < n %d", lda, n);
  if (!A || !feat) return fail(handle, RSVD_E_INVALID, "NULL pointer");
  if (!workspace || ws_bytes < need)
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const CtrlLayout L = ctrl_layout(workspace, m, n, 16, handle->sms, 0);
  cudaMemsetAsync(L.blk, 0, sizeof(RsvdCtrlBlock), s);
  run_probe(handle, m, n, A, lda, seed, L, s);
  cudaMemcpyAsync(feat, L.blk->feat, RSVD_CTRL_D_IN * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (fro2) cudaMemcpyAsync(fro2, &L.blk->fro2, sizeof(double), cudaMemcpyDeviceToDevice, s);
  return check_launch(handle, "rsvd_probe_features");
}

rsvd_status rsvd_mlp_workspace_size(rsvd_handle_t handle, int batch, size_t* bytes) {
  if (!handle || !bytes || batch < 0) return RSVD_E_INVALID;
  *bytes = mlp_workspace_bytes(batch > 0 ? batch : 1);
  return RSVD_OK;
}

rsvd_status rsvd_mlp_forward(rsvd_handle_t handle, int batch, const float* X, const float* theta, float* logits,
                             rsvd_stream_t stream) {
  if (!handle) return RSVD_E_INVALID;
  if (batch < 0) return fail(handle, RSVD_E_INVALID, "negative batch");
  if (batch == 0) return RSVD_OK;
  if (!X || !theta || !logits) return fail(handle, RSVD_E_INVALID, "NULL pointer");
  cudaError_t e = launch_mlp(-1, batch, X, nullptr, nullptr, 0.f, theta, logits, nullptr, nullptr, nullptr, 0, 0.f,
                             nullptr, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_mlp_forward: %s", cudaGetErrorString(e));
  return RSVD_OK;
}

namespace {
rsvd_status mlp_common(rsvd_handle_t h, int batch, const float* X, const int* yl, const int* yq, float lam,
                       const void* theta, void* ws, size_t ws_bytes) {
  if (!h) return RSVD_E_INVALID;
  if (batch < 1) return fail(h, RSVD_E_INVALID, "batch must be >= 1");
  if (!X || !yl || !yq || !theta) return fail(h, RSVD_E_INVALID, "NULL pointer");
  if (!(lam >= 0.f)) return fail(h, RSVD_E_INVALID, "lam must be >= 0");
  const size_t need = mlp_workspace_bytes(batch);
  if (!ws || ws_bytes < need) return fail(h, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  if (((uintptr_t)ws & 255) != 0) return fail(h, RSVD_E_INVALID, "workspace not 256-byte aligned");
  return RSVD_OK;
}
}  // namespace

rsvd_status rsvd_mlp_grad(rsvd_handle_t handle, int batch, const float* X, const int* yl, const int* yq, float lam,
                          const float* theta, float* grad, double* loss, void* workspace, size_t ws_bytes,
                          rsvd_stream_t stream) {
  rsvd_status st = mlp_common(handle, batch, X, yl, yq, lam, theta, workspace, ws_bytes);
  if (st != RSVD_OK) return st;
  if (!grad) return fail(handle, RSVD_E_INVALID, "NULL grad");
  cudaError_t e = launch_mlp(0, batch, X, yl, yq, lam, theta, nullptr, grad, nullptr, nullptr, 0, 0.f, loss,
                             workspace, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_mlp_grad: %s", cudaGetErrorString(e));
  return RSVD_OK;
}

rsvd_status rsvd_mlp_train_step(rsvd_handle_t handle, int batch, const float* X, const int* yl, const int* yq,
                                float lam, float* theta, float* m1, float* m2, int step, float lr, double* loss,
                                void* workspace, size_t ws_bytes, rsvd_stream_t stream) {
  rsvd_status st = mlp_common(handle, batch, X, yl, yq, lam, theta, workspace, ws_bytes);
  if (st != RSVD_OK) return st;
  if (!m1 || !m2) return fail(handle, RSVD_E_INVALID, "NULL Adam moments");
  if (step < 1) return fail(handle, RSVD_E_INVALID, "step must be >= 1");
  if (!(lr > 0.f)) return fail(handle, RSVD_E_INVALID, "lr must be > 0");
  cudaError_t e = launch_mlp(1, batch, X, yl, yq, lam, theta, nullptr, nullptr, m1, m2, step, lr, loss, workspace,
                             (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "rsvd_mlp_train_step: %s", cudaGetErrorString(e));
  return RSVD_OK;
}

rsvd_status rsvd_controller_attach(rsvd_handle_t handle, const float* theta, double quantile, double safety) {
  if (!handle) return RSVD_E_INVALID;
  if (!(quantile > 0.0 && quantile <= 1.0)) return fail(handle, RSVD_E_INVALID, "quantile must lie in (0, 1]");
  if (!(safety > 0.0 && safety <= 1.0)) return fail(handle, RSVD_E_INVALID, "safety must lie in (0, 1]");
  handle->ctrl_theta = theta;
  handle->ctrl_quantile = quantile;
  handle->ctrl_safety = safety;
  return RSVD_OK;
}

rsvd_status rsvd_controller_fallback(rsvd_handle_t handle, int mode) {
  if (!handle) return RSVD_E_INVALID;
  if (mode != 0 && mode != 1) return fail(handle, RSVD_E_INVALID, "fallback mode must be 0 or 1");
  handle->ctrl_fallback = mode;
  return RSVD_OK;
}

rsvd_status rsvd_controller_last(rsvd_handle_t handle, int* info, double* est) {
  if (!handle || !info || !est) return RSVD_E_INVALID;
  for (int i = 0; i < 5; ++i) info[i] = handle->ctrl_info[i];
  est[0] = handle->ctrl_est[0];
  est[1] = handle->ctrl_est[1];
  return RSVD_OK;
}

rsvd_status rsvd_certify_workspace_size(rsvd_handle_t handle, int m, int n, int r, size_t* bytes) {
  if (!handle || !bytes) return RSVD_E_INVALID;
  if (m < 1 || n < 1 || r < 0 || r > 1024) return fail(handle, RSVD_E_INVALID, "need m, n >= 1 and 0 <= r <= 1024");
  *bytes = ctrl_layout(nullptr, m, n, r > 0 ? r : 1, handle->sms, 0).bytes;
  return RSVD_OK;
}

rsvd_status rsvd_certify(rsvd_handle_t handle, int m, int n, const float* A, int lda, int r, const float* U, int ldu,
                         const double* D, const float* V, int ldv, uint64_t seed, double* out, void* workspace,
                         size_t ws_bytes, rsvd_stream_t stream) {
  size_t need = 0;
  rsvd_status st = rsvd_certify_workspace_size(handle, m, n, r, &need);
  if (st != RSVD_OK) return st;
  if (!A || !out || (r > 0 && (!U || !D || !V))) return fail(handle, RSVD_E_INVALID, "NULL argument");
  if (lda < n || (r > 0 && (ldu < r || ldv < r))) return fail(handle, RSVD_E_INVALID, "leading dimension too small");
  if (!workspace || ws_bytes < need)
    return fail(handle, RSVD_E_NOMEM, "workspace of %zu bytes < required %zu", ws_bytes, need);
  if (((uintptr_t)workspace & 255) != 0) return fail(handle, RSVD_E_INVALID, "workspace not 256-byte aligned");
  if (!device_accessible(handle, A) || (r > 0 && (!device_accessible(handle, U) || !device_accessible(handle, D) ||
                                                  !device_accessible(handle, V))))
    return fail(handle, RSVD_E_INVALID, "an input is not memory the device can access (pin host buffers)");
  cudaStream_t s = (cudaStream_t)stream;
  const int sms = handle->sms;
  const CtrlLayout L = ctrl_layout(workspace, m, n, r > 0 ? r : 1, sms, 0);
  cudaMemsetAsync(L.blk, 0, sizeof(RsvdCtrlBlock), s);
  // E = A G - U (D (V^T G)), G = 16 columns of Philox stream 2
  launch_gaussian(n, CTRL_NC, seed, 2u, 0, RSVD_DT_F32, L.G, CTRL_NC, s);
  const int nfro = launch_thin_sketch(m, n, A, lda, L.G, L.Yp, L.Y, L.fro2p, sms, s);
  launch_fro2_reduce(nfro, L.fro2p, L.blk, s);
  if (r > 0) launch_gemm_simt<float>(true, r, CTRL_NC, n, V, ldv, L.G, CTRL_NC, L.T, CTRL_NC, L.Tpart, sms, s);
  launch_judge(m, r, L.Y, U, ldu, D, L.T, L.rpart, 0.0, 1.0, L.blk, sms, s);
  st = check_launch(handle, "rsvd_certify");
  if (st != RSVD_OK) return st;
  RsvdCtrlBlock hb;
  cudaError_t e = cudaMemcpyAsync(&hb, L.blk, sizeof(hb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(handle, RSVD_E_CUDA, "certificate read: %s", cudaGetErrorString(e));
  out[0] = sqrt(hb.est2 > 0.0 ? hb.est2 : 0.0);
  out[1] = hb.spec_bound;
  out[2] = sqrt(hb.fro2 > 0.0 ? hb.fro2 : 0.0);
  if (!isfinite(out[0]) || !isfinite(out[2])) return fail(handle, RSVD_E_NONFINITE, "non-finite certificate");
  return RSVD_OK;
}

}  // extern "C"
