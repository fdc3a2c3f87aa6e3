// Implicit column centring (RSVD_FLAG_CENTER).  The paper names PCA among the
// applications of the randomized SVD (Sec. 1); PCA factors the column-centred
// matrix Abar = A - 1 mu^T, mu = A^T 1 / m, the vector of column means.
// Instead of forming Abar (a pass over A and a copy of it), every product of
// Fig. RSVDP_stabilized carries its rank-one correction:
//   Abar X   = A X   - 1 (mu^T X)       forward products A G, A W
//   Abar^T Y = A^T Y - mu (1^T Y)       transposed products A^T Q and B^T = A^T Q
// Both are applied as the definition states.  (In exact arithmetic every Q
// the solve forms is orthogonal to 1, so the transposed correction vanishes;
// in floating point it removes what rounding leaves along 1.)
//
// Sums run in binary64 across row chunks; within a chunk of CS rows the
// binary32 paths accumulate in binary32 (binary64 adds run at 1/64 of the
// binary32 rate on this part), the binary64 path in binary64.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

namespace {

constexpr int CS = 128;     // rows per binary32 chunk
constexpr int CT = 128;     // threads (= columns) per CTA

template <typename X>
struct Acc {
  using T = float;
};
template <>
struct Acc<double> {
  using T = double;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// part[slice][j] = sum over the slice's rows i of w_i M(i, j) (w == null: 1).
template <typename X>
__global__ void __launch_bounds__(CT) wcolsum_partial_kernel(int rows, int cols, const double* __restrict__ w,
                                                             const X* __restrict__ M, long long ld, int rows_per,
                                                             double* __restrict__ part) {
  using A = typename Acc<X>::T;
  const int j = blockIdx.x * CT + threadIdx.x;
  const int r0 = blockIdx.y * rows_per, r1 = min(rows, r0 + rows_per);
  if (j >= cols) return;
  double s64 = 0.0;
  for (int c0 = r0; c0 < r1; c0 += CS) {
    const int c1 = min(r1, c0 + CS);
    A s = A(0);
    // unrolled so that eight independent loads are in flight per thread
    if (w) {
#pragma unroll 8
      for (int i = c0; i < c1; ++i) s = fma((A)w[i], (A)to_f(M[(size_t)i * ld + j]), s);
    } else {
#pragma unroll 8
      for (int i = c0; i < c1; ++i) s += (A)to_f(M[(size_t)i * ld + j]);
    }
    s64 += (double)s;
  }
  part[(size_t)blockIdx.y * cols + j] = s64;
}

// out[j] = scale * sum over slices of part (fixed order).
__global__ void wcolsum_reduce_kernel(int cols, int slices, const double* __restrict__ part, double scale,
                                      double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  double s = 0.0;
  for (int z = 0; z < slices; ++z) s += part[(size_t)z * cols + j];
  out[j] = s * scale;
}

// Y(i, j) -= u_i v_j (u == null: 1).
template <typename T>
__global__ void rank1_sub_kernel(int rows, int cols, T* __restrict__ Y, int ldy, const double* __restrict__ u,
                                 const double* __restrict__ v) {
  const long long total = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    const double ui = u ? u[i] : 1.0;
    T* p = Y + (size_t)i * ldy + j;
    *p = (T)((double)*p - ui * v[j]);
  }
}

int slices_for(int rows, int cols, int sms) {
  const int cblocks = ceil_div(cols, CT);
  int sl = ceil_div(sms * 8, cblocks);
  const int maxsl = ceil_div(rows, 4 * CS);  // at least four chunks per slice
  if (sl > maxsl) sl = maxsl;
  if (sl < 1) sl = 1;
  if (sl > 1024) sl = 1024;
  return sl;
}

template <typename X>
void wcolsum(int rows, int cols, const double* w, const X* M, long long ld, double scale, double* part, double* out,
             int sms, cudaStream_t s) {
  const int sl = slices_for(rows, cols, sms);
  const int rows_per = ceil_div(ceil_div(rows, sl), CS) * CS;
  const int slices = ceil_div(rows, rows_per);
  wcolsum_partial_kernel<X><<<dim3(ceil_div(cols, CT), slices), CT, 0, s>>>(rows, cols, w, M, ld, rows_per, part);
  note_launch();
  wcolsum_reduce_kernel<<<ceil_div(cols, 256), 256, 0, s>>>(cols, slices, part, scale, out);
  note_launch();
}

template <typename T>
void rank1_sub(int rows, int cols, T* Y, int ldy, const double* u, const double* v, int sms, cudaStream_t s) {
  const long long total = (long long)rows * cols;
  if (total == 0) return;
  long long want = ceil_div(total, 4LL * 256);
  const int blocks = (int)(want < sms * 8 ? want : sms * 8);
  rank1_sub_kernel<T><<<blocks, 256, 0, s>>>(rows, cols, Y, ldy, u, v);
  note_launch();
}

}  // namespace

size_t centre_workspace_bytes(int m, int n, int l, int sms) {
  Carver c(nullptr);
  c.take<double>((size_t)n);      // mu
  c.take<double>((size_t)l);      // c or s
  const int big = m > n ? m : n;
  const int cols = n > l ? n : l;
  c.take<double>((size_t)slices_for(big, cols, sms) * cols + 64);  // partials
  return c.size();
}

CentreBufs centre_carve(void* ws, int m, int n, int l, int sms) {
  Carver c(ws);
  CentreBufs B;
  B.mu = c.take<double>((size_t)n);
  B.vec = c.take<double>((size_t)l);
  const int big = m > n ? m : n;
  const int cols = n > l ? n : l;
  B.part = c.take<double>((size_t)slices_for(big, cols, sms) * cols + 64);
  return B;
}

template <typename T>
void centre_means(int m, int n, const T* A, int lda, const CentreBufs& B, int sms, cudaStream_t s) {
  wcolsum<T>(m, n, nullptr, A, lda, 1.0 / (double)m, B.part, B.mu, sms, s);
}

template <typename T, typename X>
void centre_forward(int m, int n, int l, const X* Xop, int ldx, T* Y, int ldy, const CentreBufs& B, int sms,
                    cudaStream_t s) {
  wcolsum<X>(n, l, B.mu, Xop, ldx, 1.0, B.part, B.vec, sms, s);  // c = mu^T X
  rank1_sub<T>(m, l, Y, ldy, nullptr, B.vec, sms, s);             // Y -= 1 c^T
}

template <typename T, typename Q>
void centre_adjoint(int m, int n, int l, const Q* Qm, int ldq, T* Z, int ldz, const CentreBufs& B, int sms,
                    cudaStream_t s) {
  wcolsum<Q>(m, l, nullptr, Qm, ldq, 1.0, B.part, B.vec, sms, s);  // s = 1^T Q
  rank1_sub<T>(n, l, Z, ldz, B.mu, B.vec, sms, s);                  // Z -= mu s^T
}

template void centre_means<float>(int, int, const float*, int, const CentreBufs&, int, cudaStream_t);
template void centre_means<double>(int, int, const double*, int, const CentreBufs&, int, cudaStream_t);
template void centre_forward<float, float>(int, int, int, const float*, int, float*, int, const CentreBufs&, int,
                                           cudaStream_t);
template void centre_forward<double, double>(int, int, int, const double*, int, double*, int, const CentreBufs&, int,
                                             cudaStream_t);
template void centre_forward<float, __nv_bfloat16>(int, int, int, const __nv_bfloat16*, int, float*, int,
                                                   const CentreBufs&, int, cudaStream_t);
template void centre_adjoint<float, float>(int, int, int, const float*, int, float*, int, const CentreBufs&, int,
                                           cudaStream_t);
template void centre_adjoint<double, double>(int, int, int, const double*, int, double*, int, const CentreBufs&, int,
                                             cudaStream_t);
template void centre_adjoint<float, __nv_bfloat16>(int, int, int, const __nv_bfloat16*, int, float*, int,
                                                   const CentreBufs&, int, cudaStream_t);

}  // namespace rsvd
