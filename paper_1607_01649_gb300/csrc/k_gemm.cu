// SIMT sketch products for the binary64 and plain-binary32 paths
// (Fig. RSVDP_stabilized: the products A G, A^T Q, A W and Q^T A).
//
//   NN:  Y[M x N] = A[M x K] X[K x N]        A row-major (lda)
//   TN:  Y[M x N] = A^T[M x K] X[K x N]      A is K x M row-major (lda)
//
// CTA tile 128 x 64, k-step 16, 256 threads, 8 x 4 outputs per thread.
// Long K is split over gridDim.z; each split writes its partial tile to the
// workspace and a second kernel adds the splits in a fixed order, so results
// are bitwise reproducible.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

constexpr int GBM = 128, GBN = 64, GBK = 16;

template <typename T, bool TRANS>
__global__ void __launch_bounds__(256)
    gemm_simt_kernel(int M, int N, int K, const T* __restrict__ A, int lda, const T* __restrict__ X,
                     int ldx, T* __restrict__ Y, int ldy, int kchunk, long long split_stride) {
  __shared__ T As[GBK][GBM + 4];
  __shared__ T Xs[GBK][GBN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);

  T acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + 256 * t;
      int r, kk;
      if (!TRANS) {
        kk = e % GBK;
        r = e / GBK;
      } else {
        r = e % GBM;
        kk = e / GBM;
      }
      const int gr = m0 + r, gk = k0 + kk;
      T v = T(0);
      if (gr < M && gk < kend) v = TRANS ? A[(size_t)gk * lda + gr] : A[(size_t)gr * lda + gk];
      As[kk][r] = v;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t;
      const int c = e % GBN, kk = e / GBN;
      const int gc = n0 + c, gk = k0 + kk;
      Xs[kk][c] = (gc < N && gk < kend) ? X[(size_t)gk * ldx + gc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      T a[8], x[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    __syncthreads();
  }

  T* out = Y;
  int ldo = ldy;
  if (split_stride > 0) {
    out = Y + (size_t)blockIdx.z * split_stride;
    ldo = N;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx + 16 * j;
      if (c < N) out[(size_t)r * ldo + c] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void splitk_reduce_kernel(int M, int N, int splits, const T* __restrict__ P,
                                     long long split_stride, T* __restrict__ Y, int ldy) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int r = (int)(idx / N), c = (int)(idx % N);
  T s = T(0);
  for (int z = 0; z < splits; ++z) s += P[(size_t)z * split_stride + idx];
  Y[(size_t)r * ldy + c] = s;
}

// Choose the number of K-splits so that the grid covers the GPU about twice.
int simt_splits(int M, int N, int K, int sms) {
  const long long tiles = (long long)ceil_div(M, GBM) * ceil_div(N, GBN);
  long long s = (2LL * sms + tiles - 1) / tiles;
  const long long kmax = ceil_div(K, 4 * GBK);  // keep >= 64 k per split
  if (s > kmax) s = kmax;
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  return (int)s;
}

size_t simt_gemm_workspace(int M, int N, int K, int sms, size_t elem) {
  const int s = simt_splits(M, N, K, sms);
  return s > 1 ? (size_t)s * M * N * elem : 0;
}

template <typename T>
void launch_gemm_simt(bool trans, int M, int N, int K, const T* A, int lda, const T* X, int ldx, T* Y,
                      int ldy, T* partial, int sms, cudaStream_t s) {
  if (M == 0 || N == 0) return;
  int splits = simt_splits(M, N, K, sms);
  if (partial == nullptr) splits = 1;
  int kchunk = ceil_div(ceil_div(K, splits), GBK) * GBK;
  splits = ceil_div(K, kchunk);
  if (splits < 1) splits = 1;
  dim3 grid(ceil_div(M, GBM), ceil_div(N, GBN), splits);
  const long long stride = splits > 1 ? (long long)M * N : 0;
  T* out = splits > 1 ? partial : Y;
  if (trans)
    gemm_simt_kernel<T, true><<<grid, 256, 0, s>>>(M, N, K, A, lda, X, ldx, out, ldy, kchunk, stride);
  else
    gemm_simt_kernel<T, false><<<grid, 256, 0, s>>>(M, N, K, A, lda, X, ldx, out, ldy, kchunk, stride);
  note_launch();
  if (splits > 1) {
    const long long total = (long long)M * N;
    splitk_reduce_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(M, N, splits, partial, stride,
                                                                           Y, ldy);
    note_launch();
  }
}

template void launch_gemm_simt<float>(bool, int, int, int, const float*, int, const float*, int, float*,
                                      int, float*, int, cudaStream_t);
template void launch_gemm_simt<double>(bool, int, int, int, const double*, int, const double*, int,
                                       double*, int, double*, int, cudaStream_t);

}  // namespace rsvd
