// Fig. RSVD with the subsampled randomized Fourier transform as the test
// matrix (Sec. "A method with complexity O(mn log k)", eq. SRFT):
//   Omega = D F S (n x l, complex): D = diag(e^{i theta_j}), F the unitary DFT,
//   S = l distinct columns of the identity;
//   Y = A Omega,  Q = orth(Y),  B = Q^* A,  B = Uhat Sigma V^*,  U = Q Uhat.
// For a real A the factors Y, Q, B, U, V are complex; D is real.
//
// On this part the sketch is a bandwidth-bound pass over A whichever test
// matrix it uses, so Omega is formed explicitly (its real and imaginary parts
// as 2l real columns) and applied by the ordinary sketch product, bf16 tensor
// cores or binary32/64 SIMT; the FFT's saving in flops would not shorten the
// pass.  The complex steps run on the realification: a complex Y (m x l)
// spans the same real space as
//       Yhat = [ Yr  -Yi ]   (2m x 2l, real),
//              [ Yi   Yr ]
// so Qhat = orth(Yhat) is a real orthonormal basis of realify(span Y), and
// Bhat = Qhat^T diag(A, A) has the singular values of B = Q^* A, each twice,
// with singular vectors that are realifications [x_r; x_i] of complex ones.
// The real kernels (CholeskyQR, Jacobi) therefore give D and the complex U, V:
// every second value of the sorted Bhat spectrum, u = u_top + i u_bottom,
// v = v_top + i v_bottom, each pair phased so that the largest-magnitude entry
// of v_i is real and positive.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

namespace {

constexpr uint32_t STREAM_SRFT_D = 6u, STREAM_SRFT_S = 7u;

// 64-bit sort key of column j: (w0 << 32) | w1 of counter (j, 0, 7, 0)
__global__ void srft_key_kernel(int n, uint32_t k0, uint32_t k1, unsigned long long* __restrict__ key) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Philox4 r = philox4x32_10((uint32_t)j, 0u, STREAM_SRFT_S, 0u, k0, k1);
  key[j] = ((unsigned long long)r.x[0] << 32) | r.x[1];
}

// S: the l indices with the smallest keys (ties to the smaller index), in key
// order: rank_j = #{i : key_i < key_j, or key_i == key_j and i < j}.
__global__ void srft_subset_kernel(int n, int l, const unsigned long long* __restrict__ key, int* __restrict__ S) {
  __shared__ unsigned long long tile[1024];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long kj = j < n ? key[j] : 0ull;
  int rank = 0;
  for (int t0 = 0; t0 < n; t0 += 1024) {
    __syncthreads();
    for (int e = threadIdx.x; e < 1024 && t0 + e < n; e += blockDim.x) tile[e] = key[t0 + e];
    __syncthreads();
    const int tn = min(1024, n - t0);
    for (int e = 0; e < tn; ++e) {
      const unsigned long long ki = tile[e];
      rank += (ki < kj) || (ki == kj && t0 + e < j);
    }
  }
  if (j < n && rank < l) S[rank] = j;
}

// Om2 (n x 2l): columns 0..l-1 the real parts, l..2l-1 the imaginary parts of
// Omega(p, s) = e^{i theta_p} e^{-2 pi i p S_s / n} / sqrt(n); the phase
// fraction theta_p / (2 pi) - (p S_s mod n) / n is formed in binary64.
template <typename T>
__global__ void srft_omega_kernel(int n, int l, uint32_t k0, uint32_t k1, const int* __restrict__ S,
                                  T* __restrict__ Om, int ldo) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * l) return;
  const int p = idx / l, s = idx % l;
  const Philox4 r = philox4x32_10((uint32_t)(p >> 2), 0u, STREAM_SRFT_D, 0u, k0, k1);
  const double u = (double)(r.x[p & 3] >> 8) * 5.9604644775390625e-08;  // theta / (2 pi)
  const long long pq = ((long long)p * (long long)S[s]) % n;
  double f = u - (double)pq / (double)n;                                  // in (-1, 1)
  double sn, cs;
  sincospi(2.0 * f, &sn, &cs);
  const double sc = 1.0 / sqrt((double)n);
  Om[(size_t)p * ldo + s] = (T)(cs * sc);
  Om[(size_t)p * ldo + l + s] = (T)(sn * sc);
}

// Yhat (2m x 2l) from Y2 = [Yr | Yi] (m x 2l).
template <typename T>
__global__ void realify_kernel(int m, int l, const T* __restrict__ Y2, T* __restrict__ Yh) {
  const long long total = (long long)m * l;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / l), c = (int)(e % l);
    const T yr = Y2[(size_t)i * 2 * l + c], yi = Y2[(size_t)i * 2 * l + l + c];
    Yh[(size_t)i * 2 * l + c] = yr;
    Yh[(size_t)i * 2 * l + l + c] = -yi;
    Yh[((size_t)m + i) * 2 * l + c] = yi;
    Yh[((size_t)m + i) * 2 * l + l + c] = yr;
  }
}

// Every second column of the sorted 2l-wide factors: D[c] = Dall[2c],
// W2(:, c) = Wsel(:, 2c), J2(:, c) = Jsel(:, 2c)  (rows 2l, ld of sources 2l).
template <typename T>
__global__ void take_pairs_kernel(int l2, int kk, const double* __restrict__ Dall, const T* __restrict__ Wsel,
                                  const T* __restrict__ Jsel, double* __restrict__ D, T* __restrict__ W2,
                                  T* __restrict__ J2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < kk) D[idx] = Dall[2 * idx];
  if (idx >= l2 * kk) return;
  const int r = idx / kk, c = idx % kk;
  W2[idx] = Wsel[(size_t)r * l2 + 2 * c];
  J2[idx] = Jsel[(size_t)r * l2 + 2 * c];
}

// Complex outputs (interleaved re, im; ld in complex entries) from the
// realified vectors, phased so that the largest-magnitude entry of v_c (lowest
// index on ties) is real and positive.  One CTA per column.
template <typename T>
__global__ void srft_pack_kernel(int m, int n, int kk, const T* __restrict__ Uh, const T* __restrict__ Vh,
                                 T* __restrict__ U, int ldu, T* __restrict__ V, int ldv) {
  const int c = blockIdx.x;
  __shared__ double sm[256];
  __shared__ int si[256];
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double vr = (double)Vh[(size_t)j * kk + c], vi = (double)Vh[((size_t)n + j) * kk + c];
    const double a = vr * vr + vi * vi;
    if (a > best) {
      best = a;
      bi = j;
    }
  }
  sm[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double b2 = sm[threadIdx.x + o];
      const int i2 = si[threadIdx.x + o];
      if (b2 > sm[threadIdx.x] || (b2 == sm[threadIdx.x] && i2 < si[threadIdx.x])) {
        sm[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const int jp = si[0];
  const double pr = (double)Vh[(size_t)jp * kk + c], pi = (double)Vh[((size_t)n + jp) * kk + c];
  const double mag = sqrt(pr * pr + pi * pi);
  const double hr = mag > 0.0 ? pr / mag : 1.0, hi = mag > 0.0 ? -pi / mag : 0.0;  // conj(piv) / |piv|
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double vr = (double)Vh[(size_t)j * kk + c], vi = (double)Vh[((size_t)n + j) * kk + c];
    V[((size_t)j * ldv + c) * 2] = (T)(vr * hr - vi * hi);
    V[((size_t)j * ldv + c) * 2 + 1] = (T)(vr * hi + vi * hr);
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double ur = (double)Uh[(size_t)i * kk + c], ui = (double)Uh[((size_t)m + i) * kk + c];
    U[((size_t)i * ldu + c) * 2] = (T)(ur * hr - ui * hi);
    U[((size_t)i * ldu + c) * 2 + 1] = (T)(ur * hi + ui * hr);
  }
}

// Interleaved realification of kk complex columns held as Xh (2 rows x kk:
// real parts on top, imaginary parts below): Xi (2 rows x 2 kk) has column
// 2c = [x_r; x_i] and column 2c + 1 = [-x_i; x_r] (the realification of i x).
// In this column order the real Cholesky factor of Xi^T Xi is the
// realification of the complex Cholesky factor of X^H X, so a real
// CholeskyQR of Xi returns the realified complex QR.
template <typename T>
__global__ void pair_realify_kernel(int rows, int kk, const T* __restrict__ Xh, T* __restrict__ Xi) {
  const long long total = (long long)rows * kk;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / kk), c = (int)(e % kk);
    const T xr = Xh[(size_t)r * kk + c], xi = Xh[((size_t)rows + r) * kk + c];
    Xi[(size_t)r * 2 * kk + 2 * c] = xr;
    Xi[(size_t)r * 2 * kk + 2 * c + 1] = -xi;
    Xi[((size_t)rows + r) * 2 * kk + 2 * c] = xi;
    Xi[((size_t)rows + r) * 2 * kk + 2 * c + 1] = xr;
  }
}

// Xh(:, c) = Xi(:, 2c) (2 rows x kk)
template <typename T>
__global__ void take_even_kernel(int rows2, int kk, const T* __restrict__ Xi, T* __restrict__ Xh) {
  const long long total = (long long)rows2 * kk;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / kk), c = (int)(e % kk);
    Xh[(size_t)r * kk + c] = Xi[(size_t)r * 2 * kk + 2 * c];
  }
}

int grid_of(long long total) { return (int)((total + 255) / 256 > 0 ? (total + 255) / 256 : 1); }

}  // namespace

SrftLayout srft_layout(void* ws, int m, int n, int l, int kk, size_t es, int sms, bool mixed) {
  Carver c(ws);
  SrftLayout L;
  const int l2 = 2 * l;
  const int big = 2 * (m > n ? m : n);
  L.st = c.take<DevStatus>(1);
  L.key = c.take<unsigned long long>((size_t)n);
  L.S = c.take<int>((size_t)l);
  L.Om = c.take<unsigned char>((size_t)n * l2 * es);
  L.Y2 = c.take<unsigned char>((size_t)m * l2 * es);
  L.Yh = c.take<unsigned char>((size_t)2 * m * l2 * es);
  L.Z = c.take<unsigned char>((size_t)2 * n * l2 * es);
  L.orthws = c.take<unsigned char>(mixed ? orth_tc_workspace_bytes(big, l2, sms) : orth_workspace_bytes(big, l2, sms, es));
  L.Rb = c.take<double>((size_t)l2 * l2);
  L.Wt = c.take<unsigned char>((size_t)l2 * l2 * es);
  L.Jt = c.take<unsigned char>((size_t)l2 * l2 * es);
  L.sig = c.take<double>((size_t)l2);
  L.Dall = c.take<double>((size_t)l2);
  L.Wsel = c.take<unsigned char>((size_t)l2 * l2 * es);
  L.Jsel = c.take<unsigned char>((size_t)l2 * l2 * es);
  L.W2 = c.take<unsigned char>((size_t)l2 * kk * es);
  L.J2 = c.take<unsigned char>((size_t)l2 * kk * es);
  L.Uh = c.take<unsigned char>((size_t)2 * m * kk * es);
  L.Vh = c.take<unsigned char>((size_t)2 * n * kk * es);
  L.Xi = c.take<unsigned char>((size_t)big * 2 * kk * es);
  size_t pw = simt_gemm_workspace(m, l2, n, sms, es);
  if (simt_gemm_workspace(n, l2, m, sms, es) > pw) pw = simt_gemm_workspace(n, l2, m, sms, es);
  L.part = c.take<unsigned char>(pw + 256);
  if (mixed) {
    const int n8 = (n + 7) / 8 * 8, l28 = (l2 + 7) / 8 * 8;
    L.Ah = c.take<__nv_bfloat16>((size_t)m * n8);
    L.Al = c.take<__nv_bfloat16>((size_t)m * n8);
    L.Omb = c.take<__nv_bfloat16>((size_t)n * l28);
    L.Qh = c.take<__nv_bfloat16>((size_t)2 * m * l28);
    L.Ql = c.take<__nv_bfloat16>((size_t)2 * m * l28);
    size_t tw = tc_gemm_workspace(m, l2, n, sms);
    if (tc_gemm_workspace(n, l2, m, sms) > tw) tw = tc_gemm_workspace(n, l2, m, sms);
    L.tcpart = c.take<float>(tw / sizeof(float) + 1);
  } else {
    L.Ah = L.Al = L.Omb = L.Qh = L.Ql = nullptr;
    L.tcpart = nullptr;
  }
  L.bytes = c.size();
  return L;
}

template <typename T>
cudaError_t run_srft(int m, int n, const T* A, int lda, int k, int p, int kk, uint64_t seed, T* U, int ldu, double* D,
                     T* V, int ldv, const SrftLayout& L, int sms, bool mixed, cudaStream_t s) {
  const int l = k + p, l2 = 2 * l;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  T* Om = (T*)L.Om;
  T* Y2 = (T*)L.Y2;
  T* Yh = (T*)L.Yh;
  T* Z = (T*)L.Z;
  T* part = (T*)L.part;
  // Omega = D F S as 2l real columns
  srft_key_kernel<<<grid_of(n), 256, 0, s>>>(n, k0, k1, L.key);
  srft_subset_kernel<<<grid_of(n), 256, 0, s>>>(n, l, L.key, L.S);
  srft_omega_kernel<T><<<grid_of((long long)n * l), 256, 0, s>>>(n, l, k0, k1, L.S, Om, l2);
  note_launch();
  note_launch();
  note_launch();
  // Y = A Omega (m x 2l: real and imaginary parts), then its realification
  const bool tc = mixed && sizeof(T) == 4;
  const int n8 = (n + 7) / 8 * 8, l28 = (l2 + 7) / 8 * 8;
  if (tc) {
    launch_split_bf16(m, n, (const float*)A, lda, L.Ah, L.Al, n8, sms, s);
    launch_split_bf16(n, l2, (const float*)Om, l2, L.Omb, nullptr, l28, sms, s);
    cudaError_t e = launch_tc_gemm(false, false, m, l2, n, L.Ah, n8, nullptr, L.Omb, l28, nullptr, (float*)Y2, l2,
                                   L.tcpart, sms, L.st, s);
    if (e != cudaSuccess) return e;
  } else {
    launch_gemm_simt<T>(false, m, l2, n, A, lda, Om, l2, Y2, l2, part, sms, s);
  }
  realify_kernel<T><<<grid_of((long long)m * l), 256, 0, s>>>(m, l, Y2, Yh);
  note_launch();
  // Qhat = orth(Yhat) (2m x 2l); Bhat^T = [A^T Qhat_top; A^T Qhat_bottom] (2n x 2l)
  if (tc) {
    run_orth_tc(2 * m, l2, (float*)Yh, l2, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
    launch_split_bf16(2 * m, l2, (const float*)Yh, l2, L.Qh, L.Ql, l28, sms, s);
    for (int h = 0; h < 2; ++h) {
      cudaError_t e = launch_tc_gemm(true, true, n, l2, m, L.Ah, n8, L.Al, L.Qh + (size_t)h * m * l28, l28,
                                     L.Ql + (size_t)h * m * l28, (float*)Z + (size_t)h * n * l2, l2, L.tcpart, sms,
                                     L.st, s);
      if (e != cudaSuccess) return e;
    }
  } else {
    run_orth<T, T>(2 * m, l2, Yh, l2, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
    for (int h = 0; h < 2; ++h)
      launch_gemm_simt<T>(true, n, l2, m, A, lda, Yh + (size_t)h * m * l2, l2, Z + (size_t)h * n * l2, l2, part, sms,
                          s);
  }
  // SVD of Bhat: Bhat^T = Q_B R_B, Jacobi on R_B^T; the values come in pairs
  if (tc)
    run_orth_tc(2 * n, l2, (float*)Z, l2, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  else
    run_orth<T, T>(2 * n, l2, Z, l2, L.Rb, nullptr, 0, L.orthws, L.st, sms, s);
  cudaError_t e = launch_jacobi<T>(l2, L.Rb, (T*)L.Wt, (T*)L.Jt, L.sig, L.st, s);
  if (e != cudaSuccess) return e;
  launch_sort_gather<T>(l2, l2, L.sig, (const T*)L.Wt, (const T*)L.Jt, L.Dall, (T*)L.Wsel, (T*)L.Jsel, s);
  take_pairs_kernel<T><<<grid_of((long long)l2 * kk), 256, 0, s>>>(l2, kk, L.Dall, (const T*)L.Wsel,
                                                                   (const T*)L.Jsel, D, (T*)L.W2, (T*)L.J2);
  note_launch();
  // realified lifts: Uhat = Qhat W2 (2m x kk), Vhat = Q_B J2 (2n x kk)
  launch_gemm_simt<T>(false, 2 * m, kk, l2, Yh, l2, (const T*)L.W2, kk, (T*)L.Uh, kk, nullptr, sms, s);
  launch_gemm_simt<T>(false, 2 * n, kk, l2, Z, l2, (const T*)L.J2, kk, (T*)L.Vh, kk, nullptr, sms, s);
  // The realified Jacobi keeps the 2l real vectors orthonormal but not the
  // complex ones: a pair's partner i x is only approximately a computed
  // vector, and neighbouring pairs mix at the level u sigma_1 / gap.  A
  // complex CholeskyQR of U and of V (realified, interleaved) restores
  // complex orthonormality; it moves each vector by that same small amount
  // (the largest singular values first, least), well below the method's own
  // approximation error.
  for (int side = 0; side < 2; ++side) {
    const int rows = side == 0 ? m : n;
    T* Xh = (T*)(side == 0 ? L.Uh : L.Vh);
    T* Xi = (T*)L.Xi;
    pair_realify_kernel<T><<<grid_of((long long)rows * kk), 256, 0, s>>>(rows, kk, Xh, Xi);
    note_launch();
    if (tc)
      run_orth_tc(2 * rows, 2 * kk, (float*)Xi, 2 * kk, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
    else
      run_orth<T, T>(2 * rows, 2 * kk, Xi, 2 * kk, nullptr, nullptr, 0, L.orthws, L.st, sms, s);
    take_even_kernel<T><<<grid_of((long long)2 * rows * kk), 256, 0, s>>>(2 * rows, kk, Xi, Xh);
    note_launch();
  }
  srft_pack_kernel<T><<<kk, 256, 0, s>>>(m, n, kk, (const T*)L.Uh, (const T*)L.Vh, U, ldu, V, ldv);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t run_srft<float>(int, int, const float*, int, int, int, int, uint64_t, float*, int, double*,
                                     float*, int, const SrftLayout&, int, bool, cudaStream_t);
template cudaError_t run_srft<double>(int, int, const double*, int, int, int, int, uint64_t, double*, int, double*,
                                      double*, int, const SrftLayout&, int, bool, cudaStream_t);

}  // namespace rsvd
