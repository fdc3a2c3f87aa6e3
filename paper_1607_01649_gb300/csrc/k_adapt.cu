// Tolerance-driven range finder: the blocked greedy scheme of Sec. 12.3
// (Fig. greedy_blocked) with the residual norm computed directly from the
// explicitly updated matrix (Sec. 12.4 gives the downdate; in binary32 it
// cannot resolve small tolerances, so the remainder's norm is accumulated in
// binary64 during the update itself).
//
// One step t (b = block columns, tb = t * b columns accepted so far):
//   G_t  = randn(n, b), columns tb .. tb + b - 1 of Philox stream 1
//   Y    = A_j G_t                        -> written into Q(:, tb : tb + b)
//   q times (power variant of the figure's caption, orth between products):
//          Y = orth(Y);  Z = orth(A_j^T Y);  Y = A_j Z
//   Y   -= Q(:, :tb) (Q(:, :tb)^T Y)      (no-op in exact arithmetic; keeps Q orthonormal)
//   Q_new = orth(Y)                       (CholeskyQR2, in place)
//   B_new^T = A_j^T Q_new                 -> Bt(:, tb : tb + b)
//   A_j  -= Q_new B_new                   (deflation)
//   B2^T = A_j^T Q_new; A_j -= Q_new B2; B_new += B2, ||A_j||_F^2 in binary64
// The second deflation is zero in exact arithmetic.  A binary32 CholeskyQR2
// block is orthonormal only to about 1e-6, so one deflation leaves that much of
// A_j inside span(Q_new), which the projection of later samples would hide
// from every later step (the residual would stall near tol = 1e-6); the second
// pass leaves only the square of that.
//   stop when ||A_j||_F <= tol ||A||_F, or the rank reaches max_rank.
// Spectral mode (Sec. 13, Fig. adaptive2 and Lemma thm:aposteriori): before
// a block is appended, its fresh samples A_j G_t = (I - Q Q^T) A G_t serve as
// the b probes; if each has norm at most eps / (10 sqrt(2/pi)), then
// ||A - Q B||_2 <= eps with probability at least 1 - 10^-b and the loop stops
// without appending (no power steps in this mode).
// Every kernel of a step returns at once when the device flag `done` is set,
// so the host enqueues ceil(max_rank / b) steps without synchronizing.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

constexpr int AD_THREADS = 256;

// Aj = A, per-CTA binary64 partial sums of squares.
template <typename T>
__global__ void adapt_init_kernel(int m, int n, const T* __restrict__ A, int lda, T* __restrict__ Aj,
                                  double* __restrict__ pnorm) {
  __shared__ double red[AD_THREADS / 32];
  double acc = 0.0;
  const long long total = (long long)m * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const T v = A[(size_t)i * lda + j];
    Aj[e] = v;
    acc += (double)v * (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < AD_THREADS / 32; ++w) s += red[w];
    pnorm[blockIdx.x] = s;
  }
}

__global__ void adapt_norm_kernel(int nparts, const double* __restrict__ pnorm, double tol, int max_rank,
                                  DevStatus* st) {
  if (threadIdx.x != 0) return;
  double a2 = 0.0;
  for (int p = 0; p < nparts; ++p) a2 += pnorm[p];
  st->fro2_a = a2;
  st->fro2_res = a2;
  st->scratch[0] = tol * tol * a2;  // eps^2
  st->rank = 0;
  st->done = (a2 == 0.0 || max_rank == 0) ? 1 : 0;
  if (!isfinite(a2)) {
    set_status(st, RSVD_E_NONFINITE);
    st->done = 1;
  }
}

// Y(i, c) = sum_k Aj(i, k) G(k, c), c < bb; warp per row, G staged in shared
// memory in chunks of KCH rows.
constexpr int KCH = 128;
template <typename T>
__global__ void adapt_sketch_kernel(int m, int n, int bb, const T* __restrict__ Aj, const T* __restrict__ G, int ldg,
                                    T* __restrict__ Y, int ldy, const int* done) {
  if (*done) return;
  __shared__ T gs[KCH * 32];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const int i = blockIdx.x * nw + warp;
  T acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = T(0);
  for (int k0 = 0; k0 < n; k0 += KCH) {
    const int kw = min(KCH, n - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kw * 32; e += blockDim.x) {
      const int kk = e / 32, c = e % 32;
      gs[e] = (c < bb) ? G[(size_t)(k0 + kk) * ldg + c] : T(0);
    }
    __syncthreads();
    if (i < m) {
      for (int kk = lane; kk < kw; kk += 32) {
        const T a = Aj[(size_t)i * n + k0 + kk];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = fma(a, gs[kk * 32 + c], acc[c]);
      }
    }
  }
  if (i >= m) return;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    T v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == c && c < bb) Y[(size_t)i * ldy + c] = v;
  }
}

// Partial C_part(split)(k, c) = sum over this split's rows of Q(i, k) Y(i, c), k < tb, c < bb.
template <typename T>
__global__ void adapt_coef_kernel(int m, int tb, int bb, const T* __restrict__ Q, int ldq, const T* __restrict__ Y,
                                  int ldy, int rows_per, T* __restrict__ Cp, const int* done) {
  if (*done) return;
  const int r0 = blockIdx.y * rows_per, r1 = min(m, r0 + rows_per);
  // thread -> (k, c) with k = blockIdx.x * 8 + threadIdx.x / 32, c = lane
  const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, c = threadIdx.x % 32;
  if (k >= tb || c >= bb) return;
  T acc = T(0);
  for (int i = r0; i < r1; ++i) acc = fma(Q[(size_t)i * ldq + k], Y[(size_t)i * ldy + c], acc);
  Cp[((size_t)blockIdx.y * tb + k) * bb + c] = acc;
}

// Y(i, c) -= sum_k Q(i, k) C(k, c), with C = sum over splits of C_part (fixed order).
template <typename T>
__global__ void adapt_project_kernel(int m, int tb, int bb, int splits, const T* __restrict__ Q, int ldq,
                                     const T* __restrict__ Cp, T* __restrict__ Y, int ldy, const int* done) {
  if (*done) return;
  extern __shared__ unsigned char smem_raw[];
  T* cs = reinterpret_cast<T*>(smem_raw);  // tb x bb
  for (int e = threadIdx.x; e < tb * bb; e += blockDim.x) {
    T s = T(0);
    for (int z = 0; z < splits; ++z) s += Cp[(size_t)z * tb * bb + e];
    cs[e] = s;
  }
  __syncthreads();
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  for (int i = blockIdx.x * nw + warp; i < m; i += gridDim.x * nw) {
    if (lane >= bb) continue;
    T acc = T(0);
    for (int k = 0; k < tb; ++k) acc = fma(Q[(size_t)i * ldq + k], cs[k * bb + lane], acc);
    Y[(size_t)i * ldy + lane] -= acc;
  }
}

// Partial Bt_part(split)(j, c) = sum over this split's rows of Aj(i, j) Qn(i, c),
// in the working precision over chunks of 64 rows, folded into binary64 (a
// long binary32 sum would leave an error near sqrt(m) u ||A|| in B, which the
// update would carry into the remainder and keep it above small tolerances).
template <typename T>
__global__ void __launch_bounds__(128) adapt_bt_kernel(int m, int n, int bb, const T* __restrict__ Aj,
                                                       const T* __restrict__ Qn, int ldq, int rows_per,
                                                       double* __restrict__ Btp, const int* done) {
  if (*done) return;
  __shared__ T qs[64 * 32];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = blockIdx.y * rows_per, r1 = min(m, r0 + rows_per);
  double acc64[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc64[c] = 0.0;
  for (int i0 = r0; i0 < r1; i0 += 64) {
    const int iw = min(64, r1 - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < iw * 32; e += blockDim.x) {
      const int ii = e / 32, c = e % 32;
      qs[e] = (c < bb) ? Qn[(size_t)(i0 + ii) * ldq + c] : T(0);
    }
    __syncthreads();
    if (j < n) {
      T acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = T(0);
      for (int ii = 0; ii < iw; ++ii) {
        const T a = Aj[(size_t)(i0 + ii) * n + j];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = fma(a, qs[ii * 32 + c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) acc64[c] += (double)acc[c];
    }
  }
  if (j >= n) return;
#pragma unroll
  for (int c = 0; c < 32; ++c)
    if (c < bb) Btp[((size_t)blockIdx.y * n + j) * 32 + c] = acc64[c];
}

// Bt(j, c) = sum over splits of Bt_part (fixed order, binary64).
template <typename T>
__global__ void adapt_bt_reduce_kernel(int n, int bb, int splits, const double* __restrict__ Btp, T* __restrict__ Bt,
                                       int ldbt, T* __restrict__ Bacc, const int* done) {
  if (*done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * bb) return;
  const int j = e / bb, c = e % bb;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += Btp[((size_t)z * n + j) * 32 + c];
  Bt[(size_t)j * ldbt + c] = (T)s;  // this pass's coefficients
  if (Bacc) Bacc[(size_t)j * ldbt + c] = (T)((double)Bacc[(size_t)j * ldbt + c] + s);  // B_new += B2
}

// Aj(i, j) -= sum_c Qn(i, c) Bt(j, c); per-CTA binary64 sum of the updated squares.
template <typename T>
__global__ void adapt_update_kernel(int m, int n, int bb, T* __restrict__ Aj, const T* __restrict__ Qn, int ldq,
                                    const T* __restrict__ Bt, int ldbt, double* __restrict__ pnorm, const int* done) {
  if (*done) return;
  __shared__ T qs[32 * 33];
  __shared__ T bs[32 * 33];
  __shared__ double red[8];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 8 x 32 threads
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e / 32, c = e % 32;
    qs[r * 33 + c] = (i0 + r < m && c < bb) ? Qn[(size_t)(i0 + r) * ldq + c] : T(0);
    bs[r * 33 + c] = (j0 + r < n && c < bb) ? Bt[(size_t)(j0 + r) * ldbt + c] : T(0);
  }
  __syncthreads();
  double acc2 = 0.0;
  const int j = j0 + tx;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    if (i >= m || j >= n) continue;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 32; ++c) s = fma(qs[r * 33 + c], bs[tx * 33 + c], s);
    const T v = Aj[(size_t)i * n + j] - s;
    Aj[(size_t)i * n + j] = v;
    acc2 += (double)v * (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  if (tx == 0) red[ty] = acc2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    pnorm[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// Stopping test after step t: rank = tb + bb; ||A_j||_F^2 = sum of the update
// partials (fixed order); done when <= eps^2 (Frobenius mode only) or the
// rank reaches max_rank.
__global__ void adapt_check_kernel(int nparts, const double* __restrict__ pnorm, int new_rank, int max_rank,
                                   int spectral, DevStatus* st) {
  if (threadIdx.x != 0 || st->done) return;
  double r2 = 0.0;
  for (int p = 0; p < nparts; ++p) r2 += pnorm[p];
  st->fro2_res = r2;
  st->rank = new_rank;
  if (!isfinite(r2)) {
    set_status(st, RSVD_E_NONFINITE);
    st->done = 1;
  } else if (!spectral && r2 <= st->scratch[0]) {
    st->done = 1;
  } else if (new_rank >= max_rank) {
    set_status(st, RSVD_E_NOT_CONVERGED);
    st->done = 1;
  }
}

// Spectral-norm stopping test (Fig. adaptive2 with Lemma thm:aposteriori,
// alpha = 1/10): the fresh block Y = A_j G_t, drawn independently of the
// current Q, holds b samples (I - Q Q^T) A g_i.  Partial column sums of
// squares in binary64 over row slices, then the test.
constexpr int PROBE_ROWS = 2048;
template <typename T>
__global__ void __launch_bounds__(256) adapt_probe_partial_kernel(int m, int bb, const T* __restrict__ Y, int ldy,
                                                                  double* __restrict__ pp, const int* done) {
  if (*done) return;
  __shared__ double red[8][32];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int r0 = blockIdx.x * PROBE_ROWS, r1 = min(m, r0 + PROBE_ROWS);
  double acc = 0.0;
  if (lane < bb)
    for (int i = r0 + warp; i < r1; i += 8) {
      const double v = (double)Y[(size_t)i * ldy + lane];
      acc = fma(v, v, acc);
    }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][lane];
    pp[(size_t)blockIdx.x * 32 + lane] = s;
  }
}

// Sums the partials in a fixed order; stops the loop (rank unchanged) when
// every probe norm is at most thresh = eps / (10 sqrt(2/pi)).  The largest
// probe norm is kept in scratch[1].
__global__ void adapt_probe_check_kernel(int parts, int bb, const double* __restrict__ pp, double thresh,
                                         DevStatus* st) {
  if (st->done) return;
  const int lane = threadIdx.x;
  double s = 0.0;
  if (lane < bb)
    for (int p = 0; p < parts; ++p) s += pp[(size_t)p * 32 + lane];
  double mx = lane < bb ? s : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    const double nrm = sqrt(mx);
    st->scratch[1] = nrm;
    if (!isfinite(nrm)) {
      set_status(st, RSVD_E_NONFINITE);
      st->done = 1;
    } else if (nrm <= thresh) {
      st->scratch[2] = 1.0;  // converged on the spectral test
      st->done = 1;
    }
  }
}

// ------------------------------------------------------------------ host --
size_t adapt_workspace_bytes(int m, int n, int R, int b, int sms, size_t es) {
  Carver c(nullptr);
  c.take<unsigned char>((size_t)m * n * es);  // Aj
  c.take<unsigned char>((size_t)m * R * es);  // Q
  c.take<unsigned char>((size_t)n * R * es);  // Bt
  c.take<unsigned char>((size_t)n * R * es);  // B2 (second deflation)
  c.take<unsigned char>((size_t)n * b * es);  // G
  c.take<unsigned char>((size_t)64 * R * b * es);  // projection coefficient partials
  const int splits = 64;
  c.take<double>((size_t)splits * n * 32);                   // Bt partials (binary64)
  const size_t np = (size_t)ceil_div(m, 32) * ceil_div(n, 32);
  c.take<double>(np > 4096 ? np : 4096);                     // norm partials
  c.take<double>((size_t)ceil_div(m, PROBE_ROWS) * 32);       // probe partials
  (void)sms;
  return c.size();
}

template <typename T>
struct AdaptBufs {
  T *Aj, *Q, *Bt, *B2, *G, *Cp;
  double* Btp;
  double* pn;
  double* pp;
};

template <typename T>
AdaptBufs<T> adapt_carve(void* ws, int m, int n, int R, int b) {
  Carver c(ws);
  AdaptBufs<T> B;
  B.Aj = c.take<T>((size_t)m * n);
  B.Q = c.take<T>((size_t)m * R);
  B.Bt = c.take<T>((size_t)n * R);
  B.B2 = c.take<T>((size_t)n * R);
  B.G = c.take<T>((size_t)n * b);
  B.Cp = c.take<T>((size_t)64 * R * b);
  B.Btp = c.take<double>((size_t)64 * n * 32);
  const size_t np = (size_t)ceil_div(m, 32) * ceil_div(n, 32);
  B.pn = c.take<double>(np > 4096 ? np : 4096);
  B.pp = c.take<double>((size_t)ceil_div(m, PROBE_ROWS) * 32);
  return B;
}

// Enqueues the whole tolerance loop (ceil(R / b) gated steps) for an m x n
// matrix A.  Afterwards Q (m x rank, ld R) and Bt (n x rank, ld R) hold the
// factorization A ~= Q B, st->rank the rank, st->fro2_res and st->fro2_a the
// squared norms.
template <typename T, typename C>
void run_adaptive(int m, int n, const T* A, int lda, double tol, int R, int b, int q, uint64_t seed, void* ws,
                  void* orthws, DevStatus* st, int sms, cudaStream_t s, T** Qout, T** Btout, double spectral_eps) {
  const bool spectral = spectral_eps > 0.0;
  AdaptBufs<T> B = adapt_carve<T>(ws, m, n, R, b);
  *Qout = B.Q;
  *Btout = B.Bt;
  const int* done = &st->done;
  const int init_blocks = sms * 4;
  adapt_init_kernel<T><<<init_blocks, AD_THREADS, 0, s>>>(m, n, A, lda, B.Aj, B.pn);
  note_launch();
  adapt_norm_kernel<<<1, 32, 0, s>>>(init_blocks, B.pn, tol, R, st);
  note_launch();
  const int dt = sizeof(T) == 8 ? RSVD_DT_F64 : RSVD_DT_F32;
  for (int t = 0; t * b < R; ++t) {
    const int tb = t * b;
    const int bb = (R - tb) < b ? (R - tb) : b;
    T* Y = B.Q + tb;
    launch_gaussian(n, bb, seed, 1u, tb, dt, B.G, b, s);
    adapt_sketch_kernel<T><<<ceil_div(m, 8), 256, 0, s>>>(m, n, bb, B.Aj, B.G, b, Y, R, done);
    note_launch();
    if (spectral) {
      // the fresh samples are the probes: stop before appending them if
      // max_i ||A_j g_i|| <= eps / (10 sqrt(2/pi))
      const int parts = ceil_div(m, PROBE_ROWS);
      adapt_probe_partial_kernel<T><<<parts, 256, 0, s>>>(m, bb, Y, R, B.pp, done);
      note_launch();
      adapt_probe_check_kernel<<<1, 32, 0, s>>>(parts, bb, B.pp, spectral_eps / (10.0 * sqrt(2.0 / M_PI)), st);
      note_launch();
    }
    for (int j = 0; j < q; ++j) {
      // Y = orth(Y); Z = orth(A_j^T Y) (into the G buffer, binary64 row sums);
      // Y = A_j Z
      run_orth<T, C>(m, bb, Y, R, nullptr, nullptr, 0, orthws, st, sms, s, done);
      const int splits = ceil_div(m, 256) < 64 ? ceil_div(m, 256) : 64;
      const int rows_per = ceil_div(m, splits);
      adapt_bt_kernel<T><<<dim3(ceil_div(n, 128), splits), 128, 0, s>>>(m, n, bb, B.Aj, Y, R, rows_per, B.Btp,
                                                                        done);
      note_launch();
      adapt_bt_reduce_kernel<T><<<ceil_div(n * bb, 256), 256, 0, s>>>(n, bb, splits, B.Btp, B.G, b, nullptr, done);
      note_launch();
      run_orth<T, C>(n, bb, B.G, b, nullptr, nullptr, 0, orthws, st, sms, s, done);
      adapt_sketch_kernel<T><<<ceil_div(m, 8), 256, 0, s>>>(m, n, bb, B.Aj, B.G, b, Y, R, done);
      note_launch();
    }
    if (tb > 0) {
      const int splits = ceil_div(m, 512) < 64 ? ceil_div(m, 512) : 64;
      const int rows_per = ceil_div(m, splits);
      adapt_coef_kernel<T><<<dim3(ceil_div(tb, 8), splits), 256, 0, s>>>(m, tb, bb, B.Q, R, Y, R, rows_per, B.Cp,
                                                                         done);
      note_launch();
      const size_t smem = (size_t)tb * bb * sizeof(T);
      adapt_project_kernel<T><<<sms, 256, smem, s>>>(m, tb, bb, splits, B.Q, R, B.Cp, Y, R, done);
      note_launch();
    }
    run_orth<T, C>(m, bb, Y, R, nullptr, nullptr, 0, orthws, st, sms, s, done);
    dim3 ug(ceil_div(n, 32), ceil_div(m, 32));
    for (int pass = 0; pass < 2; ++pass) {
      const int splits = ceil_div(m, 256) < 64 ? ceil_div(m, 256) : 64;
      const int rows_per = ceil_div(m, splits);
      adapt_bt_kernel<T><<<dim3(ceil_div(n, 128), splits), 128, 0, s>>>(m, n, bb, B.Aj, Y, R, rows_per, B.Btp,
                                                                        done);
      note_launch();
      // pass 0 writes B_new into Bt; pass 1 writes B2 into scratch and adds it to B_new
      T* dst = pass == 0 ? B.Bt + tb : B.B2 + tb;
      adapt_bt_reduce_kernel<T><<<ceil_div(n * bb, 256), 256, 0, s>>>(n, bb, splits, B.Btp, dst, R,
                                                                      pass == 0 ? nullptr : B.Bt + tb, done);
      note_launch();
      adapt_update_kernel<T><<<ug, 256, 0, s>>>(m, n, bb, B.Aj, Y, R, dst, R, B.pn, done);
      note_launch();
    }
    adapt_check_kernel<<<1, 32, 0, s>>>((int)(ug.x * ug.y), B.pn, tb + bb, R, spectral ? 1 : 0, st);
    note_launch();
  }
}

template void run_adaptive<float, float>(int, int, const float*, int, double, int, int, int, uint64_t, void*,
                                         void*, DevStatus*, int, cudaStream_t, float**, float**, double);
template void run_adaptive<double, double>(int, int, const double*, int, double, int, int, int, uint64_t, void*,
                                           void*, DevStatus*, int, cudaStream_t, double**, double**, double);

}  // namespace rsvd
