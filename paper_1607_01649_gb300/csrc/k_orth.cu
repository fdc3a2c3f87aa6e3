// Unpivoted orthonormalization "orth" (Sec. 2.3), as CholeskyQR2 with an
// optional shifted first pass (shifted CholeskyQR3: Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa, SISC 42 (2020)).
//
// One pass on a rows x l block Y (row-major, updated in place):
//   1. G = Y^T Y                    (gram_partial + gram_reduce; binary64 sums)
//   2. G = D Gt D, Gt = Lt Lt^T      (chol: unit-diagonal scaling in binary64,
//                                     Cholesky of Gt (+ s I when needed))
//   3. Y <- Y D^-1 Lt^-T             (apply: one warp per row, forward
//                                     substitution against Lt^T)
// so Y = Q R with R = Lt^T D upper triangular, diag(R) > 0.
//
// Binary64 on this part runs at 1/58 of binary32 (measured 1.20 TFLOP/s vs
// 70 TFLOP/s), so the plain-binary32 and mixed paths form each product of the
// Gram in binary32 over chunks of 128 rows and carry the running sums in
// binary64; the O(l^3) Cholesky and solve arithmetic is binary32 on a
// binary64-scaled matrix.  The binary64 path is binary64 throughout.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

// ------------------------------------------------------------------ Gram --
constexpr int GT = 64;       // Gram tile
constexpr int GCH = 32;      // rows per chunk in shared memory
constexpr int GFOLD = 4;     // chunks per binary64 fold (128 rows)

// Partial Gram of rows [r_beg, r_end) for the upper-triangular tile
// (bi, bj), bi <= bj, written to P[split][bi*GT + i][bj*GT + j] (ld = l).
template <typename T>
__global__ void __launch_bounds__(256)
    gram_partial_kernel(int rows, int l, const T* __restrict__ Y, int ldy, double* __restrict__ P,
                        int rows_per_split, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ T Yi[GCH][GT];
  __shared__ T Yj[GCH][GT];
  // tile index -> (bi, bj) with bi <= bj
  const int nb = ceil_div(l, GT);
  int t = blockIdx.x, bi = 0;
  while (t >= nb - bi) {
    t -= nb - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int r_beg = blockIdx.y * rows_per_split;
  const int r_end = min(rows, r_beg + rows_per_split);

  double acc[4][4];
  T part[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = 0.0;
      part[a][b] = T(0);
    }

  for (int r0 = r_beg; r0 < r_end; r0 += GCH) {
#pragma unroll
    for (int s = 0; s < (GCH * GT) / 256; ++s) {
      const int e = tid + 256 * s;
      const int rr = e / GT, c = e % GT;
      const int gr = r0 + rr;
      const int ci = bi * GT + c, cj = bj * GT + c;
      Yi[rr][c] = (gr < r_end && ci < l) ? Y[(size_t)gr * ldy + ci] : T(0);
      Yj[rr][c] = (gr < r_end && cj < l) ? Y[(size_t)gr * ldy + cj] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GCH; ++rr) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Yi[rr][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = Yj[rr][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) part[u][v] = fma(a[u], b[v], part[u][v]);
    }
    // every GFOLD rows (and at the end) fold the binary32 (or binary64) chunk
    // sums into the binary64 running sums
    if (((r0 - r_beg) / GCH) % GFOLD == GFOLD - 1 || r0 + GCH >= r_end) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[u][v] += (double)part[u][v];
          part[u][v] = T(0);
        }
    }
    __syncthreads();
  }
  double* out = P + (size_t)blockIdx.y * l * l;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = bi * GT + ty + 16 * u;
    if (i >= l) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = bj * GT + tx + 16 * v;
      if (j < l) out[(size_t)i * l + j] = acc[u][v];
    }
  }
}

// G[i][j] = sum over splits (fixed order) of the upper-triangular partials.
__global__ void gram_reduce_kernel(int l, int splits, const double* __restrict__ P, double* __restrict__ G,
                                   const int* gate) {
  if (gate && *gate == 0) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * l) return;
  int i = idx / l, j = idx % l;
  // tiles with bi > bj were not computed: read the mirrored entry instead
  if (i / GT > j / GT) {
    const int t = i;
    i = j;
    j = t;
  }
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += P[(size_t)z * l * l + (size_t)i * l + j];
  G[idx] = s;
}

int gram_splits(int rows, int l, int sms) {
  const int nb = ceil_div(l, GT);
  const int tiles = nb * (nb + 1) / 2;
  int s = ceil_div(2 * sms, tiles);
  const int smax = ceil_div(rows, 4 * GCH);
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  if (s > 256) s = 256;
  return s;
}

template <typename T>
void launch_gram(int rows, int l, const T* Y, int ldy, double* P, double* G, int sms, const int* gate,
                 cudaStream_t s) {
  const int nb = ceil_div(l, GT);
  const int tiles = nb * (nb + 1) / 2;
  const int splits = gram_splits(rows, l, sms);
  const int rps = ceil_div(ceil_div(rows, splits), GCH) * GCH;
  const int used = ceil_div(rows, rps);
  gram_partial_kernel<T><<<dim3(tiles, used), 256, 0, s>>>(rows, l, Y, ldy, P, rps, gate);
  note_launch();
  gram_reduce_kernel<<<ceil_div(l * l, 256), 256, 0, s>>>(l, used, P, G, gate);
  note_launch();
}

// -------------------------------------------------------------- Cholesky --
// Packed column-major lower triangle: column j holds rows j..l-1.
__device__ __forceinline__ int pk(int l, int i, int j) { return j * l - (j * (j - 1)) / 2 + (i - j); }

template <typename C>
struct Eps;
template <>
struct Eps<float> {
  static constexpr double u = 5.9604644775390625e-08;  // 2^-24
};
template <>
struct Eps<double> {
  static constexpr double u = 1.1102230246251565e-16;  // 2^-53
};

// Single CTA.  In:  G (l x l binary64).  Out:
//   Ut : packed row-major upper triangle of Lt^T (row r holds columns r..l-1), type C
//   dinv : 1 / d (type C), d_i = sqrt(G_ii)
//   R  : l x l row-major binary64, R = Lt^T D (zeros below the diagonal)
// Pivots below tau (unit-diagonal scale) restart the factorization on Gt + s I,
// s = s0, 32 s0, ...; four failures give RSVD_E_BREAKDOWN.
template <typename C>
__global__ void __launch_bounds__(1024)
    chol_kernel(int l, const double* __restrict__ G, C* __restrict__ Ut, C* __restrict__ dinv,
                double* __restrict__ R, DevStatus* st, int pass, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ unsigned char smem_raw[];
  C* a = reinterpret_cast<C*>(smem_raw);                    // packed lower, l(l+1)/2
  double* d = reinterpret_cast<double*>(smem_raw + (((size_t)l * (l + 1) / 2 * sizeof(C) + 15) & ~15));
  C* diag = reinterpret_cast<C*>(d + l);
  __shared__ int s_fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid / 32, lane = tid % 32, nw = nt / 32;
  const double u = Eps<C>::u;
  const double tau = 1024.0 * u;
  const double s0 = 16384.0 * u;

  C* rdc = diag + l;  // 1 / d_i in the working precision
  bool bad = false;
  for (int i = tid; i < l; i += nt) {
    const double gii = G[(size_t)i * l + i];
    if (!isfinite(gii)) bad = true;
    d[i] = gii > 0.0 ? sqrt(gii) : 1.0;
    rdc[i] = (C)(1.0 / d[i]);
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  if (bad) atomicExch(&s_fail, 2);
  __syncthreads();
  if (s_fail == 2) {
    if (tid == 0) set_status(st, RSVD_E_NONFINITE);
    return;
  }

  double shift = 0.0;
  int attempt = 0;
  for (;;) {
    const int npk = l * (l + 1) / 2;
    // unit-diagonal scaling Gt = D^-1 G D^-1 in the working precision (a
    // binary64 divide per entry would cost more than the factorization here)
    for (int e = tid; e < l * l; e += nt) {
      const int i = e / l, j = e % l;
      if (i < j) continue;
      C v = (C)G[(size_t)i * l + j] * rdc[i] * rdc[j];
      if (i == j) v += (C)shift;
      if (!isfinite(v)) v = C(0);
      a[pk(l, i, j)] = v;
    }
    (void)npk;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int k = 0; k < l; ++k) {
      const C akk = a[pk(l, k, k)];
      if (!((double)akk > tau) || !isfinite((double)akk)) {  // uniform decision
        if (tid == 0) s_fail = 1;
        break;
      }
      const C piv = sqrt(akk);
      if (tid == 0) diag[k] = piv;
      const C rp = C(1) / piv;
      for (int i = k + 1 + tid; i < l; i += nt) a[pk(l, i, k)] *= rp;
      __syncthreads();
      // trailing update a(i, j) -= l(i, k) l(j, k) for k < j <= i < l.  Lane
      // owns rows i = lane + 32 r (r < 8); its multipliers l(i, k) are loaded
      // once, then each column of the warp is updated with 8 independent FMAs.
      C lik[8];
      const int ck = pk(l, k, k);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int i = lane + 32 * r;
        lik[r] = (i > k && i < l) ? a[ck + (i - k)] : C(0);
      }
      for (int j = k + 1 + warp; j < l; j += nw) {
        const C ljk = a[ck + (j - k)];
        const int cj = pk(l, j, j);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = lane + 32 * r;
          if (i >= j && i < l) a[cj + (i - j)] -= lik[r] * ljk;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (s_fail == 0) break;
    ++attempt;
    if (attempt > 4) {
      if (tid == 0) set_status(st, RSVD_E_BREAKDOWN);
      return;
    }
    shift = (shift == 0.0) ? s0 : shift * 32.0;
    __syncthreads();
  }
  if (tid == 0) {
    if (pass == 1)
      st->shifted = shift > 0.0 ? 1 : 0;
    else if (shift > 0.0)
      st->shifted = 1;
    if (shift > 0.0) atomicAdd(&st->shift_count, 1);
  }
  // outputs
  for (int e = tid; e < l * l; e += nt) {
    const int i = e / l, j = e % l;  // R[i][j] = Lt[j][i] d_j for i <= j
    if (R) {
      C v = C(0);
      if (i < j)
        v = a[pk(l, j, i)] * (C)d[j];
      else if (i == j)
        v = diag[i] * (C)d[i];
      R[e] = (double)v;
    }
    if (i <= j) {
      const int off = i * l - (i * (i - 1)) / 2 + (j - i);  // packed row-major upper
      Ut[off] = (i == j) ? diag[i] : a[pk(l, j, i)];
    }
  }
  for (int i = tid; i < l; i += nt) dinv[i] = rdc[i];
}

size_t chol_smem_bytes(int l, size_t csize) {
  return (((size_t)l * (l + 1) / 2 * csize + 15) & ~(size_t)15) + (size_t)l * sizeof(double) +
         (size_t)2 * l * csize;
}

// ----------------------------------------------------------------- apply --
// In place: each warp takes RW rows y at a time; ytilde = y * dinv; solves
// q Lt^T = ytilde by forward substitution (lanes own columns c = lane + 32 t;
// the RW independent rows give the warp RW-way instruction-level parallelism).
// Optionally writes a bf16 copy of Q (row-major, ld = lb).
template <typename T, typename C, int NT>
__global__ void __launch_bounds__(1024)
    apply_kernel(int rows, int l, T* __restrict__ Y, int ldy, const C* __restrict__ Ut,
                 const C* __restrict__ dinv, __nv_bfloat16* __restrict__ Ybf, int lb, const int* gate) {
  if (gate && *gate == 0) return;
  constexpr int RW = 4;
  extern __shared__ unsigned char smem_raw[];
  C* u = reinterpret_cast<C*>(smem_raw);
  C* rdiag = u + (size_t)l * (l + 1) / 2;
  const int npk = l * (l + 1) / 2;
  for (int e = threadIdx.x; e < npk; e += blockDim.x) u[e] = Ut[e];
  for (int c = threadIdx.x; c < l; c += blockDim.x) rdiag[c] = C(1) / Ut[c * l - (c * (c - 1)) / 2];
  __syncthreads();
  const int lane = threadIdx.x % 32;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int nwarps = gridDim.x * blockDim.x / 32;
  C dv[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int c = lane + 32 * t;
    dv[t] = c < l ? dinv[c] : C(0);
  }
  for (int r0 = gw * RW; r0 < rows; r0 += nwarps * RW) {
    C s[RW][NT];
#pragma unroll
    for (int w = 0; w < RW; ++w) {
      const int r = r0 + w;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int c = lane + 32 * t;
        s[w][t] = (r < rows && c < l) ? (C)Y[(size_t)r * ldy + c] * dv[t] : C(0);
      }
    }
    int off = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      for (int cl = 0; cl < 32; ++cl) {
        const int c = 32 * t + cl;
        if (c >= l) break;
        const C rd = rdiag[c];
        C qc[RW];
#pragma unroll
        for (int w = 0; w < RW; ++w) {
          C v = C(0);
          if (lane == cl) {
            v = s[w][t] * rd;
            s[w][t] = v;
          }
          qc[w] = __shfl_sync(0xffffffffu, v, cl);
        }
#pragma unroll
        for (int t2 = 0; t2 < NT; ++t2) {
          const int c2 = lane + 32 * t2;
          if (t2 >= t && c2 > c && c2 < l) {
            const C uc = u[off + (c2 - c)];
#pragma unroll
            for (int w = 0; w < RW; ++w) s[w][t2] -= qc[w] * uc;
          }
        }
        off += l - c;
      }
    }
#pragma unroll
    for (int w = 0; w < RW; ++w) {
      const int r = r0 + w;
      if (r >= rows) continue;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int c = lane + 32 * t;
        if (c < l) {
          Y[(size_t)r * ldy + c] = (T)s[w][t];
          if (Ybf) Ybf[(size_t)r * lb + c] = __float2bfloat16_rn((float)s[w][t]);
        }
      }
    }
  }
}

template <typename T, typename C>
void launch_apply(int rows, int l, T* Y, int ldy, const C* Ut, const C* dinv, __nv_bfloat16* Ybf, int lb,
                  int sms, const int* gate, cudaStream_t s) {
  const size_t smem = ((size_t)l * (l + 1) / 2 + l) * sizeof(C);
  const int threads = 1024;
  const int blocks = sms;
#define RSVD_APPLY(NTV)                                                                              \
  do {                                                                                               \
    auto kfn = apply_kernel<T, C, NTV>;                                                              \
    cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);              \
    kfn<<<blocks, threads, smem, s>>>(rows, l, Y, ldy, Ut, dinv, Ybf, lb, gate);                     \
  } while (0)
  const int nt = ceil_div(l, 32);
  note_launch();
  if (nt <= 1)
    RSVD_APPLY(1);
  else if (nt <= 2)
    RSVD_APPLY(2);
  else if (nt <= 4)
    RSVD_APPLY(4);
  else
    RSVD_APPLY(8);
#undef RSVD_APPLY
}

template <typename C>
void launch_chol(int l, const double* G, C* Ut, C* dinv, double* R, DevStatus* st, int pass,
                 const int* gate, cudaStream_t s) {
  const size_t smem = chol_smem_bytes(l, sizeof(C));
  auto kfn = chol_kernel<C>;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kfn<<<1, 1024, smem, s>>>(l, G, Ut, dinv, R, st, pass, gate);
  note_launch();
}

// ------------------------------------------------- triangular products --
// C = A B for l x l row-major binary64 upper-triangular A, B (C upper too).
__global__ void triu_mm_kernel(int l, const double* __restrict__ A, const double* __restrict__ B,
                               double* __restrict__ Cm, const int* gate, int copy_if_gated) {
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  if (i >= l || j >= l) return;
  if (gate && *gate == 0) {
    if (copy_if_gated) Cm[(size_t)i * l + j] = B[(size_t)i * l + j];
    return;
  }
  double s = 0.0;
  for (int k = i; k <= j; ++k) s += A[(size_t)i * l + k] * B[(size_t)k * l + j];
  Cm[(size_t)i * l + j] = (i <= j) ? s : 0.0;
}

void launch_triu_mm(int l, const double* A, const double* B, double* Cm, const int* gate, int copy_if_gated,
                    cudaStream_t s) {
  dim3 grid(ceil_div(l, 16), ceil_div(l, 16));
  triu_mm_kernel<<<grid, dim3(16, 16), 0, s>>>(l, A, B, Cm, gate, copy_if_gated);
  note_launch();
}

// ------------------------------------------------------------ orth driver --
size_t orth_workspace_bytes(int rows, int l, int sms, size_t csize) {
  Carver c(nullptr);
  c.take<double>((size_t)gram_splits(rows, l, sms) * l * l);  // Gram partials
  c.take<double>((size_t)l * l);                              // G
  c.take<unsigned char>((size_t)l * (l + 1) / 2 * csize);     // Ut
  c.take<unsigned char>((size_t)l * csize);                   // dinv
  c.take<double>((size_t)3 * l * l);                          // R per pass
  c.take<double>((size_t)2 * l * l);                          // R products
  return c.size();
}

template <typename T, typename C>
void run_orth(int rows, int l, T* Y, int ldy, double* Rout, __nv_bfloat16* Ybf, int lb, void* ws,
              DevStatus* st, int sms, cudaStream_t s) {
  Carver c(ws);
  double* P = c.take<double>((size_t)gram_splits(rows, l, sms) * l * l);
  double* G = c.take<double>((size_t)l * l);
  C* Ut = c.take<C>((size_t)l * (l + 1) / 2);
  C* dinv = c.take<C>((size_t)l);
  double* Rp = c.take<double>((size_t)3 * l * l);
  double* Rm = c.take<double>((size_t)2 * l * l);
  const int* gate3 = &st->shifted;
  for (int pass = 1; pass <= 3; ++pass) {
    const int* gate = pass == 3 ? gate3 : nullptr;
    launch_gram<T>(rows, l, Y, ldy, P, G, sms, gate, s);
    launch_chol<C>(l, G, Ut, dinv, Rout ? Rp + (size_t)(pass - 1) * l * l : nullptr, st, pass, gate, s);
    launch_apply<T, C>(rows, l, Y, ldy, Ut, dinv, nullptr, lb, sms, gate, s);
  }
  if (Ybf) launch_copy_bf16<T>(rows, l, Y, ldy, Ybf, lb, s);
  if (Rout) {
    // R = R3 R2 R1 (R3 only if the third pass ran)
    launch_triu_mm(l, Rp + (size_t)l * l, Rp, Rm, nullptr, 0, s);
    launch_triu_mm(l, Rp + (size_t)2 * l * l, Rm, Rout, gate3, 1, s);
  }
}

template void run_orth<float, float>(int, int, float*, int, double*, __nv_bfloat16*, int, void*, DevStatus*,
                                     int, cudaStream_t);
template void run_orth<double, double>(int, int, double*, int, double*, __nv_bfloat16*, int, void*,
                                       DevStatus*, int, cudaStream_t);
template void launch_gram<float>(int, int, const float*, int, double*, double*, int, const int*, cudaStream_t);
template void launch_gram<double>(int, int, const double*, int, double*, double*, int, const int*,
                                  cudaStream_t);

// ------------------------------------------------------------ bf16 copy --
template <typename T>
__global__ void copy_bf16_kernel(int rows, int l, const T* __restrict__ Y, int ldy, __nv_bfloat16* __restrict__ Yb,
                                 int lb) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * l) return;
  const int r = (int)(idx / l), c = (int)(idx % l);
  Yb[(size_t)r * lb + c] = __float2bfloat16_rn((float)Y[(size_t)r * ldy + c]);
}

template <typename T>
void launch_copy_bf16(int rows, int l, const T* Y, int ldy, __nv_bfloat16* Yb, int lb, cudaStream_t s) {
  const long long total = (long long)rows * l;
  if (total == 0) return;
  copy_bf16_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(rows, l, Y, ldy, Yb, lb);
  note_launch();
}
template void launch_copy_bf16<float>(int, int, const float*, int, __nv_bfloat16*, int, cudaStream_t);
template void launch_copy_bf16<double>(int, int, const double*, int, __nv_bfloat16*, int, cudaStream_t);

}  // namespace rsvd
