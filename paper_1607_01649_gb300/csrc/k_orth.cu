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
                        int rows_per_split, const int* gate, const int* skip) {
  if ((gate && *gate == 0) || (skip && *skip != 0)) return;
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

// G[i][j] = sum over splits (fixed order) of the upper-triangular partials;
// Gf receives G rounded to binary32 (the Cholesky kernel's input on the
// binary32 path; converting here spreads the binary64 conversions over the GPU).
__global__ void gram_reduce_kernel(int l, int splits, const double* __restrict__ P, double* __restrict__ G,
                                   float* __restrict__ Gf, const int* gate, const int* skip) {
  if ((gate && *gate == 0) || (skip && *skip != 0)) return;
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
  if (Gf) Gf[idx] = (float)s;
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
void launch_gram(int rows, int l, const T* Y, int ldy, double* P, double* G, float* Gf, int sms, const int* gate,
                 cudaStream_t s, const int* skip) {
  const int nb = ceil_div(l, GT);
  const int tiles = nb * (nb + 1) / 2;
  const int splits = gram_splits(rows, l, sms);
  const int rps = ceil_div(ceil_div(rows, splits), GCH) * GCH;
  const int used = ceil_div(rows, rps);
  gram_partial_kernel<T><<<dim3(tiles, used), 256, 0, s>>>(rows, l, Y, ldy, P, rps, gate, skip);
  note_launch();
  gram_reduce_kernel<<<ceil_div(l * l, 256), 256, 0, s>>>(l, used, P, G, Gf, gate, skip);
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

// Single CTA of 1024 threads.  In: G (l x l binary64) and Gf (G rounded to
// binary32, used on the binary32 path).  Out:
//   Ub   : l x l row-major, type C: the upper triangular factor Lt^T whose
//          32 x 32 diagonal blocks are replaced by their inverses; with
//          dinv it defines Q = (Y D^-1) Lt^-T (blocked triangular solve)
//   dinv : 1 / d_i, d_i = sqrt(G_ii)
//   R    : optional l x l row-major binary64, R = Lt^T D (zeros below the diagonal)
// where G = D Gt D and Gt = Lt Lt^T.  Pivots below tau (unit-diagonal scale)
// restart the factorization on Gt + s I, s = s0, 32 s0, ...; four failures
// give RSVD_E_BREAKDOWN.
//
// Factorization: blocked right-looking on 32-column panels.  For each panel:
//   (b) the 32 x 32 diagonal block is factored by warp 0, lane i holding row i
//       in registers (pivot columns broadcast by shuffles);
//   (c) the rows below are solved against it, one thread per row;
//   (d) the trailing lower triangle is updated, A22 -= L21 L21^T, by all
//       threads in 4 x 4 register tiles.
// Finally the diagonal blocks are inverted, one warp per block.

// Warp-level Cholesky of a w x w block held as rows (lane i: row[0..31] =
// A(i, 0..31), lower part valid).  On return row[] holds row i of L.  Returns
// false (warp-uniformly) on a pivot below tau.
template <typename C>
__device__ __forceinline__ bool warp_chol32(C (&row)[32], int w, C tau) {
  const int lane = threadIdx.x % 32;
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if (q < w && ok) {  // warp-uniform; no break, so q stays a compile-time index
      const C akk = __shfl_sync(0xffffffffu, row[q], q);
      if (!(akk > tau) || !isfinite(akk)) {
        ok = false;
      } else {
        const C piv = sqrt(akk), rp = C(1) / piv;
        const C liq = (lane == q) ? piv : (lane > q ? row[q] * rp : C(0));
        row[q] = liq;
        // row i -= l(i, q) * l(j, q) for q < j <= i
#pragma unroll
        for (int j = q + 1; j < 32; ++j) {
          const C ljq = __shfl_sync(0xffffffffu, liq, j);
          if (lane >= j) row[j] = fma(-liq, ljq, row[j]);
        }
      }
    }
  }
  return ok;
}

// Warp-level inverse of the lower triangular w x w diagonal block at
// (c0, c0) of the packed factor.  Lane i ends with x[] = row i of L^-1.
// x doubles as the accumulator: lanes i > k add L(i, k) X(k, :) at step k,
// when lane k turns its accumulator into its final row.
template <typename C>
__device__ __forceinline__ void warp_trinv32(const C* a, const int* cb, int c0, int w, C (&x)[32]) {
  const int lane = threadIdx.x % 32;
  const int i = c0 + lane;
#pragma unroll
  for (int c = 0; c < 32; ++c) x[c] = C(0);
  const C rd = (lane < w) ? C(1) / a[cb[i] + i] : C(0);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k >= w) continue;  // warp-uniform; keeps k a compile-time index
    if (lane == k) {
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = ((c == k ? C(1) : C(0)) - x[c]) * rd;
    }
    const C lik = (lane > k && lane < w) ? a[cb[c0 + k] + i] : C(0);
#pragma unroll
    for (int c = 0; c <= k; ++c) {
      const C xkc = __shfl_sync(0xffffffffu, x[c], k);
      if (lane > k) x[c] = fma(lik, xkc, x[c]);
    }
  }
}

template <typename C, int NT>
__global__ void __launch_bounds__(NT)
    chol_kernel(int l, const double* __restrict__ G, const float* __restrict__ Gf, C* __restrict__ Ub,
                C* __restrict__ dinv, double* __restrict__ R, DevStatus* st, int pass, const int* gate,
                const int* skip) {
  if ((gate && *gate == 0) || (skip && *skip != 0)) return;
  extern __shared__ unsigned char smem_raw[];
  C* a = reinterpret_cast<C*>(smem_raw);  // packed lower, l(l+1)/2
  double* d = reinterpret_cast<double*>(smem_raw + (((size_t)l * (l + 1) / 2 * sizeof(C) + 15) & ~15));
  C* rdiag = reinterpret_cast<C*>(d + l);
  C* rdc = rdiag + l;
  int* cb = reinterpret_cast<int*>(rdc + l);  // pk(i, j) = cb[j] + i
  __shared__ int s_fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid / 32, lane = tid % 32;
  const double u = Eps<C>::u;
  const C ctau = (C)(1024.0 * u);
  const double s0 = 16384.0 * u;

  bool bad = false;
  for (int i = tid; i < l; i += nt) {
    const double gii = G[(size_t)i * l + i];
    if (!isfinite(gii)) bad = true;
    d[i] = gii > 0.0 ? sqrt(gii) : 1.0;
    rdc[i] = (C)(1.0 / d[i]);
    cb[i] = i * l - (i * (i - 1)) / 2 - i;
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  if (bad) atomicExch(&s_fail, 2);
  __syncthreads();
  if (s_fail == 2) {
    if (tid == 0) set_status(st, RSVD_E_NONFINITE);
    return;
  }

  C shift = C(0);
  int attempt = 0;
  for (;;) {
    // unit-diagonal scaling Gt = D^-1 G D^-1 in the working precision (a
    // binary64 divide per entry would cost more than the factorization)
    for (int j = warp; j < l; j += nt / 32) {
      const int base = cb[j];
      const C rj = rdc[j];
      for (int i = j + lane; i < l; i += 32) {
        C v = (sizeof(C) == 4 ? (C)Gf[(size_t)i * l + j] : (C)G[(size_t)i * l + j]) * rdc[i] * rj;
        if (i == j) v += shift;
        if (!isfinite(v)) v = C(0);
        a[base + i] = v;
      }
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int c0 = 0; c0 < l; c0 += 32) {
      const int w = min(32, l - c0);
      // (b) diagonal block
      if (warp == 0) {
        C row[32];
        const int i = c0 + lane;
#pragma unroll
        for (int j = 0; j < 32; ++j) row[j] = (lane < w && j < w && j <= lane) ? a[cb[c0 + j] + i] : C(0);
        const bool ok = warp_chol32<C>(row, w, ctau);
        if (!ok) {
          if (lane == 0) s_fail = 1;
        } else if (lane < w) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j <= lane) a[cb[c0 + j] + i] = row[j];
          C dii = C(1);
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j == lane) dii = row[j];
          rdiag[i] = C(1) / dii;
        }
      }
      __syncthreads();
      if (s_fail) break;
      // (c) rows below: x L11^T = a(i, c0 : c0 + w), thread per row
      for (int i = c0 + w + tid; i < l; i += nt) {
        C x[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) x[q] = q < w ? a[cb[c0 + q] + i] : C(0);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          if (q < w) {
            x[q] *= rdiag[c0 + q];
            const int bq = cb[c0 + q];
#pragma unroll
            for (int r2 = q + 1; r2 < 32; ++r2)
              if (r2 < w) x[r2] = fma(-x[q], a[bq + c0 + r2], x[r2]);
          }
        }
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (q < w) a[cb[c0 + q] + i] = x[q];
      }
      __syncthreads();
      // (d) trailing update A22 -= L21 L21^T over the lower triangle, 4 x 4 tiles
      const int t0 = c0 + w;
      const int n2 = l - t0;
      if (n2 > 0) {
        const int nq = (n2 + 3) / 4;             // row/column quads
        const int ntiles = nq * (nq + 1) / 2;    // lower-triangular tiles
        for (int tI = tid; tI < ntiles; tI += nt) {
          // tile index -> (rq, cq) with cq <= rq
          int rq = (int)((sqrtf(8.0f * tI + 1.0f) - 1.0f) * 0.5f);
          while ((rq + 1) * (rq + 2) / 2 <= tI) ++rq;
          while (rq * (rq + 1) / 2 > tI) --rq;
          const int cq = tI - rq * (rq + 1) / 2;
          const int i0 = t0 + 4 * rq, j0 = t0 + 4 * cq;
          C acc[4][4];
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = C(0);
          for (int k = c0; k < c0 + w; ++k) {
            const int base = cb[k];
            C av[4], bv[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) av[x] = (i0 + x < l) ? a[base + i0 + x] : C(0);
#pragma unroll
            for (int y = 0; y < 4; ++y) bv[y] = (j0 + y < l) ? a[base + j0 + y] : C(0);
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < 4; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              const int ii = i0 + x, jj = j0 + y;
              if (ii < l && jj < l && ii >= jj) a[cb[jj] + ii] -= acc[x][y];
            }
        }
        __syncthreads();
      }
    }
    __syncthreads();
    if (s_fail == 0) break;
    ++attempt;
    if (attempt > 4) {
      if (tid == 0) set_status(st, RSVD_E_BREAKDOWN);
      return;
    }
    shift = (shift == C(0)) ? (C)s0 : shift * C(32);
    __syncthreads();
  }
  if (tid == 0) {
    if (pass == 1)
      st->shifted = shift > C(0) ? 1 : 0;
    else if (shift > C(0))
      st->shifted = 1;
    if (shift > C(0)) atomicAdd(&st->shift_count, 1);
  }
  // outputs, row i of Ub / R by warp, columns by lane: Lt^T[i][j] = L(j, i), j >= i
  for (int i = warp; i < l; i += nt / 32) {
    const int bi = i >> 5;
    for (int j = lane; j < l; j += 32) {
      const C v = (j >= i) ? a[cb[i] + j] : C(0);
      if (R) R[(size_t)i * l + j] = (double)(v * (C)d[j]);
      if (bi != (j >> 5)) Ub[(size_t)i * l + j] = v;
    }
  }
  // diagonal blocks of Ub: (L(bb, bb)^-1)^T, one warp per block
  const int nb = (l + 31) / 32;
  for (int bb = warp; bb < nb; bb += nt / 32) {
    const int c0 = 32 * bb, w = min(32, l - c0);
    const int i = c0 + lane;
    C x[32];
    warp_trinv32<C>(a, cb, c0, w, x);
    // x = row `lane` of L^-1; Ub(c0 + c, c0 + lane) = L^-1(lane, c), i.e. column lane of the transposed inverse
    if (lane < w) {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < w) Ub[(size_t)(c0 + c) * l + c0 + lane] = x[c];
    }
  }
  for (int i = tid; i < l; i += nt) dinv[i] = rdc[i];
}

size_t chol_smem_bytes(int l, size_t csize) {
  return (((size_t)l * (l + 1) / 2 * csize + 15) & ~(size_t)15) + (size_t)l * sizeof(double) +
         (size_t)2 * l * csize + (size_t)l * sizeof(int);
}

// ----------------------------------------------------------------- apply --
// In place Q = (Y D^-1) Lt^-T as a blocked triangular solve.  One CTA per
// 64-row stripe, staged in shared memory before any row is rewritten.  For
// each 32-column block b (in order), with the block's 32 rows of Ub streamed
// into shared memory:
//   r_b = ytilde_b - (sum over earlier blocks, held in registers)
//   q_b = r_b Ub(b, b)                      (Ub(b, b) = inverse of the diagonal block)
//   acc_c += q_b Ub(b, c) for later blocks c (each thread owns a 8 x 8 tile:
//            rows ty + 8 x, columns tx + 32 y)
// Optionally writes a bf16 copy of Q.
template <typename T, typename C>
__global__ void __launch_bounds__(256)
    apply_kernel(int rows, int l, T* __restrict__ Y, int ldy, const C* __restrict__ Ub, const C* __restrict__ dinv,
                 __nv_bfloat16* __restrict__ Ybf, int lb, const int* gate, const int* skip) {
  if ((gate && *gate == 0) || (skip && *skip != 0)) return;
  extern __shared__ unsigned char smem_raw[];
  C* ys = reinterpret_cast<C*>(smem_raw);  // 64 x l
  C* rs = ys + (size_t)64 * l;             // 32 x l rows of Ub
  const int tid = threadIdx.x, tx = tid % 32, ty = tid / 32;
  const int r0 = blockIdx.x * 64;
  const int nr = min(64, rows - r0);
  // stage the stripe (row by row, no index division), scaled by dinv
  for (int r = 0; r < 64; ++r)
    for (int c = tid; c < l; c += 256)
      ys[(size_t)r * l + c] = (r < nr) ? (C)Y[(size_t)(r0 + r) * ldy + c] * dinv[c] : C(0);
  C acc[8][8];
#pragma unroll
  for (int x = 0; x < 8; ++x)
#pragma unroll
    for (int y = 0; y < 8; ++y) acc[x][y] = C(0);
  const int nb = (l + 31) / 32;
  // block b is a compile-time index, so the update below touches only the
  // later column blocks y > b
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b < nb) {
      const int k0 = 32 * b, kw = min(32, l - k0);
      __syncthreads();  // previous block's reads of rs / ys are done
      for (int kk = ty; kk < 32; kk += 8)
        for (int c = tx; c < l; c += 32)
          rs[(size_t)kk * l + c] = (kk < kw && c >= k0) ? Ub[(size_t)(k0 + kk) * l + c] : C(0);
      // r_b into ys (thread's column k0 + tx, rows ty + 8 x)
      const int cb_ = k0 + tx;
      if (tx < kw) {
#pragma unroll
        for (int x = 0; x < 8; ++x) ys[(size_t)(ty + 8 * x) * l + cb_] -= acc[x][b];
      }
      __syncthreads();
      // q_b = r_b Ub(b, b)
      C qv[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) qv[x] = C(0);
      if (tx < kw) {
        for (int kk = 0; kk < kw; ++kk) {
          const C ub = rs[(size_t)kk * l + cb_];
#pragma unroll
          for (int x = 0; x < 8; ++x) qv[x] = fma(ys[(size_t)(ty + 8 * x) * l + k0 + kk], ub, qv[x]);
        }
      }
      __syncthreads();  // all reads of r_b done
      if (tx < kw) {
#pragma unroll
        for (int x = 0; x < 8; ++x) ys[(size_t)(ty + 8 * x) * l + cb_] = qv[x];
      }
      __syncthreads();
      // acc_c += q_b Ub(b, c) for the later column blocks c > b
      if (b + 1 < nb) {
        for (int kk = 0; kk < kw; ++kk) {
          C yv[8];
#pragma unroll
          for (int x = 0; x < 8; ++x) yv[x] = ys[(size_t)(ty + 8 * x) * l + k0 + kk];
#pragma unroll
          for (int y = b + 1; y < 8; ++y) {
            const int c = tx + 32 * y;
            const C rv = (c < l) ? rs[(size_t)kk * l + c] : C(0);
#pragma unroll
            for (int x = 0; x < 8; ++x) acc[x][y] = fma(yv[x], rv, acc[x][y]);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int r = 0; r < nr; ++r)
    for (int c = tid; c < l; c += 256) {
      const C v = ys[(size_t)r * l + c];
      Y[(size_t)(r0 + r) * ldy + c] = (T)v;
      if (Ybf) Ybf[(size_t)(r0 + r) * lb + c] = __float2bfloat16_rn((float)v);
    }
}

template <typename T, typename C>
void launch_apply(int rows, int l, T* Y, int ldy, const C* Ub, const C* dinv, __nv_bfloat16* Ybf, int lb,
                  const int* gate, cudaStream_t s, const int* skip) {
  if (rows == 0) return;
  const size_t smem = (size_t)(64 + 32) * l * sizeof(C);
  auto kfn = apply_kernel<T, C>;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kfn<<<ceil_div(rows, 64), 256, smem, s>>>(rows, l, Y, ldy, Ub, dinv, Ybf, lb, gate, skip);
  note_launch();
}

template <typename C>
void launch_chol(int l, const double* G, const float* Gf, C* Ub, C* dinv, double* R, DevStatus* st, int pass,
                 const int* gate, cudaStream_t s, const int* skip) {
  // binary32: 1024 threads; binary64 (l <= 128): 256 threads with room for registers
  constexpr int NT = sizeof(C) == 4 ? 1024 : 256;
  const size_t smem = chol_smem_bytes(l, sizeof(C));
  auto kfn = chol_kernel<C, NT>;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kfn<<<1, NT, smem, s>>>(l, G, Gf, Ub, dinv, R, st, pass, gate, skip);
  note_launch();
}

// ------------------------------------------------- triangular products --
// C = A B for l x l row-major binary64 upper-triangular A, B (C upper too).
__global__ void triu_mm_kernel(int l, const double* __restrict__ A, const double* __restrict__ B,
                               double* __restrict__ Cm, const int* gate, int copy_if_gated, const int* skip) {
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  if (i >= l || j >= l) return;
  if (skip && *skip != 0) return;
  if (gate && *gate == 0) {
    if (copy_if_gated) Cm[(size_t)i * l + j] = B[(size_t)i * l + j];
    return;
  }
  double s = 0.0;
  for (int k = i; k <= j; ++k) s += A[(size_t)i * l + k] * B[(size_t)k * l + j];
  Cm[(size_t)i * l + j] = (i <= j) ? s : 0.0;
}

void launch_triu_mm(int l, const double* A, const double* B, double* Cm, const int* gate, int copy_if_gated,
                    cudaStream_t s, const int* skip) {
  dim3 grid(ceil_div(l, 16), ceil_div(l, 16));
  triu_mm_kernel<<<grid, dim3(16, 16), 0, s>>>(l, A, B, Cm, gate, copy_if_gated, skip);
  note_launch();
}

// ------------------------------------------------------------ orth driver --
size_t orth_workspace_bytes(int rows, int l, int sms, size_t csize) {
  Carver c(nullptr);
  c.take<double>((size_t)gram_splits(rows, l, sms) * l * l);  // Gram partials
  c.take<double>((size_t)l * l);                              // G
  c.take<float>((size_t)l * l);                               // Gf
  c.take<unsigned char>((size_t)l * l * csize);               // Ub
  c.take<unsigned char>((size_t)l * csize);                   // dinv
  c.take<double>((size_t)3 * l * l);                          // R per pass
  c.take<double>((size_t)2 * l * l);                          // R products
  return c.size();
}

template <typename T, typename C>
void run_orth(int rows, int l, T* Y, int ldy, double* Rout, __nv_bfloat16* Ybf, int lb, void* ws,
              DevStatus* st, int sms, cudaStream_t s, const int* skip) {
  Carver c(ws);
  double* P = c.take<double>((size_t)gram_splits(rows, l, sms) * l * l);
  double* G = c.take<double>((size_t)l * l);
  float* Gf = c.take<float>((size_t)l * l);
  C* Ub = c.take<C>((size_t)l * l);
  C* dinv = c.take<C>((size_t)l);
  double* Rp = c.take<double>((size_t)3 * l * l);
  double* Rm = c.take<double>((size_t)2 * l * l);
  const int* gate3 = &st->shifted;
  for (int pass = 1; pass <= 3; ++pass) {
    const int* gate = pass == 3 ? gate3 : nullptr;
    launch_gram<T>(rows, l, Y, ldy, P, G, sizeof(C) == 4 ? Gf : nullptr, sms, gate, s, skip);
    launch_chol<C>(l, G, Gf, Ub, dinv, Rout ? Rp + (size_t)(pass - 1) * l * l : nullptr, st, pass, gate, s, skip);
    launch_apply<T, C>(rows, l, Y, ldy, Ub, dinv, nullptr, lb, gate, s, skip);
  }
  if (Ybf) launch_copy_bf16<T>(rows, l, Y, ldy, Ybf, lb, s);
  if (Rout) {
    // R = R3 R2 R1 (R3 only if the third pass ran)
    launch_triu_mm(l, Rp + (size_t)l * l, Rp, Rm, nullptr, 0, s, skip);
    launch_triu_mm(l, Rp + (size_t)2 * l * l, Rm, Rout, gate3, 1, s, skip);
  }
}

template void run_orth<float, float>(int, int, float*, int, double*, __nv_bfloat16*, int, void*, DevStatus*,
                                     int, cudaStream_t, const int*);
template void run_orth<double, double>(int, int, double*, int, double*, __nv_bfloat16*, int, void*,
                                       DevStatus*, int, cudaStream_t, const int*);
template void launch_gram<float>(int, int, const float*, int, double*, double*, float*, int, const int*,
                                 cudaStream_t, const int*);
template void launch_gram<double>(int, int, const double*, int, double*, double*, float*, int, const int*,
                                  cudaStream_t, const int*);

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
