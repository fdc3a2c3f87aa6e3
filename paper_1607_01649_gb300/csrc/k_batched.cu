// Batched tolerance-driven randomized SVD: many independent binary32 problems
// (1 <= m, n <= 1024) in ONE persistent launch.  Each CTA takes problems from a
// queue ordered largest-first (an atomic counter; nothing waits on another
// CTA) and runs, for each, the blocked greedy range finder of Sec. 12.3 (Fig.
// greedy_blocked, with the projection and the double deflation of the
// single-problem path) and then Stage B of Sec. 3, on its own SM:
//
//   A_j = A;  loop while ||A_j||_F > tol ||A||_F and rank < R:
//     G = randn(n, b) (Philox stream 1, columns b t ..; key = seed + problem)
//     Y = A_j G;  Y -= Q (Q^T Y);  Q_new = CholeskyQR2(Y)
//     C1 = Q_new^T A_j;  A_j -= Q_new C1;  C2 = Q_new^T A_j;  A_j -= Q_new C2
//     B_new = C1 + C2;  Q = [Q Q_new];  B = [B; B_new]
//   Stage B: B^T = Q_B R_B (CholeskyQR2), one-sided Jacobi on R_B^T,
//            U = Q Uhat, V = Q_B J, sign convention (largest |v_i| entry > 0).
//
// The passes over A_j are fused so that each step reads A_j three times and
// writes it twice:
//   pass C   C1 = Q_new^T A_j                         (column-owned threads)
//   pass U1  A_j -= Q_new C1, C2 = Q_new^T A_j        (column-owned threads)
//   pass U2  A_j -= Q_new C2, ||A_j||_F^2, Y = A_j G  (row-owned warps)
// where the Y of pass U2 is the next step's sample, formed before the
// stopping test (and unused after the last step).  The first step reads A
// itself and writes the working copy.  Arithmetic is binary32, with binary64
// norms and binary64 folds of 64-term binary32 partial sums in the reductions
// over rows; the only waits are CTA barriers.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

namespace {

constexpr int BT = 256;      // threads per CTA
constexpr int BW = BT / 32;  // warps per CTA
constexpr int BB = 16;       // largest block width b (row stride of Y, G, C)
constexpr int RMAX = 64;     // rank cap
constexpr int NMAX = 1024;   // largest m, n
// binary32 partial-sum length before a binary64 fold (binary64 adds run at
// 1/64 of the binary32 rate on this part)
constexpr int CHUNK = 256;
constexpr int YLD = BB + 1;  // odd row stride of the copy of Y being orthonormalized

// dynamic shared memory, in floats
constexpr int SQ_OFF = 0;                   // Y / Q_new, [i][16]   (NMAX x 16)
constexpr int SG_OFF = NMAX * BB;           // G, [j][16]; partials (NMAX x 16)
constexpr int SC_OFF = 2 * NMAX * BB;       // C1 / C2, [j][16]     (NMAX x 16)
constexpr int SP_OFF = 3 * NMAX * BB;       // Q^T Y, [k][16]       (RMAX x 16)
constexpr int SS_OFF = SP_OFF + RMAX * BB;  // Gram (16 x 16 binary64), L, U of the LU, dinv
constexpr int SMEM_FLOATS = SS_OFF + 2 * BB * BB + 2 * BB * BB + 2 * BB;
constexpr size_t SMEM_BYTES = (size_t)SMEM_FLOATS * sizeof(float);

// per-CTA working slot in the workspace, in floats
constexpr size_t SLOT_FLOATS = (size_t)NMAX * NMAX    // A_j, row stride n
                               + (size_t)RMAX * NMAX  // Q^T, [k][i]
                               + (size_t)NMAX * RMAX; // B^T, [j][k]

struct Prob {
  int m, n, lda;
  const float* A;
  float* U;
  double* D;
  float* V;
};

__device__ __forceinline__ double block_sum_f64(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < BW; ++w) s += red[w];  // the same order in every thread
  __syncthreads();
  return s;
}

__device__ __forceinline__ void lds16(const float* p, float (&v)[BB]) {
#pragma unroll
  for (int c = 0; c < BB; c += 4) {
    const float4 t = *reinterpret_cast<const float4*>(p + c);
    v[c] = t.x;
    v[c + 1] = t.y;
    v[c + 2] = t.z;
    v[c + 3] = t.w;
  }
}

// Swizzled 16-wide rows (G and C): element (j, c) at j 16 + 4 ((c / 4) xor
// ((j / 2) mod 4)) + c mod 4.  Rows are 64 bytes, so without the swizzle the
// 16-byte chunks that 8 consecutive rows read at the same c fall in 2 bank
// groups (4-way conflicts); with it they fall in 8 distinct ones.
__device__ __forceinline__ int swz(int j, int c) { return j * BB + ((((c >> 2) ^ (j >> 1)) & 3) << 2) + (c & 3); }

__device__ __forceinline__ void lds16s(const float* base, int j, float (&v)[BB]) {
  const float* p = base + j * BB;
  const int x = (j >> 1) & 3;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 t = *reinterpret_cast<const float4*>(p + 4 * (q ^ x));
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
}

// ------------------------------------------------------------ Gaussians --
// G(j, c) for c < bb (swizzled rows): column col0 + c of Philox stream 1
// under key (k0, k1); element 4 g + t of a column is Box-Muller output t of
// counter (g, col, 1, 0).  Columns bb .. 15 are zero.
__device__ void gen_gauss(int n, int bb, int col0, uint32_t k0, uint32_t k1, float* sG) {
  const int groups = (n + 3) >> 2;
  for (int e = threadIdx.x; e < groups * BB; e += BT) {
    const int g = e / BB, c = e % BB;
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (c < bb) {
      const Philox4 w = philox4x32_10((uint32_t)g, (uint32_t)(col0 + c), 1u, 0u, k0, k1);
      box_muller_f32(w.x[0], w.x[1], z[0], z[1]);
      box_muller_f32(w.x[2], w.x[3], z[2], z[3]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (4 * g + t < n) sG[swz(4 * g + t, c)] = z[t];
  }
  __syncthreads();
}

// ------------------------------------------------- warp reduce-scatter --
// Sums v[0..63] over the 32 lanes of a warp; afterwards lane l holds the
// totals of indices scatter_index64(l) and scatter_index64(l) + 1 in v[0] and
// v[1].  At partner offset o the lane keeps the upper half of its values if
// (lane & o) is set, else the lower half, and adds the partner's copy of it.
__device__ __forceinline__ void warp_reduce_scatter64(float (&v)[64]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int o = 16 >> s;
    const int half = 32 >> s;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float send = up ? v[k] : v[k + half];
      const float keep = up ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}
// Lane bits 16, 8, 4, 2, 1 chose index bits 32, 16, 8, 4, 2.
__device__ __forceinline__ int scatter_index64(int lane) {
  return ((lane >> 4) & 1) * 32 + ((lane >> 3) & 1) * 16 + ((lane >> 2) & 1) * 8 + ((lane >> 1) & 1) * 4 +
         (lane & 1) * 2;
}

// ------------------------------------------------------- row-owned pass --
// Warp w takes row groups of 4 rows, lanes take columns lane, lane + 32, ...
// For every element:
//   a = src(i, j) [- sum_c q(i, c) C(c, j)]        (UPD; q = sQ rows, C = sC)
//   dst(i, j) = a                                  (UPD)
//   norm += a^2
//   y(i, c) += a G(j, c)                           (AG)
// y overwrites the rows of sQ the warp owns, after their q has been read.
// Returns ||a||_F^2 (binary64; the same value in every thread).
// One column j of a row-owned pass over the warp's 4 rows (rows valid): with
// UPD, a(r) -= Q_new(r, :) . C(:, j), stored; then ||a||^2 and y(r, :) +=
// a(r) G(j, :).  Rows past `rows` hold zeros and stay zero (selects, not
// branches, so the four dependent chains interleave).
template <bool UPD, bool AG>
__device__ __forceinline__ void row_col(const float (&ain)[4], int j, int rows, int n, const float (&q)[4][BB],
                                        const float* sC, const float* sG, float* d0, float& nrm, float (&y)[64]) {
  float a[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) a[r] = ain[r];
  if (UPD) {
    float cj[BB];
    lds16s(sC, j, cj);
    float s[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      s[r] = 0.f;
#pragma unroll
      for (int c = 0; c < BB; ++c) s[r] = fmaf(q[r][c], cj[c], s[r]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      a[r] = r < rows ? a[r] - s[r] : 0.f;
      if (r < rows) d0[(size_t)r * n + j] = a[r];
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) nrm = fmaf(a[r], a[r], nrm);
  if (AG) {
    float g[BB];
    lds16s(sG, j, g);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < BB; ++c) y[r * BB + c] = fmaf(a[r], g[c], y[r * BB + c]);
  }
}

template <bool UPD, bool AG, int PD>
__device__ double pass_rows(int m, int n, const float* src, int lds, float* dst, float* sQ, const float* sC,
                            const float* sG, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double norm = 0.0;
  for (int i0 = 4 * warp; i0 < m; i0 += 4 * BW) {
    const int rows = min(4, m - i0);
    float q[4][BB];
    if (UPD) {
#pragma unroll
      for (int r = 0; r < 4; ++r) lds16(sQ + min(i0 + r, m - 1) * BB, q[r]);
    }
    float y[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) y[k] = 0.f;
    float nrm = 0.f;
    const float* s0 = src + (size_t)i0 * lds;
    float* d0 = UPD ? dst + (size_t)i0 * n : nullptr;
    // double-buffered loads: the next PD columns' values are loaded while
    // the current PD are processed
    float nb[PD][4];
#pragma unroll
    for (int d = 0; d < PD; ++d) {
      const int j = lane + 32 * d;
#pragma unroll
      for (int r = 0; r < 4; ++r) nb[d][r] = (r < rows && j < n) ? s0[(size_t)r * lds + j] : 0.f;
    }
    for (int j0 = lane; j0 < n; j0 += 32 * PD) {
      float cur[PD][4];
#pragma unroll
      for (int d = 0; d < PD; ++d)
#pragma unroll
        for (int r = 0; r < 4; ++r) cur[d][r] = nb[d][r];
      if (j0 + 32 * PD < n) {
#pragma unroll
        for (int d = 0; d < PD; ++d) {
          const int jn = j0 + 32 * (PD + d);
#pragma unroll
          for (int r = 0; r < 4; ++r) nb[d][r] = (r < rows && jn < n) ? s0[(size_t)r * lds + jn] : 0.f;
        }
      }
      if ((j0 - lane) + 32 * PD <= n) {
        // a full batch of columns: no branches between them
#pragma unroll
        for (int d = 0; d < PD; ++d)
          row_col<UPD, AG>(cur[d], j0 + 32 * d, rows, n, q, sC, sG, d0, nrm, y);
      } else {
#pragma unroll
        for (int d = 0; d < PD; ++d) {
          const int j = j0 + 32 * d;
          if (j < n) row_col<UPD, AG>(cur[d], j, rows, n, q, sC, sG, d0, nrm, y);
        }
      }
    }
    norm += (double)nrm;
    if (AG) {
      warp_reduce_scatter64(y);
      const int idx = scatter_index64(lane);  // idx and idx + 1 lie in one row
      const int r = idx / BB, c = idx % BB;
      __syncwarp();
      if (r < rows) {
        sQ[(i0 + r) * BB + c] = y[0];
        sQ[(i0 + r) * BB + c + 1] = y[1];
      }
    }
  }
  return block_sum_f64(norm, red);
}

// ---------------------------------------------------- column-owned passes --
// The CTA is split into `groups` row groups of `ncol` threads (ncol = 32, 64,
// 128 or 256, groups = 256 / ncol); thread tj of group g owns column j0 + tj
// of each column chunk and rows g, g + groups, ...  The split is the one with
// the fewest row visits per thread, ceil(n / ncol) ceil(m / groups), plus
// the cost of a partial-sum exchange per chunk when groups > 1.
struct ColSplit {
  int ncol, groups;
};
__device__ __forceinline__ ColSplit col_split(int m, int n) {
  ColSplit best{BT, 1};
  int bc = 0x7fffffff;
  for (int ncol = BT; ncol >= 32; ncol >>= 1) {
    const int groups = BT / ncol;
    const int cost = ((n + ncol - 1) / ncol) * ((m + groups - 1) / groups + (groups > 1 ? 24 : 0));
    if (cost < bc) {
      bc = cost;
      best = ColSplit{ncol, groups};
    }
  }
  return best;
}

// UPD = false (pass C):  C(j, c) = sum_i Q_new(i, c) src(i, j)
// UPD = true  (pass U1): with C1 = C on entry,
//     dst(i, j) = src(i, j) - sum_c Q_new(i, c) C1(c, j),
//     C(j, c)   = sum_i Q_new(i, c) dst(i, j)                  (C2)
//     Bt[j][k0 + c] = C1(c, j) + C2(c, j)   for c < bb
// C lives in sC (swizzled rows).  Binary32 sums over CHUNK rows are folded
// into binary64; row-group partial sums meet in `part` (binary64, in the sG
// region).  Each thread keeps PF rows' loads in flight; PF changes only the
// load schedule, never the order of the arithmetic.
// One row of a column-owned pass: with UPD, a -= Q_new(i, :) . C1(:, j) and
// the result stored; then acc(c) += Q_new(i, c) a.
template <bool UPD>
__device__ __forceinline__ void col_row(float av, int i, int n, int j, const float* sQ, const float (&c1)[BB],
                                        float* dst, float (&acc)[BB]) {
  float qi[BB];
  lds16(sQ + i * BB, qi);
  if (UPD) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < BB; ++c) s = fmaf(qi[c], c1[c], s);
    av -= s;
    dst[(size_t)i * n + j] = av;
  }
#pragma unroll
  for (int c = 0; c < BB; ++c) acc[c] = fmaf(qi[c], av, acc[c]);
}

template <bool UPD, int PF>
__device__ void pass_cols(int m, int n, const float* src, int lds, float* dst, const float* sQ, float* sC,
                          double* part, float* Bt, int k0, int bb) {
  static_assert(CHUNK % PF == 0, "the fold points must fall on batch boundaries");
  const ColSplit cs = col_split(m, n);
  const int g = threadIdx.x / cs.ncol, tj = threadIdx.x % cs.ncol;
  const int G = cs.groups;
  for (int j0 = 0; j0 < n; j0 += cs.ncol) {
    const int j = j0 + tj;
    const bool live = j < n;
    float c1[BB];
    if (UPD) {
      if (live) lds16s(sC, j, c1);
      else {
#pragma unroll
        for (int c = 0; c < BB; ++c) c1[c] = 0.f;
      }
    }
    double acc64[BB];
    float acc[BB];
#pragma unroll
    for (int c = 0; c < BB; ++c) {
      acc64[c] = 0.0;
      acc[c] = 0.f;
    }
    if (live) {
      int cnt = 0;
      const float* sp = src + j;
      // double-buffered loads: the next PF rows are loaded while the current
      // PF are processed
      float nb[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int i = g + u * G;
        nb[u] = i < m ? sp[(size_t)i * lds] : 0.f;
      }
      for (int i0 = g; i0 < m; i0 += PF * G) {
        float cur[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) cur[u] = nb[u];
        if (i0 + PF * G < m) {
#pragma unroll
          for (int u = 0; u < PF; ++u) {
            const int i = i0 + (PF + u) * G;
            nb[u] = i < m ? sp[(size_t)i * lds] : 0.f;
          }
        }
        if (i0 + (PF - 1) * G < m) {
          // a full batch: no branch between its rows, so their dependent
          // chains interleave; the binary64 fold comes at batch granularity
          // (PF divides CHUNK: the fold points are the same rows)
#pragma unroll
          for (int u = 0; u < PF; ++u) col_row<UPD>(cur[u], i0 + u * G, n, j, sQ, c1, dst, acc);
          cnt += PF;
          if (cnt == CHUNK) {
#pragma unroll
            for (int c = 0; c < BB; ++c) {
              acc64[c] += (double)acc[c];
              acc[c] = 0.f;
            }
            cnt = 0;
          }
        } else {
#pragma unroll
          for (int u = 0; u < PF; ++u) {
            const int i = i0 + u * G;
            if (i < m) {
              col_row<UPD>(cur[u], i, n, j, sQ, c1, dst, acc);
              if (++cnt == CHUNK) {
#pragma unroll
                for (int c = 0; c < BB; ++c) {
                  acc64[c] += (double)acc[c];
                  acc[c] = 0.f;
                }
                cnt = 0;
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < BB; ++c) acc64[c] += (double)acc[c];
    if (G > 1) {
      __syncthreads();  // the sG region is free for the partials; earlier chunks' sums are read
      if (live) {
#pragma unroll
        for (int c = 0; c < BB; ++c) part[((size_t)g * cs.ncol + tj) * BB + c] = acc64[c];
      }
      __syncthreads();
      if (g == 0 && live) {
#pragma unroll
        for (int c = 0; c < BB; ++c) {
          double sum = 0.0;
          for (int h = 0; h < G; ++h) sum += part[((size_t)h * cs.ncol + tj) * BB + c];
          acc64[c] = sum;
        }
      }
    }
    if (g == 0 && live) {
#pragma unroll
      for (int c = 0; c < BB; ++c) sC[swz(j, c)] = (float)acc64[c];
      if (UPD) {
#pragma unroll
        for (int c = 0; c < BB; ++c)
          if (c < bb) Bt[(size_t)j * RMAX + k0 + c] = (float)((double)c1[c] + acc64[c]);
      }
    }
  }
  __syncthreads();
}

// --------------------------------------------------------- small algebra --
// Gram of the rows x l block Y (row stride ldy >= 16, l <= 16, columns l..15
// zero) into g64 (l x l, binary64).  Warp w sums rows w, w + 8, ...; lane
// holds the pairs (lane / 2, 8 (lane % 2) + 0..7); binary32 partials of CHUNK
// rows are folded into binary64.
__device__ void gram16(int rows, int l, const float* Y, int ldy, double* g64, double* wpart) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c1 = lane >> 1, cb = (lane & 1) * 8;
  double acc64[8];
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    acc64[k] = 0.0;
    acc[k] = 0.f;
  }
  int cnt = 0;
  for (int i = warp; i < rows; i += BW) {
    const float a = Y[i * ldy + c1];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = fmaf(a, Y[i * ldy + cb + k], acc[k]);
    if (++cnt == CHUNK) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        acc64[k] += (double)acc[k];
        acc[k] = 0.f;
      }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) wpart[(warp * BB + c1) * BB + cb + k] = acc64[k] + (double)acc[k];
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += BT) {
    const int i = e / l, j = e % l;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < BW; ++w) s += wpart[(w * BB + i) * BB + j];
    g64[e] = s;
  }
  __syncthreads();
}

// Gram of a rows x l block (l <= 64, shared or global memory, row stride
// ldy): one thread per upper-triangle entry; four binary32 partial sums over
// interleaved rows of each CHUNK-row chunk, added in binary32 and folded into
// binary64 per chunk.
__device__ void gram_wide(int rows, int l, const float* Y, int ldy, double* g64) {
  const int nent = l * (l + 1) / 2;
  for (int e = threadIdx.x; e < nent; e += BT) {
    int i = 0, rem = e;
    while (rem >= l - i) {
      rem -= l - i;
      ++i;
    }
    const int j = i + rem;
    double acc = 0.0;
    for (int r0 = 0; r0 < rows; r0 += CHUNK) {
      float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
      const int r1 = min(rows, r0 + CHUNK);
      int r = r0;
      for (; r + 3 < r1; r += 4) {
        const float* y = Y + (size_t)r * ldy;
        p0 = fmaf(y[i], y[j], p0);
        p1 = fmaf(y[ldy + i], y[ldy + j], p1);
        p2 = fmaf(y[2 * ldy + i], y[2 * ldy + j], p2);
        p3 = fmaf(y[3 * ldy + i], y[3 * ldy + j], p3);
      }
      for (; r < r1; ++r) p0 = fmaf(Y[(size_t)r * ldy + i], Y[(size_t)r * ldy + j], p0);
      acc += (double)((p0 + p1) + (p2 + p3));  // one binary64 add per chunk
    }
    g64[i * l + j] = acc;
    g64[j * l + i] = acc;
  }
  __syncthreads();
}

// Cholesky of the unit-diagonal scaling D G D (D = diag(G_ii^-1/2)) by ONE
// warp (no CTA barriers): the binary32 lower factor goes to L (l x l,
// row-major, l <= 64) and D to dinv.  On a non-positive pivot the
// factorization restarts with a diagonal shift (shifted CholeskyQR, Fukaya et
// al. 2020), growing 32x per retry.  Returns false (in lane 0's view and
// every other lane's) if every shift failed; the caller's CTA barrier
// publishes L and dinv.
__device__ bool chol_warp(int l, const double* g64, float* L, float* dinv) {
  const int lane = threadIdx.x & 31;
  const float u = 5.9604644775390625e-08f;
  float shift = 0.f;
  // the scaling d_i = G_ii^-1/2 in binary64 (rounded to binary32), once per
  // diagonal entry: binary64 square roots and divisions run at a small
  // fraction of the binary32 rate on this part
  for (int i = lane; i < l; i += 32) {
    const double gii = g64[i * l + i];
    dinv[i] = gii > 0.0 ? (float)(1.0 / sqrt(gii)) : 0.f;
  }
  __syncwarp();
  for (int attempt = 0; attempt < 6; ++attempt) {
    for (int i = 0; i < l; ++i) {
      const float di = dinv[i];
      const bool pos = g64[i * l + i] > 0.0;
      for (int j = lane; j < l; j += 32) {
        float v = (float)g64[i * l + j] * di * dinv[j];
        if (i == j) v = (pos ? 1.f : 0.f) + shift;
        L[i * l + j] = (i >= j) ? v : 0.f;
      }
    }
    __syncwarp();
    bool ok = true;
    for (int k = 0; k < l; ++k) {
      const float akk = L[k * l + k];  // the same value in every lane
      if (!(akk > 64.f * u) || !isfinite(akk)) {
        ok = false;
        break;
      }
      const float rp = 1.f / sqrtf(akk);
      for (int i = k + 1 + lane; i < l; i += 32) L[i * l + k] *= rp;
      __syncwarp();
      if (lane == 0) L[k * l + k] = akk * rp;
      // trailing update, lane j owning column j: row i of the update reads
      // L(i, k) once for the whole warp and L(i, j) from consecutive banks
      for (int jb = k + 1; jb < l; jb += 32) {
        const int j = jb + lane;
        const bool act = j < l;
        const float ljk = act ? L[j * l + k] : 0.f;
        for (int i = jb; i < l; ++i) {
          const float lik = L[i * l + k];
          if (act && j <= i) L[i * l + j] = fmaf(-lik, ljk, L[i * l + j]);
        }
      }
      __syncwarp();
    }
    if (ok) return true;
    shift = shift == 0.f ? 64.f * 11.f * (float)l * u : shift * 32.f;
  }
  return false;
}

// In place Y <- Y D L^-T (rows x l, row stride ldy): a thread per row.
__device__ void apply_rows(int rows, int l, float* Y, int ldy, const float* L, const float* dinv) {
  for (int r = threadIdx.x; r < rows; r += BT) {
    float* y = Y + (size_t)r * ldy;
    for (int c = 0; c < l; ++c) {
      float s = y[c] * dinv[c];
#pragma unroll 4
      for (int k = 0; k < c; ++k) s = fmaf(-y[k], L[c * l + k], s);
      y[c] = s / L[c * l + c];
    }
  }
  __syncthreads();
}

// LU factorization with partial pivoting of the rows x l block Y (row stride
// ldy, l <= 64), in place and without moving rows: afterwards Y holds L (row
// p_k carries the unit pivot of column k and zeros to its right) and U (l x
// l, row-major, upper) the other factor, Y_in = L U.  A column with no nonzero
// candidate pivot takes the lowest unused row as its unit column of L and a
// zero diagonal in U.  Two CTA barriers per column.
__device__ void lu_rows(int rows, int l, float* Y, int ldy, float* U, unsigned char* used, float* rv, int* ri) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < rows; i += BT) used[i] = 0;
  __syncthreads();
  for (int k = 0; k < l; ++k) {
    // pivot: the largest |Y(i, k)| over unused rows (lowest row on ties)
    float bv = -1.f;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < rows; i += BT) {
      if (used[i]) continue;
      const float a = fabsf(Y[(size_t)i * ldy + k]);
      if (a > bv) {  // rows visited in increasing order: ties keep the lower row
        bv = a;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      rv[warp] = bv;
      ri[warp] = bi;
    }
    __syncthreads();
    float pv = -1.f;
    int p = 0x7fffffff;
#pragma unroll
    for (int w = 0; w < BW; ++w) {
      if (rv[w] > pv || (rv[w] == pv && ri[w] < p)) {
        pv = rv[w];
        p = ri[w];
      }
    }
    // p < rows always: rows >= l and only k < l rows are used
    const float* yp = Y + (size_t)p * ldy;
    const float piv = yp[k];
    for (int j = threadIdx.x; j < l; j += BT) U[k * l + j] = j >= k ? yp[j] : 0.f;
    const float rpiv = piv != 0.f ? 1.f / piv : 0.f;
    if (threadIdx.x == 0) used[p] = 1;  // read again only after the next barrier
    for (int i = threadIdx.x; i < rows; i += BT) {
      if (used[i] || i == p) continue;
      float* yi = Y + (size_t)i * ldy;
      const float lik = yi[k] * rpiv;
      yi[k] = lik;
#pragma unroll 4
      for (int j = k + 1; j < l; ++j) yi[j] = fmaf(-lik, yp[j], yi[j]);
    }
    __syncthreads();
    // row p becomes the unit pivot row of L: it is used, so no later column of
    // this factorization reads it; the final barrier orders it before any use
    for (int j = k + threadIdx.x; j < l; j += BT) Y[(size_t)p * ldy + j] = j == k ? 1.f : 0.f;
  }
  __syncthreads();
}

// Gram of Y (binary32 partials folded into binary64) and its warp Cholesky
// into L, dinv; false (in every thread) if the Cholesky failed.
template <bool GLOBAL>
__device__ bool chol_factor(int rows, int l, const float* Y, int ldy, double* g64, double* wpart, float* L,
                            float* dinv, int* s_flag) {
  if (GLOBAL) gram_wide(rows, l, Y, ldy, g64);
  else gram16(rows, l, Y, ldy, g64, wpart);
  if (threadIdx.x < 32) {
    const bool ok = chol_warp(l, g64, L, dinv);
    if (threadIdx.x == 0) *s_flag = ok ? 0 : 1;
  }
  __syncthreads();
  const int f = *s_flag;
  __syncthreads();
  return f == 0;
}

// Thin QR of the rows x l block Y in place by LU-Cholesky QR (Terao, Ozaki,
// Ogita 2020): Y = L U by lu_rows, then CholeskyQR2 of the well-conditioned
// L (binary32 Gram folded into binary64, warp Cholesky, triangular solve), so
// that Y_in = Q R with R = R2 R1 U.  Holds for any kappa(Y) below the binary32
// limit, where CholeskyQR2 of Y itself would lose orthogonality.  R
// (optional, l x l row-major upper) needs Rt and Ra as scratch.  Returns false
// if the Cholesky failed after every shift.
template <bool GLOBAL>
__device__ bool lu_cholqr2(int rows, int l, float* Y, int ldy, double* g64, double* wpart, float* L, float* dinv,
                           float* Ulu, float* R, float* Rt, unsigned char* used, float* rv, int* ri, int* s_flag) {
  lu_rows(rows, l, Y, ldy, Ulu, used, rv, ri);
  if (R) {
    for (int e = threadIdx.x; e < l * l; e += BT) R[e] = Ulu[e];
  }
  for (int pass = 0; pass < 2; ++pass) {
    if (!chol_factor<GLOBAL>(rows, l, Y, ldy, g64, wpart, L, dinv, s_flag)) return false;
    if (R) {
      // R <- (L^T D^-1) R, both upper: a thread per entry into the scratch
      // Ulu (free once the LU's U was copied to R), then copied back
      for (int e = threadIdx.x; e < l * l; e += BT) {
        const int i = e / l, j = e % l;
        Rt[e] = (i <= j && dinv[j] > 0.f) ? L[j * l + i] / dinv[j] : 0.f;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < l * l; e += BT) {
        const int i = e / l, j = e % l;
        float s = 0.f;
        for (int k = i; k <= j; ++k) s = fmaf(Rt[i * l + k], R[k * l + j], s);
        Ulu[e] = s;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < l * l; e += BT) R[e] = Ulu[e];
    }
    apply_rows(rows, l, Y, ldy, L, dinv);
  }
  return true;
}

// Y -= Q (Q^T Y) for the rows x 16 block Y in shared memory (row stride ldy,
// odd, so that a thread per row reads conflict-free) and the rank columns of
// Q stored transposed (Qt[k][i], row stride NMAX); P (rank x 16, 16-byte
// aligned) is scratch.  A warp per k forms P, a thread per row applies it.
__device__ void project_out(int rows, int rank, const float* Qt, float* Y, int ldy, float* P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < rank; k += BW) {
    float acc[BB];
#pragma unroll
    for (int c = 0; c < BB; ++c) acc[c] = 0.f;
    const float* qk = Qt + (size_t)k * NMAX;
#pragma unroll 2
    for (int i = lane; i < rows; i += 32) {
      const float qv = qk[i];
      const float* yi = Y + i * ldy;
#pragma unroll
      for (int c = 0; c < BB; ++c) acc[c] = fmaf(qv, yi[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < BB; ++c) {
      float v = acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) P[k * BB + c] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < rows; i += BT) {
    float acc[BB];
#pragma unroll
    for (int c = 0; c < BB; ++c) acc[c] = 0.f;
#pragma unroll 4
    for (int k = 0; k < rank; ++k) {
      const float qv = Qt[(size_t)k * NMAX + i];
      float pk[BB];
      lds16(P + k * BB, pk);
#pragma unroll
      for (int c = 0; c < BB; ++c) acc[c] = fmaf(qv, pk[c], acc[c]);
    }
    float* yi = Y + i * ldy;
#pragma unroll
    for (int c = 0; c < BB; ++c) yi[c] -= acc[c];
  }
  __syncthreads();
}

// One-sided Jacobi on the columns of X (l x l, column c at X + c l),
// accumulating the rotations in J (same layout, identity on entry).  Round-
// robin pair order, one half-warp per pair (all pairs of a step at once for
// l <= 32), at most 30 sweeps.
__device__ void jacobi_cols(int l, float* X, float* J, int* s_cnt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, hl = lane & 15;
  const int P = (l & 1) ? l + 1 : l;
  const float tol = 4.f * (float)l * 5.9604644775390625e-08f;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (threadIdx.x == 0) *s_cnt = 0;
    __syncthreads();
    for (int step = 0; step < P - 1; ++step) {
      // the loop is uniform over the warp: both halves run every round and
      // take part in every shuffle
      for (int base = 2 * warp; base < P / 2; base += 2 * BW) {
        const int pr = base + half;
        int ia = 0, ib = 0;
        if (pr < P / 2) {
          ia = pr == 0 ? 0 : 1 + (pr - 1 + step) % (P - 1);
          const int qq = P - 1 - pr;
          ib = 1 + (qq - 1 + step) % (P - 1);
        }
        const bool live = pr < P / 2 && ia < l && ib < l;
        float* xa = X + ia * l;
        float* xb = X + ib * l;
        float al = 0.f, be = 0.f, ga = 0.f;
        if (live) {
          for (int i = hl; i < l; i += 16) {
            const float a = xa[i], b = xb[i];
            al = fmaf(a, a, al);
            be = fmaf(b, b, be);
            ga = fmaf(a, b, ga);
          }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (live && ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be)) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
          const float cs = 1.f / sqrtf(fmaf(t, t, 1.f)), sn = cs * t;
          float* ja = J + ia * l;
          float* jb = J + ib * l;
          for (int i = hl; i < l; i += 16) {
            const float a = xa[i], b = xb[i];
            xa[i] = cs * a - sn * b;
            xb[i] = sn * a + cs * b;
            const float p = ja[i], w = jb[i];
            ja[i] = cs * p - sn * w;
            jb[i] = sn * p + cs * w;
          }
          if (hl == 0) atomicAdd(s_cnt, 1);
        }
      }
      __syncthreads();
    }
    const int cnt = *s_cnt;
    __syncthreads();
    if (cnt == 0) break;
  }
}

// ------------------------------------------------------------- a problem --
// CTA-shared scalars and small arrays (static shared memory)
struct Work {
  double* red;          // BW binary64 partial sums
  float* rv;            // BW pivot magnitudes
  int* ri;              // BW pivot rows
  int* flag;            // one int
  unsigned char* used;  // NMAX row flags of the LU
};

template <int PF, int PD>
__device__ void solve_one(const Prob& P, int p, uint64_t seed, double tol, int R, int b, float* base, float* sm,
                          const Work& W, int* rank_out, double* err_out, int* status_out, DevStatus* st) {
  double* red = W.red;
  const int m = P.m, n = P.n, tid = threadIdx.x;
  float* Aj = base;
  float* Qt = Aj + (size_t)NMAX * NMAX;
  float* Bt = Qt + (size_t)RMAX * NMAX;
  float* sQ = sm + SQ_OFF;
  float* sG = sm + SG_OFF;
  float* sC = sm + SC_OFF;
  float* sP = sm + SP_OFF;
  double* g16 = reinterpret_cast<double*>(sm + SS_OFF);  // 16 x 16 binary64
  float* sL = sm + SS_OFF + 2 * BB * BB;
  float* sU = sL + BB * BB;
  float* sDinv = sU + BB * BB;
  double* wpart = reinterpret_cast<double*>(sG);  // 8 x 16 x 16 binary64 Gram partials
  float* Yo = sC;                                 // m x YLD copy of Y during the orthonormalization
  float* sPj = sG + 2 * BW * BB * BB;             // rank x 16 projection scratch, after wpart
  const int rmax = min(R, min(m, n));
  const uint64_t key = seed + (uint64_t)p;
  const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
  int status = RSVD_OK;

  // first pass: Y = A G_0 and ||A||_F^2
  int bb = min(b, rmax);
  gen_gauss(n, bb, 0, k0, k1, sG);
  const double a2 = pass_rows<false, true, PD>(m, n, P.A, P.lda, nullptr, sQ, sC, sG, red);
  const double eps2 = tol * tol * a2;
  double r2 = a2;
  const float* src = P.A;
  int lds = P.lda;
  int rank = 0, t = 0;
  while (!(r2 <= eps2) && rank < rmax) {
    if (!isfinite(r2)) {
      status = RSVD_E_NONFINITE;
      break;
    }
    bb = min(b, rmax - rank);
    // the orthonormalization works on a copy of Y with the odd row stride
    // YLD (in the sC and sP regions, free until the next pass): every thread-
    // per-row walk below is then free of bank conflicts
    for (int e = tid; e < m * BB; e += BT) Yo[(e / BB) * YLD + e % BB] = sQ[e];
    __syncthreads();
    if (rank > 0) project_out(m, rank, Qt, Yo, YLD, sPj);
    // Q_new = CholeskyQR2(Y)
    if (!lu_cholqr2<false>(m, bb, Yo, YLD, g16, wpart, sL, sDinv, sU, nullptr, nullptr, W.used, W.rv, W.ri,
                           W.flag)) {
      status = RSVD_E_BREAKDOWN;
      break;
    }
    if (rank > 0) {
      // Q_new = qr(Y R^-1) amplifies what round-off left of span(Q) in Y by up
      // to kappa(Y): project once more and renormalize (block Gram-Schmidt,
      // twice), so that Q^T Q_new stays at the binary32 round-off level
      for (int e = tid; e < m * BB; e += BT)
        if (e % BB >= bb) Yo[(e / BB) * YLD + e % BB] = 0.f;
      __syncthreads();
      project_out(m, rank, Qt, Yo, YLD, sPj);
      if (!chol_factor<false>(m, bb, Yo, YLD, g16, wpart, sL, sDinv, W.flag)) {
        status = RSVD_E_BREAKDOWN;
        break;
      }
      apply_rows(m, bb, Yo, YLD, sL, sDinv);
    }
    for (int e = tid; e < m * BB; e += BT) {
      const int i = e / BB, c = e % BB;
      const float v = c < bb ? Yo[i * YLD + c] : 0.f;
      sQ[e] = v;
      if (c < bb) Qt[(size_t)(rank + c) * NMAX + i] = v;
    }
    __syncthreads();
    pass_cols<false, PF>(m, n, src, lds, nullptr, sQ, sC, reinterpret_cast<double*>(sG), Bt, rank, bb);
    pass_cols<true, PF>(m, n, src, lds, Aj, sQ, sC, reinterpret_cast<double*>(sG), Bt, rank, bb);
    src = Aj;
    lds = n;
    const int bnext = min(b, rmax - rank - bb);
    if (bnext > 0) {
      gen_gauss(n, bnext, (t + 1) * b, k0, k1, sG);
      r2 = pass_rows<true, true, PD>(m, n, Aj, n, Aj, sQ, sC, sG, red);
    } else {
      r2 = pass_rows<true, false, PD>(m, n, Aj, n, Aj, sQ, sC, sG, red);
    }
    rank += bb;
    ++t;
  }
  if (status == RSVD_OK && !isfinite(r2)) status = RSVD_E_NONFINITE;
  if (status == RSVD_OK && !(r2 <= eps2)) status = RSVD_E_NOT_CONVERGED;
  __syncthreads();

  // Stage B on A ~= Q B with l = rank: B^T = Q_B R_B (LU-CholeskyQR2), one-
  // sided Jacobi on X = R_B^T (X J = W), V = Q_B J, U = Q W / sigma.  B^T is
  // copied into shared memory (odd row stride) when it fits beside the
  // small l x l arrays, else the factorization runs on it in place in the
  // CTA's workspace slot.
  const int l = rank;
  const bool have = l > 0 && status != RSVD_E_BREAKDOWN && status != RSVD_E_NONFINITE;
  bool ok = true;
  if (have) {
    const int LP = (l + 31) / 32 * 32;  // row stride of the permuted lift operands
    const int ldb = l | 1;
    const bool in_smem = (size_t)n * ldb + 8 * l * l + 2 * l * LP + 6 * l + 64 <= (size_t)SMEM_FLOATS;
    float* Y;
    int ldy;
    double* g64;
    float *Xc, *Jm, *L, *Rb, *Rt, *Ulu, *Jp, *Xp, *dv, *sig, *flip;
    int* perm;
    unsigned long long* keys;
    if (in_smem) {
      size_t off = 0;
      auto take = [&](size_t nf) {
        float* p = sm + off;
        off += (nf + 3) & ~(size_t)3;
        return p;
      };
      Y = take((size_t)n * ldb);
      ldy = ldb;
      g64 = reinterpret_cast<double*>(take((size_t)2 * l * l));
      Xc = take((size_t)l * l);
      Jm = take((size_t)l * l);
      L = take((size_t)l * l);
      Rb = take((size_t)l * l);
      Rt = take((size_t)l * l);
      Ulu = take((size_t)l * l);
      Jp = take((size_t)l * LP);
      Xp = take((size_t)l * LP);
      dv = take(l);
      sig = take(l);
      flip = take(l);
      perm = reinterpret_cast<int*>(take(l));
      keys = reinterpret_cast<unsigned long long*>(take((size_t)2 * l));
      for (int e = tid; e < n * l; e += BT) {
        const int j = e / l, c = e % l;
        Y[(size_t)j * ldb + c] = Bt[(size_t)j * RMAX + c];
      }
      __syncthreads();
    } else {
      Y = Bt;
      ldy = RMAX;
      g64 = reinterpret_cast<double*>(sG);  // l x l binary64
      Xc = sG + 2 * RMAX * RMAX;            // l x l, column c at Xc + c l
      Jm = Xc + RMAX * RMAX;                // l x l
      L = sC;                               // l x l
      Rb = L + RMAX * RMAX;                 // R_B
      Rt = Rb + RMAX * RMAX;                // scratch
      Ulu = Rt + RMAX * RMAX;               // U of the LU
      Jp = sQ;                              // l x LP
      Xp = sQ + RMAX * RMAX;                // l x LP
      dv = sP;
      sig = dv + RMAX;
      flip = sig + RMAX;
      perm = reinterpret_cast<int*>(flip + RMAX);
      keys = reinterpret_cast<unsigned long long*>(flip + 2 * RMAX);
    }
    ok = lu_cholqr2<true>(n, l, Y, ldy, g64, nullptr, L, dv, Ulu, Rb, Rt, W.used, W.rv, W.ri, W.flag);
    if (ok) {
      for (int e = tid; e < l * l; e += BT) {  // X = R_B^T: column c is row c of R_B
        const int c = e / l, r = e % l;
        Xc[e] = Rb[c * l + r];
        Jm[e] = c == r ? 1.f : 0.f;
      }
      __syncthreads();
      jacobi_cols(l, Xc, Jm, W.flag);
      for (int c = tid; c < l; c += BT) {
        float sq = 0.f;
        for (int r = 0; r < l; ++r) sq = fmaf(Xc[c * l + r], Xc[c * l + r], sq);
        sig[c] = sqrtf(sq);
      }
      __syncthreads();
      for (int c = tid; c < l; c += BT) {  // descending; ties by index
        int rk = 0;
        for (int c2 = 0; c2 < l; ++c2) rk += (sig[c2] > sig[c]) || (sig[c2] == sig[c] && c2 < c);
        perm[rk] = c;
        keys[c] = 0ull;
      }
      __syncthreads();
      // Jp(c, k) = J(c, perm k), zero for k >= l
      for (int e = tid; e < l * LP; e += BT) {
        const int c = e / LP, k = e % LP;
        Jp[e] = k < l ? Jm[perm[k] * l + c] : 0.f;
      }
      __syncthreads();
      // V = Q_B Jp, a thread per row and 32 columns; the largest |V(:, k)|
      // (lowest row on ties) is recorded as a 64-bit key per column
      const bool vec4 = (R % 4) == 0 && ((reinterpret_cast<uintptr_t>(P.V) | reinterpret_cast<uintptr_t>(P.U)) & 15) == 0;
      for (int k0 = 0; k0 < l; k0 += 32) {
        for (int j = tid; j < n; j += BT) {
          float acc[32];
#pragma unroll
          for (int kk = 0; kk < 32; ++kk) acc[kk] = 0.f;
          const float* yr = Y + (size_t)j * ldy;
#pragma unroll 2
          for (int c = 0; c < l; ++c) {
            const float yv = yr[c];
            const float4* jp = reinterpret_cast<const float4*>(Jp + c * LP + k0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 t = jp[q];
              acc[4 * q] = fmaf(yv, t.x, acc[4 * q]);
              acc[4 * q + 1] = fmaf(yv, t.y, acc[4 * q + 1]);
              acc[4 * q + 2] = fmaf(yv, t.z, acc[4 * q + 2]);
              acc[4 * q + 3] = fmaf(yv, t.w, acc[4 * q + 3]);
            }
          }
          float* vr = P.V + (size_t)j * R + k0;
          const int kn = min(32, l - k0);
          if (vec4 && kn == 32) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              reinterpret_cast<float4*>(vr)[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
          } else {
#pragma unroll
            for (int kk = 0; kk < 32; ++kk)
              if (kk < kn) vr[kk] = acc[kk];
          }
#pragma unroll
          for (int kk = 0; kk < 32; ++kk)
            if (kk < kn) {
              const unsigned long long key = ((unsigned long long)__float_as_uint(fabsf(acc[kk])) << 32) |
                                             (unsigned long long)(0xffffffffu - (unsigned)j);
              atomicMax(&keys[k0 + kk], key);
            }
        }
      }
      __syncthreads();
      for (int k = tid; k < l; k += BT) {
        const int jb = (int)(0xffffffffu - (unsigned)(keys[k] & 0xffffffffull));
        flip[k] = (jb < n && P.V[(size_t)jb * R + k] < 0.f) ? -1.f : 1.f;
        P.D[k] = (double)sig[perm[k]];
      }
      __syncthreads();
      for (int e = tid; e < n * l; e += BT) {
        const int j = e / l, k = e % l;
        if (flip[k] < 0.f) P.V[(size_t)j * R + k] = -P.V[(size_t)j * R + k];
      }
      // Xp(c, k) = flip_k W(c, perm k) / sigma_perm k, zero for k >= l
      for (int e = tid; e < l * LP; e += BT) {
        const int c = e / LP, k = e % LP;
        float v = 0.f;
        if (k < l) {
          const int sc = perm[k];
          const float inv = sig[sc] > 0.f ? 1.f / sig[sc] : 0.f;
          v = flip[k] * (Xc[sc * l + c] * inv);
        }
        Xp[e] = v;
      }
      __syncthreads();
      // U = Q Xp, a thread per row and 32 columns (Q^T rows read coalesced)
      for (int k0 = 0; k0 < l; k0 += 32) {
        for (int i = tid; i < m; i += BT) {
          float acc[32];
#pragma unroll
          for (int kk = 0; kk < 32; ++kk) acc[kk] = 0.f;
#pragma unroll 4
          for (int c = 0; c < l; ++c) {
            const float qv = Qt[(size_t)c * NMAX + i];
            const float4* xp = reinterpret_cast<const float4*>(Xp + c * LP + k0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 t = xp[q];
              acc[4 * q] = fmaf(qv, t.x, acc[4 * q]);
              acc[4 * q + 1] = fmaf(qv, t.y, acc[4 * q + 1]);
              acc[4 * q + 2] = fmaf(qv, t.z, acc[4 * q + 2]);
              acc[4 * q + 3] = fmaf(qv, t.w, acc[4 * q + 3]);
            }
          }
          float* ur = P.U + (size_t)i * R + k0;
          const int kn = min(32, l - k0);
          if (vec4 && kn == 32) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              reinterpret_cast<float4*>(ur)[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
          } else {
#pragma unroll
            for (int kk = 0; kk < 32; ++kk)
              if (kk < kn) ur[kk] = acc[kk];
          }
        }
      }
    } else {
      status = RSVD_E_BREAKDOWN;
    }
  }
  __syncthreads();
  // zero the triplets past the rank (all of them when nothing was factored)
  const int lz = (have && ok) ? l : 0;
  for (int k = lz + tid; k < R; k += BT) P.D[k] = 0.0;
  if (lz < R) {
    const int w = R - lz;
    for (int e = tid; e < m * w; e += BT) P.U[(size_t)(e / w) * R + lz + e % w] = 0.f;
    for (int e = tid; e < n * w; e += BT) P.V[(size_t)(e / w) * R + lz + e % w] = 0.f;
  }
  if (tid == 0) {
    if (rank_out) rank_out[p] = lz;
    if (err_out) err_out[p] = a2 > 0.0 ? sqrt(fmax(r2, 0.0) / a2) : 0.0;
    if (status_out) status_out[p] = status;
    if (status != RSVD_OK) set_status(st, status);
  }
  __syncthreads();
}

template <int PF, int PD>
__global__ void __launch_bounds__(BT, 1)
    batched_kernel(int count, const int* __restrict__ order, const int* __restrict__ pm, const int* __restrict__ pn,
                   const int* __restrict__ plda, const float* const* __restrict__ pA, float* const* __restrict__ pU,
                   double* const* __restrict__ pD, float* const* __restrict__ pV, int R, int b, uint64_t seed,
                   double tol, int* counter, float* slots, int* rank_out, double* err_out, int* status_out,
                   DevStatus* st) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[BW];
  __shared__ float rv[BW];
  __shared__ int ri[BW];
  __shared__ int s_idx, s_flag;
  __shared__ unsigned char used[NMAX];
  const Work W{red, rv, ri, &s_flag, used};
  float* base = slots + (size_t)blockIdx.x * SLOT_FLOATS;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= count) break;
    const int p = order[idx];
    Prob P;
    P.m = pm[p];
    P.n = pn[p];
    P.lda = plda[p];
    P.A = pA[p];
    P.U = pU[p];
    P.D = pD[p];
    P.V = pV[p];
    const bool valid = P.m >= 1 && P.n >= 1 && P.m <= NMAX && P.n <= NMAX && P.lda >= P.n && P.A && P.U && P.D &&
                       P.V;
    if (!valid) {
      if (threadIdx.x == 0) {
        if (rank_out) rank_out[p] = 0;
        if (err_out) err_out[p] = 0.0;
        if (status_out) status_out[p] = RSVD_E_INVALID;
        set_status(st, RSVD_E_INVALID);
      }
      continue;
    }
    solve_one<PF, PD>(P, p, seed, tol, R, b, base, sm, W, rank_out, err_out, status_out, st);
  }
}

// order[r] = the problem of rank r in descending m n (ties: lower index
// first); problems with invalid sizes sort last.
__device__ __forceinline__ long long size_key(const int* pm, const int* pn, int q) {
  const int m = pm[q], n = pn[q];
  return (m >= 1 && n >= 1 && m <= NMAX && n <= NMAX) ? (long long)m * n : 0;
}

__global__ void batched_order_kernel(int count, const int* __restrict__ pm, const int* __restrict__ pn,
                                     int* __restrict__ order) {
  __shared__ long long keys[BT];
  const int p = blockIdx.x * BT + threadIdx.x;
  const long long kp = p < count ? size_key(pm, pn, p) : -1;
  int rk = 0;
  for (int t0 = 0; t0 < count; t0 += BT) {
    __syncthreads();
    const int q = t0 + threadIdx.x;
    keys[threadIdx.x] = q < count ? size_key(pm, pn, q) : -1;
    __syncthreads();
    const int lim = min(BT, count - t0);
    for (int u = 0; u < lim; ++u) {
      const long long k = keys[u];
      rk += (k > kp) || (k == kp && t0 + u < p);
    }
  }
  if (p < count) order[rk] = p;
}

// The variants differ only in how far ahead each thread loads (PF rows in the
// column-owned passes, PD columns in the row-owned ones); the arithmetic and
// its order are the same in all of them, so their outputs are bit-identical.
struct Variant {
  int pf, pd;
  void (*fn)(int, const int*, const int*, const int*, const int*, const float* const*, float* const*,
             double* const*, float* const*, int, int, uint64_t, double, int*, float*, int*, double*, int*,
             DevStatus*);
};
const Variant kVariants[] = {{8, 1, batched_kernel<8, 1>},
                             {8, 2, batched_kernel<8, 2>},
                             {16, 2, batched_kernel<16, 2>},
                             {32, 2, batched_kernel<32, 2>}};
constexpr int NVAR = sizeof(kVariants) / sizeof(kVariants[0]);
constexpr int DEFAULT_VARIANT = 2;

}  // namespace

int batched_variants() { return NVAR; }
int batched_default_variant() { return DEFAULT_VARIANT; }
void batched_variant_info(int v, int* pf, int* pd) {
  *pf = kVariants[v].pf;
  *pd = kVariants[v].pd;
}

int batched_max_rank() { return RMAX; }
int batched_max_dim() { return NMAX; }
int batched_max_block() { return BB; }

size_t batched_workspace_bytes(int count, int ctas) {
  Carver c(nullptr);
  c.take<DevStatus>(1);
  c.take<int>(1);              // queue counter
  c.take<int>((size_t)count);  // order
  c.take<float>(SLOT_FLOATS * (size_t)ctas);
  return c.size();
}

cudaError_t launch_batched(int count, const int* m, const int* n, const int* lda, const float* const* A,
                           float* const* U, double* const* D, float* const* V, int R, int b, uint64_t seed,
                           double tol, int* rank_out, double* err_out, int* status_out, void* ws, int ctas,
                           cudaStream_t s, int variant) {
  if (variant < 0 || variant >= NVAR) variant = DEFAULT_VARIANT;
  Carver c(ws);
  DevStatus* st = c.take<DevStatus>(1);
  int* counter = c.take<int>(1);
  int* order = c.take<int>((size_t)count);
  float* slots = c.take<float>(SLOT_FLOATS * (size_t)ctas);
  cudaError_t e = cudaMemsetAsync(st, 0, 512, s);  // the status block and the counter (two 256-byte slices)
  if (e != cudaSuccess) return e;
  batched_order_kernel<<<(count + BT - 1) / BT, BT, 0, s>>>(count, m, n, order);
  note_launch();
  // the shared-memory opt-in is set once per device and variant, outside any
  // later graph capture
  static std::atomic<unsigned long long> smem_set[NVAR];
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(smem_set[variant].load() & bit)) {
    e = cudaFuncSetAttribute(kVariants[variant].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    smem_set[variant].fetch_or(bit);
  }
  const int grid = count < ctas ? count : ctas;
  kVariants[variant].fn<<<grid, BT, SMEM_BYTES, s>>>(count, order, m, n, lda, A, U, D, V, R, b, seed, tol, counter,
                                                     slots, rank_out, err_out, status_out, st);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rsvd
