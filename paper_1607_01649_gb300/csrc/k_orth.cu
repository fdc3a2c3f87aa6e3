// Unpivoted orthonormalization "orth" (Sec. 2.3), as CholeskyQR2 with an
// optional shifted first pass (shifted CholeskyQR3: Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa, SISC 42 (2020)).
//
// One pass on a rows x l block Y (row-major, updated in place):
//   1. G = Y^T Y                    (gram_partial + gram_reduce; sums carried
//                                     beyond binary32 precision)
//   2. G = D Gt D, Gt = Lt Lt^T      (chol: unit-diagonal scaling in binary64,
//                                     Cholesky of Gt (+ s I when needed))
//   3. Y <- Y D^-1 Lt^-T             (apply: blocked triangular solve,
//                                     64-row stripes)
// so Y = Q R with R = Lt^T D upper triangular, diag(R) > 0.
//
// Binary64 on this part runs at 1/58 of binary32 (measured 1.20 TFLOP/s vs
// 70 TFLOP/s), so the plain-binary32 and mixed paths form each product of the
// Gram in binary32 over chunks of 512 rows and carry the running sums as
// unevaluated pairs of binary32 numbers (error-free TwoSum updates, about 48
// significant bits), rounded once to binary64 at the end; the O(l^3) Cholesky
// and solve arithmetic is binary32 on a binary64-scaled matrix.  The binary64
// path is binary64 throughout.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

// ------------------------------------------------------------------ Gram --
constexpr int GT = 64;       // Gram tile
constexpr int GCH = 32;      // rows per chunk in shared memory
constexpr int GFOLD = 4;     // chunks per binary64 fold (128 rows)
// The binary32 Gram folds its partial sums into the running pair every 512
// rows.
constexpr int GFOLD32 = 16;

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

// Binary32 partial Gram, same contract as gram_partial_kernel: 64 threads,
// thread (ty, tx) owns the 8 x 8 entries in rows {4 ty .. + 3, 32 + 4 ty .. + 3}
// and columns {4 tx .. + 3, 32 + 4 tx .. + 3} of the tile (four 16-byte
// shared-memory loads per 64 FMAs; the split halves keep the loads of a
// quarter-warp on distinct banks).  32-row chunks of the two column blocks
// stream into shared memory by cp.async, double-buffered, so the next chunk
// is in flight while the current one is multiplied.  Every GFOLD32 chunks the
// binary32 sums are folded into the split's partial, an unevaluated pair of
// binary32 numbers (hi, lo) updated by an error-free two-sum (Knuth's TwoSum),
// so the running sums carry about 48 significant bits without binary64
// arithmetic (which runs at 1/64 of the binary32 rate on this part).  The
// partial is private to the CTA: the first fold writes it, later ones add.
constexpr int G32_THREADS = 64;

// s + e = a + b exactly, s = fl(a + b) (Knuth's TwoSum; explicit round-to-
// nearest adds, so that nothing is contracted or reassociated).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
  return s;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 16 : 0;  // 0: fill the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Rows r0 .. r0 + 31 (below r_end), columns c0 .. c0 + 63 (below l) of Y into
// S: 512 groups of four floats, eight per thread.  vec: cp.async (l, ldy and
// Y allow 16-byte copies); else plain loads and stores.
__device__ __forceinline__ void gram_fetch_chunk(float (*S)[GT], const float* __restrict__ Y, int ldy, int r0,
                                                 int r_end, int c0, int l, bool vec) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int e = threadIdx.x + G32_THREADS * u;
    const int rr = e / 16, c4 = e % 16;
    const int gr = r0 + rr, gc = c0 + 4 * c4;
    float* dst = &S[rr][4 * c4];
    if (vec) {
      const bool ok = gr < r_end && gc < l;
      cp_async16(dst, ok ? (const void*)(Y + (size_t)gr * ldy + gc) : (const void*)Y, ok);
    } else {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (gr < r_end) {
        const float* src = Y + (size_t)gr * ldy + gc;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (gc + q < l) v[q] = src[q];
      }
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

__global__ void __launch_bounds__(G32_THREADS, 7)
    gram_partial_f32_kernel(int rows, int l, const float* __restrict__ Y, int ldy, double* __restrict__ P,
                            int rows_per_split, const int* gate, const int* skip, __nv_bfloat16* __restrict__ Yh,
                            __nv_bfloat16* __restrict__ Yl, int lb) {
  if ((gate && *gate == 0) || (skip && *skip != 0)) return;
  __shared__ __align__(16) float Yi[2][GCH][GT];
  __shared__ __align__(16) float Yj[2][GCH][GT];
  const int nb = ceil_div(l, GT);
  int t = blockIdx.x, bi = 0;
  while (t >= nb - bi) {
    t -= nb - bi;
    ++bi;
  }
  const int bj = bi + t;
  const bool diag = bi == bj;
  const int tid = threadIdx.x, tx = tid % 8, ty = tid / 8;
  const int r_beg = blockIdx.y * rows_per_split;
  const int r_end = min(rows, r_beg + rows_per_split);
  const bool vec = (l % 4) == 0 && (ldy % 4) == 0 && (((uintptr_t)Y) & 15) == 0;
  float2* out = reinterpret_cast<float2*>(P) + (size_t)blockIdx.y * l * l;
  float part[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) part[a][b] = 0.f;
  bool first_fold = true;
  gram_fetch_chunk(Yi[0], Y, ldy, r_beg, r_end, bi * GT, l, vec);
  if (!diag) gram_fetch_chunk(Yj[0], Y, ldy, r_beg, r_end, bj * GT, l, vec);
  cp_async_commit();
  int chunk = 0;
  for (int r0 = r_beg; r0 < r_end; r0 += GCH, ++chunk) {
    const int cur = chunk & 1;
    if (r0 + GCH < r_end) {  // the next chunk into the other buffer
      gram_fetch_chunk(Yi[cur ^ 1], Y, ldy, r0 + GCH, r_end, bi * GT, l, vec);
      if (!diag) gram_fetch_chunk(Yj[cur ^ 1], Y, ldy, r0 + GCH, r_end, bj * GT, l, vec);
    }
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of the current chunk have landed
    __syncthreads();   // and every thread's
    const float(*Si)[GT] = Yi[cur];
    const float(*Sj)[GT] = diag ? Yi[cur] : Yj[cur];
    if (diag && Yh) {
      // the diagonal tiles read every element of Y exactly once: write the
      // bf16 pair Y = Yh + Yl that the tensor-core apply takes
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + G32_THREADS * u;
        const int rr = e / 16, c4 = e % 16;
        const int gr = r0 + rr, gc = bi * GT + 4 * c4;
        if (gr < r_end && gc < l) {
          const float4 a = *reinterpret_cast<const float4*>(&Si[rr][4 * c4]);
          const __nv_bfloat162 h01 = __floats2bfloat162_rn(a.x, a.y), h23 = __floats2bfloat162_rn(a.z, a.w);
          const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
          const __nv_bfloat162 l01 = __floats2bfloat162_rn(a.x - f01.x, a.y - f01.y);
          const __nv_bfloat162 l23 = __floats2bfloat162_rn(a.z - f23.x, a.w - f23.y);
          __nv_bfloat16* ph = Yh + (size_t)gr * lb + gc;
          __nv_bfloat16* pl = Yl + (size_t)gr * lb + gc;
          if (gc + 4 <= l && (lb % 4) == 0) {
            *reinterpret_cast<uint2*>(ph) = make_uint2(*reinterpret_cast<const uint32_t*>(&h01),
                                                       *reinterpret_cast<const uint32_t*>(&h23));
            *reinterpret_cast<uint2*>(pl) = make_uint2(*reinterpret_cast<const uint32_t*>(&l01),
                                                       *reinterpret_cast<const uint32_t*>(&l23));
          } else {
            const __nv_bfloat16 hv[4] = {h01.x, h01.y, h23.x, h23.y}, lv[4] = {l01.x, l01.y, l23.x, l23.y};
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (gc + q < l) {
                ph[q] = hv[q];
                pl[q] = lv[q];
              }
          }
        }
      }
    }
#pragma unroll 2
    for (int rr = 0; rr < GCH; ++rr) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Si[rr][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Si[rr][32 + 4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Sj[rr][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Sj[rr][32 + 4 * tx]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) part[u][v] = fmaf(a[u], b[v], part[u][v]);
    }
    if ((chunk % GFOLD32) == GFOLD32 - 1 || r0 + GCH >= r_end) {
      // fold through shared memory (the current buffers, free once every
      // thread is done with them), one entry per thread and step, so that
      // the fold adds no registers to the product loop
      float* Fi = &Yi[cur][0][0];  // rows 0 .. 31 of the 64 x 64 tile
      float* Fj = &Yj[cur][0][0];  // rows 32 .. 63
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int ii = u < 4 ? 4 * ty + u : 32 + 4 * ty + u - 4;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const int jj = v < 4 ? 4 * tx + v : 32 + 4 * tx + v - 4;
          (ii < 32 ? Fi + ii * GT : Fj + (ii - 32) * GT)[jj] = part[u][v];
          part[u][v] = 0.f;
        }
      }
      __syncthreads();
      // 64 entries per thread in batches of 8: the running pairs of a batch
      // are loaded together (8 loads in flight), then updated and stored
      for (int e0 = tid; e0 < GT * GT; e0 += 8 * G32_THREADS) {
        float2 h[8];
        if (!first_fold) {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * G32_THREADS;
            const int i = bi * GT + e / GT, j = bj * GT + e % GT;
            h[u] = (i < l && j < l) ? out[(size_t)i * l + j] : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * G32_THREADS;
          const int ii = e / GT, jj = e % GT;
          const int i = bi * GT + ii, j = bj * GT + jj;
          if (i < l && j < l) {
            const float pv = (ii < 32 ? Fi + ii * GT : Fj + (ii - 32) * GT)[jj];
            float2 v = make_float2(pv, 0.f);
            if (!first_fold) {
              float e2;
              const float sum = two_sum(h[u].x, pv, e2);
              v = make_float2(sum, __fadd_rn(h[u].y, e2));
            }
            out[(size_t)i * l + j] = v;
          }
        }
      }
      first_fold = false;
    }
    __syncthreads();  // every read of this buffer is done before it is refilled
  }
}

// G[i][j] = sum over splits (fixed order) of the upper-triangular partials;
// Gf receives G rounded to binary32 (the Cholesky kernel's input on the
// binary32 path; converting here spreads the conversions over the GPU).  The
// partials are (hi, lo) pairs of binary32 (PT = float2, summed the same way:
// TwoSum into running pairs, one binary64 add at the end) or binary64 (summed
// in binary64).  One CTA per 8 x 32 sub-tile (one entry per thread) of a
// computed (upper) Gram tile: it sums the sub-tile with coalesced reads and
// writes it, and for an off-diagonal Gram tile also its transpose (through
// shared memory, eight consecutive entries per row), so reads and writes walk
// rows.
constexpr int GR_R = 8, GR_C = 32;

__device__ __forceinline__ double gram_sum_entry(const double* p, size_t ll, int splits) {
  // eight interleaved binary64 sums (a fixed order): eight loads in flight
  double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int z = 0;
  for (; z + 7 < splits; z += 8) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] += p[(size_t)(z + q) * ll];
  }
  for (; z < splits; ++z) a[0] += p[(size_t)z * ll];
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

__device__ __forceinline__ double gram_sum_entry(const float2* p, size_t ll, int splits) {
  // eight interleaved running pairs (a fixed order), sixteen loads in flight
  constexpr int Q = 8, U = 16;
  float hs[Q], ls[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) hs[q] = ls[q] = 0.f;
  int z = 0;
  for (; z + U - 1 < splits; z += U) {
    float2 v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) v[q] = p[(size_t)(z + q) * ll];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      float e;
      hs[q % Q] = two_sum(hs[q % Q], v[q].x, e);
      ls[q % Q] = __fadd_rn(ls[q % Q], __fadd_rn(e, v[q].y));
    }
  }
  for (; z < splits; ++z) {
    const float2 v = p[(size_t)z * ll];
    float e;
    hs[0] = two_sum(hs[0], v.x, e);
    ls[0] = __fadd_rn(ls[0], __fadd_rn(e, v.y));
  }
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < Q; ++q) t += (double)hs[q] + (double)ls[q];
  return t;
}

template <typename PT>
__global__ void __launch_bounds__(GR_R * GR_C)
    gram_reduce_kernel(int l, int splits, const PT* __restrict__ P, double* __restrict__ G,
                       float* __restrict__ Gf, const int* gate, const int* skip) {
  if ((gate && *gate == 0) || (skip && *skip != 0)) return;
  const int ti = blockIdx.y * GR_R, tj = blockIdx.x * GR_C;
  if (ti / GT > tj / GT) return;  // the mirror of a computed tile: its CTA writes it
  const bool mirror = ti / GT < tj / GT;
  __shared__ double tile[GR_R][GR_C + 1];
  const int tx = threadIdx.x % GR_C, ty = threadIdx.x / GR_C;
  const int i = ti + ty, j = tj + tx;
  double s = 0.0;
  if (i < l && j < l) {
    s = gram_sum_entry(P + (size_t)i * l + j, (size_t)l * l, splits);
    G[(size_t)i * l + j] = s;
    if (Gf) Gf[(size_t)i * l + j] = (float)s;
  }
  if (!mirror) return;
  tile[ty][tx] = s;
  __syncthreads();
  // G(tj + a, ti + b) = G(ti + b, tj + a)
  const int a = threadIdx.x / GR_R, b = threadIdx.x % GR_R;
  const int ii = tj + a, jj = ti + b;
  if (ii < l && jj < l) {
    const double v = tile[b][a];
    G[(size_t)ii * l + jj] = v;
    if (Gf) Gf[(size_t)ii * l + jj] = (float)v;
  }
}

// CTAs of the partial-Gram kernel for Y's element size that one SM holds at
// once (occupancy query, cached per size; 1 if the query fails).
int gram_resident(size_t tsize) {
  static int cached[2] = {0, 0};
  const int w = tsize == 4 ? 0 : 1;
  if (cached[w] == 0) {
    int b = 0;
    cudaError_t e = tsize == 4
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gram_partial_f32_kernel, G32_THREADS, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gram_partial_kernel<double>, 256, 0);
    if (e != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    cached[w] = b;
  }
  return cached[w];
}

// Row splits of the partial Gram: enough CTAs to fill every SM's slots in one
// wave (a second, nearly empty wave would double the kernel's time), at least
// four chunks of rows per split.
int gram_splits(int rows, int l, int sms, size_t tsize) {
  const int nb = ceil_div(l, GT);
  const int tiles = nb * (nb + 1) / 2;
  int s = gram_resident(tsize) * sms / tiles;
  const int smax = ceil_div(rows, 4 * GCH);
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  if (s > 256) s = 256;
  return s;
}

template <typename T>
void launch_gram(int rows, int l, const T* Y, int ldy, double* P, double* G, float* Gf, int sms, const int* gate,
                 cudaStream_t s, const int* skip, __nv_bfloat16* Yh, __nv_bfloat16* Yl, int lb) {
  const int nb = ceil_div(l, GT);
  const int tiles = nb * (nb + 1) / 2;
  const int splits = gram_splits(rows, l, sms, sizeof(T));
  const int rps = ceil_div(ceil_div(rows, splits), GCH) * GCH;
  const int used = ceil_div(rows, rps);
  if (sizeof(T) == 4)
    gram_partial_f32_kernel<<<dim3(tiles, used), G32_THREADS, 0, s>>>(rows, l, (const float*)Y, ldy, P, rps, gate,
                                                                      skip, Yh, Yl, lb);
  else
    gram_partial_kernel<T><<<dim3(tiles, used), 256, 0, s>>>(rows, l, Y, ldy, P, rps, gate, skip);
  note_launch();
  const dim3 rgrid(ceil_div(l, GR_C), ceil_div(l, GR_R));
  if (sizeof(T) == 4)
    gram_reduce_kernel<float2><<<rgrid, GR_R * GR_C, 0, s>>>(l, used, reinterpret_cast<const float2*>(P), G, Gf,
                                                             gate, skip);
  else
    gram_reduce_kernel<double><<<rgrid, GR_R * GR_C, 0, s>>>(l, used, P, G, Gf, gate, skip);
  note_launch();
}

// -------------------------------------------------------------- Cholesky --
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

// Single CTA.  In: G (l x l binary64) and Gf (G rounded to binary32, used on
// the binary32 path).  Out:
//   Ub   : l x l row-major, type C: the upper triangular factor Lt^T whose
//          32 x 32 diagonal blocks are replaced by their inverses; with dinv
//          it defines Q = (Y D^-1) Lt^-T (blocked triangular solve, apply_kernel).
//          With Lblk given, the factor is written instead in its blocked
//          shared-memory form (the L blocks, then the diagonal-block inverses)
//          for the explicit inverse kernel.
//   dinv : 1 / d_i, d_i = sqrt(G_ii)
//   R    : optional l x l row-major binary64, R = Lt^T D (zeros below the diagonal)
// where G = D Gt D and Gt = Lt Lt^T.  Pivots below tau (unit-diagonal scale)
// restart the factorization on Gt + s I, s = s0, 32 s0, ...; four failures
// give RSVD_E_BREAKDOWN.
//
// Storage: the lower triangle of 32 x 32 blocks, block (bi, bj), bj <= bi, at
// index bi (bi + 1) / 2 + bj, each block 32 rows of CP = 33 entries (the pad
// keeps column reads free of bank conflicts).  l is padded to 32 NB with an
// identity block, which decouples the pad from the rest.
//
// Right-looking over block columns k, with one block of lookahead:
//   (1) L_ik = A_ik L_kk^-T, i > k, forward substitution, one thread per row;
//   (2) A_i,k+1 -= L_ik L_k+1,k^T, i > k (the next block column);
//   (3) warp 0 factors A_k+1,k+1 while the other warps apply the rest of the
//       trailing update, A_ij -= L_ik L_jk^T, k + 1 < j <= i.
// The inverses of the diagonal blocks (for Ub and the explicit inverse) come
// after the loop, one warp per block.  A warp updates a 32 x 32 block with
// each lane holding a 4 x 8 tile.
constexpr int CBK = 32;             // block size
constexpr int CP = 33;              // padded row stride within a block
constexpr int CBS = CBK * CP;       // stored entries per block
// The latest diagonal block's factor transposed (row q = column q of L), row
// stride LTP, with 32 entries of slack after the last row: the panel
// substitution reads row q from column q + 1 on at fixed offsets.
constexpr int LTP = 33;
constexpr int LT_ENTRIES = CBK * LTP + 32;

__device__ __forceinline__ int lblk(int bi, int bj) { return bi * (bi + 1) / 2 + bj; }

// Warp-level Cholesky of a 32 x 32 block.  Lane i holds row i of the block in
// row[] (lower part valid) and writes row i of L to Li[0..31] (zeros above
// the diagonal); *dii receives L(i, i).  Column q is always row[0]: each step
// updates the trailing entries and shifts them down by one, so every register
// index is static while the step loop stays rolled (a compact loop body keeps
// the code resident in the instruction cache; the fully unrolled factor ran
// slower inside the blocked factorization, where other warps run other code
// between its calls).  Steps q0 <= q < q1 touch entries 1 .. J = 31 - q0 only
// (later ones are past column 31), so the four quarters of the steps run with
// J = 31, 23, 15, 7.  A loop exit inside the unrolled body instead cost more
// than the shuffles it saved.  Returns false (warp-uniformly: the pivot is a
// shuffled value) on a pivot below tau.
template <typename C, int J>
__device__ __forceinline__ bool chol_steps(C (&row)[32], int q0, int q1, C tau, C* Li, C* dii, C* LT) {
  const int lane = threadIdx.x % 32;
#pragma unroll 1
  for (int q = q0; q < q1; ++q) {
    const C akk = __shfl_sync(0xffffffffu, row[0], q);
    if (!(akk > tau) || !isfinite(akk)) return false;
    const C rp = rsqrt(akk), piv = akk * rp;
    const C liq = (lane == q) ? piv : (lane > q ? row[0] * rp : C(0));
    Li[q] = liq;
    LT[q * LTP + lane] = liq;  // column q of L as row q of its transpose
    if (lane == q) *dii = piv;
    // row i -= l(i, q) * l(j, q) for q < j <= i, shifted down one column
#pragma unroll
    for (int j = 1; j <= J; ++j) {
      const C ljq = __shfl_sync(0xffffffffu, liq, (q + j) & 31);
      row[j - 1] = (lane >= q + j) ? fma(-liq, ljq, row[j]) : row[j];
    }
  }
  return true;
}

template <typename C>
__device__ __forceinline__ bool warp_chol32(C (&row)[32], C tau, C* Li, C* dii, C* LT) {
  return chol_steps<C, 31>(row, 0, 8, tau, Li, dii, LT) && chol_steps<C, 23>(row, 8, 16, tau, Li, dii, LT) &&
         chol_steps<C, 15>(row, 16, 24, tau, Li, dii, LT) && chol_steps<C, 7>(row, 24, 32, tau, Li, dii, LT);
}

// Warp-level inverse of the lower triangular L held as rows (lane i: row[]
// = row i of L, consumed): lane i ends with x[] = row i of L^-1.  x doubles as
// the accumulator: lanes i > t add L(i, t) X(t, :) at step t, when lane t turns
// its accumulator into its final row.  L(i, t) is row[0] at step t (the row
// shifts down one column per step), so the step loop stays rolled; steps
// t0 <= t < t0 + 8 touch X(t, c) for c <= T = t0 + 7 only (X(t, c) = 0 for
// c > t) and shift row entries below 31 - t0 only.
template <typename C, int T>
__device__ __forceinline__ void trinv_steps(C (&row)[32], C (&x)[32]) {
  const int lane = threadIdx.x % 32;
  constexpr int t0 = T - 7;
#pragma unroll 1
  for (int t = t0; t <= T; ++t) {
    const C lit = row[0];
    if (lane == t) {
      const C rd = C(1) / lit;
#pragma unroll
      for (int c = 0; c <= T; ++c) x[c] = ((c == t ? C(1) : C(0)) - x[c]) * rd;
    }
    const C m = lane > t ? lit : C(0);
#pragma unroll
    for (int c = 0; c <= T; ++c) x[c] = fma(m, __shfl_sync(0xffffffffu, x[c], t), x[c]);
#pragma unroll
    for (int j = 0; j < 31 - t0; ++j) row[j] = row[j + 1];
  }
}

template <typename C>
__device__ __forceinline__ void warp_trinv32(C (&row)[32], C (&x)[32]) {
#pragma unroll
  for (int c = 0; c < 32; ++c) x[c] = C(0);
  trinv_steps<C, 7>(row, x);
  trinv_steps<C, 15>(row, x);
  trinv_steps<C, 23>(row, x);
  trinv_steps<C, 31>(row, x);
}

// One warp: Cb = A B^T (sub == false, in place allowed: Cb may be Ab) or
// Cb -= A B^T (sub == true), 32 x 32 blocks with row stride CP.  Lane (lr, lc)
// holds rows 4 lr .. + 3, columns 8 lc .. + 7.
template <typename C>
__device__ __forceinline__ void warp_blk_nt(C* Cb, const C* Ab, const C* Bb, bool sub) {
  const int lane = threadIdx.x % 32, lr = lane >> 2, lc = lane & 3;
  C acc[4][8];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 8; ++y) acc[x][y] = C(0);
#pragma unroll 4
  for (int t = 0; t < 32; ++t) {
    C a[4], b[8];
#pragma unroll
    for (int x = 0; x < 4; ++x) a[x] = Ab[(4 * lr + x) * CP + t];
#pragma unroll
    for (int y = 0; y < 8; ++y) b[y] = Bb[(8 * lc + y) * CP + t];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 8; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
  }
  __syncwarp();
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      C* p = Cb + (4 * lr + x) * CP + 8 * lc + y;
      *p = sub ? *p - acc[x][y] : acc[x][y];
    }
  __syncwarp();
}

// Thread-per-row forward substitution x <- x L_kk^-T (L_kk lower triangular,
// given transposed in LT; rdg = 1 / diag), writing x to a[] as it goes.  x[0] is always column q: each
// step updates the later entries and shifts them down by one (static register
// indices, a rolled step loop); steps q0 <= q < q1 touch entries 1 .. J only.
// A fully unrolled substitution (528 FMAs of straight-line code per row) ran
// about three times slower inside the factorization.
template <typename C, int J>
__device__ __forceinline__ void trsm_steps(C (&x)[32], C* a, const C* LT, const C* rdg, int q0, int q1) {
#pragma unroll 1
  for (int q = q0; q < q1; ++q) {
    const C xq = x[0] * rdg[q];
    a[q] = xq;
    const C* lq = LT + q * LTP + q;  // lq[j] = L(q + j, q); past column 31 never stored
#pragma unroll
    for (int j = 1; j <= J; ++j) x[j - 1] = fma(-xq, lq[j], x[j]);
  }
}

// One warp: Cholesky of diagonal block k in place, and 1 / L(q, q) into
// rdg[32 k + q].  On a pivot failure sets *fail.
template <typename C>
__device__ __forceinline__ void diag_potrf(C* Ls, C* rdg, int k, C tau, int* fail, C* LT) {
  const int lane = threadIdx.x % 32;
  C* A = Ls + (size_t)lblk(k, k) * CBS + lane * CP;
  C row[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) row[j] = (j <= lane) ? A[j] : C(0);
  __syncwarp();
  C dii = C(1);
  const bool ok = warp_chol32<C>(row, tau, A, &dii, LT);
  __syncwarp();
  if (!ok) {
    if (lane == 0) *fail = 1;
    return;
  }
  rdg[CBK * k + lane] = C(1) / dii;
}

// One warp: X_kk = L_kk^-1 into Xs[k] (rows of L from shared memory).
template <typename C>
__device__ __forceinline__ void diag_trinv(const C* Ls, C* Xs, int k) {
  const int lane = threadIdx.x % 32;
  const C* A = Ls + (size_t)lblk(k, k) * CBS + lane * CP;
  C row[32], x[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) row[j] = (j <= lane) ? A[j] : C(0);
  warp_trinv32<C>(row, x);
  C* X = Xs + (size_t)k * CBS + lane * CP;
#pragma unroll
  for (int j = 0; j < 32; ++j) X[j] = (j <= lane) ? x[j] : C(0);
}

template <typename C, int NT>
__global__ void __launch_bounds__(NT)
    chol_kernel(int l, const double* __restrict__ G, const float* __restrict__ Gf, C* __restrict__ Ub,
                C* __restrict__ dinv, double* __restrict__ R, DevStatus* st, int pass, const int* gate,
                const int* skip, float accept, C* __restrict__ Lblk) {
  if ((gate && *gate == 0) || (skip && *skip != 0)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = (l + CBK - 1) / CBK;
  const int nblk = NB * (NB + 1) / 2;
  C* Ls = reinterpret_cast<C*>(smem_raw);  // nblk blocks
  C* Xs = Ls + (size_t)nblk * CBS;         // NB diagonal inverses
  double* d = reinterpret_cast<double*>(Xs + (size_t)NB * CBS);
  C* rdc = reinterpret_cast<C*>(d + l);
  C* rdg = rdc + l;  // 1 / L(i, i), 32 NB entries
  C* LT = rdg + CBK * NB;  // the latest diagonal factor, transposed (LT_ENTRIES)
  __shared__ int s_fail;
  __shared__ unsigned char s_bi[64], s_bj[64];
  const int tid = threadIdx.x;
  const int warp = tid / 32, lane = tid % 32, nw = NT / 32;
  const double u = Eps<C>::u;
  const C ctau = (C)(1024.0 * u);
  const double s0 = 16384.0 * u;

  bool bad = false;
  for (int i = tid; i < l; i += NT) {
    const double gii = G[(size_t)i * l + i];
    if (!isfinite(gii)) bad = true;
    d[i] = gii > 0.0 ? sqrt(gii) : 1.0;
    rdc[i] = (C)(1.0 / d[i]);
  }
  if (tid < nblk) {
    int bi = 0;
    while ((bi + 1) * (bi + 2) / 2 <= tid) ++bi;
    s_bi[tid] = (unsigned char)bi;
    s_bj[tid] = (unsigned char)(tid - bi * (bi + 1) / 2);
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
    // unit-diagonal scaling Gt = D^-1 G D^-1 (+ shift) in the working
    // precision, straight from G (row-major, symmetric) into the blocks:
    // groups of four consecutive columns of one row, eight groups in flight
    // per thread (16-byte loads where l and the base allow them)
    {
      const C* Gsrc = (sizeof(C) == 4) ? reinterpret_cast<const C*>(Gf) : reinterpret_cast<const C*>(G);
      const bool v4 = (l % 4 == 0) && ((((uintptr_t)Gsrc) & (4 * sizeof(C) - 1)) == 0);
      const int ngroups = nblk * CBK * (CBK / 4);
      for (int g0 = tid; g0 < ngroups; g0 += 8 * NT) {
        C v[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int g = g0 + u * NT;
          const int b = g >> 8, r = (g >> 3) & 31, c4 = (g & 7) * 4;
          const int i = CBK * s_bi[b < nblk ? b : 0] + r, j = CBK * s_bj[b < nblk ? b : 0] + c4;
          if (g < ngroups && i < l && j + 3 < l && v4) {
            if (sizeof(C) == 4) {
              const float4 x = *reinterpret_cast<const float4*>(Gsrc + (size_t)i * l + j);
              v[u][0] = (C)x.x;
              v[u][1] = (C)x.y;
              v[u][2] = (C)x.z;
              v[u][3] = (C)x.w;
            } else {
              const double2 x0 = *reinterpret_cast<const double2*>(Gsrc + (size_t)i * l + j);
              const double2 x1 = *reinterpret_cast<const double2*>(Gsrc + (size_t)i * l + j + 2);
              v[u][0] = (C)x0.x;
              v[u][1] = (C)x0.y;
              v[u][2] = (C)x1.x;
              v[u][3] = (C)x1.y;
            }
          } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
              v[u][t] = (g < ngroups && i < l && j + t < l) ? Gsrc[(size_t)i * l + j + t] : C(0);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int g = g0 + u * NT;
          if (g >= ngroups) break;
          const int b = g >> 8, r = (g >> 3) & 31, c4 = (g & 7) * 4;
          const int i = CBK * s_bi[b] + r, j = CBK * s_bj[b] + c4;
          C* dst = Ls + (size_t)b * CBS + r * CP + c4;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            C w;
            if (i < l && j + t < l) {
              w = v[u][t] * rdc[i] * rdc[j + t];
              if (i == j + t) w += shift;
              if (!isfinite(w)) w = C(0);
            } else {
              w = (i == j + t) ? C(1) : C(0);
            }
            dst[t] = w;
          }
        }
      }
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    if (accept > 0.f && attempt == 0) {
      // acceptance test of an intermediate basis (the previous pass's Q): its
      // Gram, scaled to unit diagonal, within accept of I entry by entry
      // (so ||Gt - I||_2 <= (l - 1) accept) and its column norms squared
      // within [1/2, 3/2]; then Q is kept and this pass does nothing more
      float mx = 0.f;
      for (int e = tid; e < nblk * CBK * CBK; e += NT) {
        const int b = e >> 10, r = (e >> 5) & 31, c = e & 31;
        const int i = CBK * s_bi[b] + r, j = CBK * s_bj[b] + c;
        if (i < l && j < l && i != j) mx = fmaxf(mx, fabsf((float)Ls[(size_t)b * CBS + r * CP + c]));
      }
      for (int i = tid; i < l; i += NT) mx = fmaxf(mx, fabsf((float)(d[i] * d[i]) - 1.f) * (2.f * accept));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) atomicMax(reinterpret_cast<unsigned int*>(&s_fail), __float_as_uint(mx));
      __syncthreads();
      const bool keep = __uint_as_float((unsigned)s_fail) <= accept;
      __syncthreads();
      if (tid == 0) {
        st->run2 = keep ? 0 : 1;
        s_fail = 0;
      }
      __syncthreads();
      if (keep) return;
    }
    if (warp == 0) diag_potrf<C>(Ls, rdg, 0, ctau, &s_fail, LT);
    __syncthreads();
    if (s_fail == 0) {
      for (int k = 0; k < NB; ++k) {
        // (1) L_ik = A_ik L_kk^-T by forward substitution, one thread per row
        {
          for (int rr = tid; rr < (NB - 1 - k) * CBK; rr += NT) {
            const int i = k + 1 + rr / CBK, r = rr % CBK;
            C* a = Ls + (size_t)lblk(i, k) * CBS + r * CP;
            C x[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) x[q] = a[q];
            const C* rk = rdg + CBK * k;
            trsm_steps<C, 31>(x, a, LT, rk, 0, 8);
            trsm_steps<C, 23>(x, a, LT, rk, 8, 16);
            trsm_steps<C, 15>(x, a, LT, rk, 16, 24);
            trsm_steps<C, 7>(x, a, LT, rk, 24, 32);
          }
        }
        __syncthreads();
        if (k + 1 >= NB) break;
        // (2) the next block column
        for (int i = k + 1 + warp; i < NB; i += nw)
          warp_blk_nt<C>(Ls + (size_t)lblk(i, k + 1) * CBS, Ls + (size_t)lblk(i, k) * CBS,
                         Ls + (size_t)lblk(k + 1, k) * CBS, true);
        __syncthreads();
        // (3) factor the next diagonal block || the rest of the trailing update
        if (warp == 0) {
          diag_potrf<C>(Ls, rdg, k + 1, ctau, &s_fail, LT);
        } else {
          const int nt = NB - k - 2;  // block columns k + 2 .. NB - 1
          const int tasks = nt * (nt + 1) / 2;
          for (int tk = warp - 1; tk < tasks; tk += nw - 1) {
            int ii = 0;
            while ((ii + 1) * (ii + 2) / 2 <= tk) ++ii;
            const int i = k + 2 + ii, j = k + 2 + (tk - ii * (ii + 1) / 2);
            warp_blk_nt<C>(Ls + (size_t)lblk(i, j) * CBS, Ls + (size_t)lblk(i, k) * CBS,
                           Ls + (size_t)lblk(j, k) * CBS, true);
          }
        }
        __syncthreads();
        if (s_fail) break;
      }
    }
    __syncthreads();
    if (s_fail == 0) {
      // the inverses of the diagonal blocks, one warp each (they are needed
      // only by the outputs, so they stay off the factorization's chain)
      for (int b = warp; b < NB; b += nw) diag_trinv<C>(Ls, Xs, b);
      __syncthreads();
      break;
    }
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
  // R(i, j) = L(j, i) d_j for i <= j; one warp per row, lane = column within
  // a 32-column block (the block's base is warp-uniform)
  if (R) {
    for (int i = warp; i < l; i += nw) {
      const int bi = i >> 5, ii = i & 31;
      double* Ri = R + (size_t)i * l;
      for (int bj = 0; bj < NB; ++bj) {
        const int j = CBK * bj + lane;
        if (j >= l) break;
        double v = 0.0;
        if (bj >= bi && i <= j) v = (double)Ls[(size_t)lblk(bj, bi) * CBS + lane * CP + ii] * d[j];
        Ri[j] = v;
      }
    }
  }
  if (Lblk) {
    // the blocked factor as it sits in shared memory (L blocks, then the
    // diagonal-block inverses), for the explicit inverse kernel: one flat,
    // 16-byte copy
    const int n4 = (nblk + NB) * CBS * (int)sizeof(C) / 16;
    const float4* s4 = reinterpret_cast<const float4*>(Ls);
    float4* d4 = reinterpret_cast<float4*>(Lblk);
    for (int e = tid; e < n4; e += NT) d4[e] = s4[e];
  } else {
    // Ub(i, j) = L(j, i) for block(i) < block(j), X_bb(j, i) inside a diagonal
    // block (i <= j), 0 below
    for (int i = warp; i < l; i += nw) {
      const int bi = i >> 5, ii = i & 31;
      C* Ui = Ub + (size_t)i * l;
      for (int bj = 0; bj < NB; ++bj) {
        const int j = CBK * bj + lane;
        if (j >= l) break;
        C v = C(0);
        if (bj >= bi && i <= j) {
          const C* blk = (bj == bi) ? Xs + (size_t)bj * CBS : Ls + (size_t)lblk(bj, bi) * CBS;
          v = blk[lane * CP + ii];
        }
        Ui[j] = v;
      }
    }
  }
  for (int i = tid; i < l; i += NT) dinv[i] = rdc[i];
}

size_t chol_smem_bytes(int l, size_t csize) {
  const int NB = (l + CBK - 1) / CBK;
  const size_t blocks = (size_t)NB * (NB + 1) / 2 + NB;  // L, X
  return blocks * CBS * csize + (size_t)l * sizeof(double) + (size_t)l * csize + (size_t)CBK * NB * csize +
         (size_t)LT_ENTRIES * csize;
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
constexpr int AP_ROWS = 64;

// dst[r * dld + c] = src[r * sld + c] for r < nrows, c < ncols (rows r >= nr
// read as zero), by the whole CTA with eight independent loads in flight per
// thread (16-byte loads when every row is 16-byte aligned).
template <typename T, typename C>
__device__ __forceinline__ void stage_rows(C* dst, int dld, const T* src, int sld, int nrows, int nr, int ncols) {
  const bool vec = sizeof(T) == 4 && sizeof(C) == 4 && (sld % 4) == 0 && (dld % 4) == 0 && (ncols % 4) == 0 &&
                   (((uintptr_t)src | (uintptr_t)dst) & 15) == 0;
  const int nt = blockDim.x;
  if (vec) {
    const int cv = ncols / 4, total = nrows * cv;
    for (int e0 = threadIdx.x; e0 < total; e0 += 8 * nt) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nt;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < total) {
          const int r = e / cv, c = e % cv;
          if (r < nr) v[u] = *reinterpret_cast<const float4*>(src + (size_t)r * sld + 4 * c);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nt;
        if (e < total) {
          const int r = e / cv, c = e % cv;
          *reinterpret_cast<float4*>(dst + (size_t)r * dld + 4 * c) = v[u];
        }
      }
    }
    return;
  }
  const int total = nrows * ncols;
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * nt) {
    C v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nt;
      v[u] = C(0);
      if (e < total) {
        const int r = e / ncols, c = e % ncols;
        if (r < nr) v[u] = (C)src[(size_t)r * sld + c];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nt;
      if (e < total) dst[(size_t)(e / ncols) * dld + e % ncols] = v[u];
    }
  }
}

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
  // stage the stripe, then scale it by dinv
  stage_rows<T, C>(ys, l, Y + (size_t)r0 * ldy, ldy, AP_ROWS, nr, l);
  __syncthreads();
  for (int e = tid; e < AP_ROWS * l; e += 256) ys[e] *= dinv[e % l];
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
      // rows k0 .. k0 + kw of Ub, columns from k0 on (Ub is zero to the left)
      stage_rows<C, C>(rs + k0, l, Ub + (size_t)k0 * l + k0, l, 32, kw, l - k0);
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
                 const int* gate, cudaStream_t s, const int* skip, float accept = 0.f, C* Lblk = nullptr) {
  // binary32: 512 threads (at most 128 registers each; a diagonal-block warp
  // keeps a row of L and a row of its inverse in registers); binary64
  // (l <= 128): 256
  constexpr int NT = sizeof(C) == 4 ? 512 : 256;
  const size_t smem = chol_smem_bytes(l, sizeof(C));
  auto kfn = chol_kernel<C, NT>;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kfn<<<1, NT, smem, s>>>(l, G, Gf, Ub, dinv, R, st, pass, gate, skip, accept, Lblk);
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

// ------------------------------------------------------- orth entry points --
size_t orth_workspace_bytes(int rows, int l, int sms, size_t csize) {
  Carver c(nullptr);
  c.take<double>((size_t)gram_splits(rows, l, sms, csize) * l * l);  // Gram partials
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
  double* P = c.take<double>((size_t)gram_splits(rows, l, sms, sizeof(T)) * l * l);
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

// CholeskyQR2 (+ shifted third pass) for the mixed-precision paths with the
// apply on tensor cores for tall blocks: Q = Y M, M = R^-1 from the Cholesky
// kernel, as the three-term split-bf16 product Yh Mh + Yh Ml + Yl Mh (relative
// error about 2^-16 instead of binary32's 2^-24; the Gram stays binary32
// products with binary64 sums).  Shorter blocks take the SIMT solve.
// ------------------------------------------------------ explicit inverse --
// M = R^-1 = D^-1 L^-T for the tensor-core apply, from the Cholesky kernel's
// blocked factor Lblk (the L blocks L_ik and the diagonal-block inverses
// X_bb = L_bb^-1, each 32 x 32 with row stride CP) and dinv.  The block columns of W = L^-1 are
// independent, so CTA j forms block column j by block forward substitution,
//   W_jj = X_jj,  W_ij = -X_ii sum_{k = j}^{i - 1} L_ik W_kj  (i > j),
// with every block it needs staged in shared memory first (L_ik for
// j <= k < i, X_ii for i >= j), and writes block row j of M:
// M(32 j + r, 32 i + c) = W_ij(c, r) / d_(32 j + r).  One CTA per block column
// spreads what the single-CTA factorization would do serially.
constexpr int INV_THREADS = 512;

__global__ void __launch_bounds__(INV_THREADS)
    inv_tri_kernel(int l, const float* __restrict__ Lblk, const float* __restrict__ dinv, float* __restrict__ M,
                   const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = (l + CBK - 1) / CBK;
  const int nblk = NB * (NB + 1) / 2;
  const int j = blockIdx.x;
  const int nw = NB - j;                      // blocks W_jj .. W_(NB-1) j
  float* Wc = reinterpret_cast<float*>(smem_raw);   // nw blocks
  float* Xd = Wc + (size_t)nw * CBS;                // X_ii, i = j .. NB-1
  float* Lb = Xd + (size_t)nw * CBS;                // L_ik, j <= k < i, packed by (i, k)
  float* Tb = Lb + (size_t)(nw * (nw - 1) / 2) * CBS;
  const int tid = threadIdx.x;
  auto lidx = [&](int i, int k) { return (i - j - 1) * (i - j) / 2 + (k - j); };  // i > k >= j
  // ---- stage X_ii (i >= j) and L_ik (i > k >= j): whole blocks of the
  // Cholesky kernel's blocked factor (its shared-memory layout: the L blocks
  // at index bi (bi + 1) / 2 + bj, then the diagonal-block inverses), copied
  // 16 bytes at a time, eight copies in flight per thread
  const int nl = nw * (nw - 1) / 2;
  __shared__ unsigned short s_src[64];
  if (tid < nw + nl) {
    if (tid < nw) {
      s_src[tid] = (unsigned short)(nblk + j + tid);
    } else {
      const int q = tid - nw;
      int a = 0;
      while ((a + 1) * (a + 2) / 2 <= q) ++a;  // q = a (a + 1) / 2 + b, b <= a
      const int i = j + 1 + a, k = j + (q - a * (a + 1) / 2);
      s_src[tid] = (unsigned short)lblk(i, k);
    }
  }
  __syncthreads();
  {
    constexpr int B4 = CBS / 4;  // float4 per block
    const int total = (nw + nl) * B4;
    const float4* src = reinterpret_cast<const float4*>(Lblk);
    float4* dst = reinterpret_cast<float4*>(Xd);  // Xd and Lb are contiguous
    for (int g0 = tid; g0 < total; g0 += 8 * INV_THREADS) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + u * INV_THREADS;
        if (g < total) v[u] = src[(size_t)s_src[g / B4] * B4 + g % B4];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + u * INV_THREADS;
        if (g < total) dst[g] = v[u];
      }
    }
  }
  __syncthreads();
  // Right-looking: once W_kj is final, every T_i = sum_k L_ik W_kj (i > k)
  // takes its term at once, and W_(k+1) j = -X_(k+1)(k+1) T_(k+1) follows.
  //   T_i += L_ik W_kj: one product per 64 threads, each thread a 4 x 4 tile
  //                     (8 shared-memory loads per 16 FMAs);
  //   W = -X T:         all 512 threads, two outputs each.
  for (int e = tid; e < CBS; e += INV_THREADS) Wc[e] = Xd[e];  // W_jj = X_jj
  for (int e = tid; e < (nw - 1) * CBS; e += INV_THREADS) Tb[e] = 0.f;
  __syncthreads();
  const int pp = tid >> 6, sub = tid & 63, tr = (sub >> 3) * 4, tc = (sub & 7) * 4;
  const int r = tid >> 4, c = (tid & 15) * 2;
  for (int k = j; k < NB - 1; ++k) {
    const int i = k + 1 + pp;  // this thread's product, T_i += L_ik W_kj
    if (i < NB) {
      const float* Lk = Lb + (size_t)lidx(i, k) * CBS;
      const float* Wk = Wc + (size_t)(k - j) * CBS;
      float* Ti = Tb + (size_t)(i - j - 1) * CBS;
      float acc[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = Ti[(tr + x) * CP + tc + y];
#pragma unroll 8
      for (int t = 0; t < CBK; ++t) {
        float av[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) av[x] = Lk[(tr + x) * CP + t];
#pragma unroll
        for (int y = 0; y < 4; ++y) bv[y] = Wk[t * CP + tc + y];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) Ti[(tr + x) * CP + tc + y] = acc[x][y];
    }
    __syncthreads();
    // W_(k+1) j = -X_(k+1)(k+1) T_(k+1)
    {
      const float* Xi = Xd + (size_t)(k + 1 - j) * CBS + r * CP;
      const float* Tk = Tb + (size_t)(k - j) * CBS;
      float w0 = 0.f, w1 = 0.f;
#pragma unroll 8
      for (int u = 0; u < CBK; ++u) {
        const float xa = Xi[u];
        w0 = fmaf(xa, Tk[u * CP + c], w0);
        w1 = fmaf(xa, Tk[u * CP + c + 1], w1);
      }
      float* Wn = Wc + (size_t)(k + 1 - j) * CBS + r * CP + c;
      Wn[0] = -w0;
      Wn[1] = -w1;
    }
    __syncthreads();
  }
  // block row j of M: M(32 j + rr, col) = W(col, 32 j + rr) / d_(32 j + rr) for
  // col >= 32 j (W_ij(col - 32 i, rr)), 0 before
  for (int e = tid; e < CBK * l; e += INV_THREADS) {
    const int rr = e / l, col = e % l;
    const int row = CBK * j + rr;
    if (row >= l) continue;
    float v = 0.f;
    if (col >= CBK * j) {
      const int i = col / CBK, cc = col % CBK;
      v = Wc[(size_t)(i - j) * CBS + cc * CP + rr] * dinv[row];
    }
    M[(size_t)row * l + col] = v;
  }
}

// Floats of the Cholesky kernel's blocked factor (L blocks and the
// diagonal-block inverses, CBS entries each).
size_t chol_blocked_floats(int l) {
  const size_t NB = (l + CBK - 1) / CBK;
  return (NB * (NB + 1) / 2 + NB) * CBS;
}

size_t inv_tri_smem_bytes(int l) {
  const int NB = (l + CBK - 1) / CBK;
  const size_t nw = NB, nl = (size_t)NB * (NB - 1) / 2;
  return (2 * nw + nl + (nw - 1)) * CBS * sizeof(float);  // W, X, L, T
}

void launch_inv_tri(int l, const float* Lblk, const float* dinv, float* M, const int* gate, cudaStream_t s) {
  const int NB = (l + CBK - 1) / CBK;
  const size_t smem = inv_tri_smem_bytes(l);
  cudaFuncSetAttribute(inv_tri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  inv_tri_kernel<<<NB, INV_THREADS, smem, s>>>(l, Lblk, dinv, M, gate);
  note_launch();
}

size_t orth_tc_workspace_bytes(int rows, int l, int sms) {
  const int l8 = (l + 7) / 8 * 8;
  Carver c(nullptr);
  c.take<unsigned char>(orth_workspace_bytes(rows, l, sms, 4));
  c.take<__nv_bfloat16>((size_t)2 * rows * l8);  // Yh, Yl
  c.take<__nv_bfloat16>((size_t)2 * l * l8);     // Mh, Ml
  c.take<unsigned char>(tc_gemm_workspace(rows, l, l, sms));
  c.take<float>((size_t)l * l);                   // M = R^-1
  c.take<float>(chol_blocked_floats(l));          // the blocked factor
  return c.size();
}

// The tensor-core apply pays for an explicit triangular inverse (inv_tri_kernel,
// one CTA per block column) and the bf16 split of M; it wins once the block is
// tall.  Measured on GB300: from 64 l rows (32768 x 256 and 2^20 x 128 both
// gain; the SIMT solve wins below).
bool orth_tc_pays(int rows, int l) { return (long long)rows >= 64LL * l; }

void run_orth_tc(int rows, int l, float* Y, int ldy, double* Rout, __nv_bfloat16* Ybf, int lb, void* ws,
                 DevStatus* st, int sms, cudaStream_t s, bool intermediate) {
  intermediate = intermediate && !Rout;  // R needs every pass
  if (!orth_tc_pays(rows, l)) {
    run_orth<float, float>(rows, l, Y, ldy, Rout, Ybf, lb, ws, st, sms, s);
    return;
  }
  const int l8 = (l + 7) / 8 * 8;
  Carver c0(ws);
  void* base = c0.take<unsigned char>(orth_workspace_bytes(rows, l, sms, 4));
  __nv_bfloat16* Yh = c0.take<__nv_bfloat16>((size_t)rows * l8);
  __nv_bfloat16* Yl = c0.take<__nv_bfloat16>((size_t)rows * l8);
  __nv_bfloat16* Mh = c0.take<__nv_bfloat16>((size_t)l * l8);
  __nv_bfloat16* Ml = c0.take<__nv_bfloat16>((size_t)l * l8);
  float* part = c0.take<float>(tc_gemm_workspace(rows, l, l, sms) / sizeof(float) + 1);
  float* Minv = c0.take<float>((size_t)l * l);
  float* Lblk = c0.take<float>(chol_blocked_floats(l));
  Carver c(base);
  double* P = c.take<double>((size_t)gram_splits(rows, l, sms, 4) * l * l);
  double* G = c.take<double>((size_t)l * l);
  float* Gf = c.take<float>((size_t)l * l);
  float* M = c.take<float>((size_t)l * l);
  float* dinv = c.take<float>((size_t)l);
  double* Rp = c.take<double>((size_t)3 * l * l);
  double* Rm = c.take<double>((size_t)2 * l * l);
  const int* gate3 = &st->shifted;
  const int* run2 = &st->run2;
  // an intermediate basis: the second pass's Gram decides whether the first
  // pass's Q is kept (entries of the unit-diagonal Gram within 1/(2 (l - 1))
  // of I, so ||Gt - I||_2 <= 1/2; column norms squared within [1/2, 3/2])
  const float accept = l > 1 ? 0.5f / (float)(l - 1) : 0.f;
  for (int pass = 1; pass <= (intermediate ? 2 : 3); ++pass) {
    const int* gate = pass == 3 ? gate3 : nullptr;
    const int* gate_rest = (intermediate && pass == 2) ? run2 : gate;
    // the Gram kernel also writes the bf16 pair Yh + Yl of Y
    launch_gram<float>(rows, l, Y, ldy, P, G, Gf, sms, gate, s, nullptr, Yh, Yl, l8);
    // the factor in its blocked form (M's slot holds it), then R^-1 by block
    // columns on NB SMs
    launch_chol<float>(l, G, Gf, M, dinv, Rout ? Rp + (size_t)(pass - 1) * l * l : nullptr, st, pass, gate, s,
                       nullptr, (intermediate && pass == 2 && !Rout) ? accept : 0.f, Lblk);
    launch_inv_tri(l, Lblk, dinv, Minv, gate_rest, s);
    // pass 3 runs only if pass 1 needed a shift (a device-side gate), the
    // second pass of an intermediate basis only if its Q failed the test: a
    // gated product returns at once and leaves Y alone (the split of M only
    // fills scratch)
    launch_split_bf16(l, l, Minv, l, Mh, Ml, l8, sms, s);
    launch_tc_gemm(false, true, rows, l, l, Yh, l8, Yl, Mh, l8, Ml, Y, ldy, part, sms, st, s, 128, gate_rest);
  }
  if (Ybf) launch_copy_bf16<float>(rows, l, Y, ldy, Ybf, lb, s);
  if (Rout) {
    launch_triu_mm(l, Rp + (size_t)l * l, Rp, Rm, nullptr, 0, s, nullptr);
    launch_triu_mm(l, Rp + (size_t)2 * l * l, Rm, Rout, gate3, 1, s, nullptr);
  }
}

// G = (B + B^T) / 2 in binary64 (and rounded to binary32 for the binary32
// Cholesky), l x l.
template <typename T>
__global__ void sym_gram_kernel(int l, const T* __restrict__ B, int ldb, double* __restrict__ G,
                                float* __restrict__ Gf) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * l) return;
  const int i = idx / l, j = idx % l;
  const double v = 0.5 * ((double)B[(size_t)i * ldb + j] + (double)B[(size_t)j * ldb + i]);
  G[idx] = v;
  if (Gf) Gf[idx] = (float)v;
}

// The Nystrom factor of Fig. nystrom: B = C^T C (Cholesky of the symmetrized
// l x l matrix B, C upper triangular; the kernel's shifted restart takes a
// B that is not numerically positive definite) and Y <- Y C^-1 in place.
// Uses the same workspace as run_orth.
template <typename T, typename C>
void run_chol_solve(int rows, int l, const T* B, int ldb, T* Y, int ldy, void* ws, DevStatus* st, int sms,
                    cudaStream_t s) {
  Carver c(ws);
  c.take<double>((size_t)gram_splits(rows, l, sms, sizeof(T)) * l * l);
  double* G = c.take<double>((size_t)l * l);
  float* Gf = c.take<float>((size_t)l * l);
  C* Ub = c.take<C>((size_t)l * l);
  C* dinv = c.take<C>((size_t)l);
  sym_gram_kernel<T><<<ceil_div(l * l, 256), 256, 0, s>>>(l, B, ldb, G, sizeof(C) == 4 ? Gf : nullptr);
  note_launch();
  launch_chol<C>(l, G, Gf, Ub, dinv, nullptr, st, 1, nullptr, s, nullptr);
  launch_apply<T, C>(rows, l, Y, ldy, Ub, dinv, nullptr, 0, nullptr, s, nullptr);
}

template void run_chol_solve<float, float>(int, int, const float*, int, float*, int, void*, DevStatus*, int,
                                           cudaStream_t);
template void run_chol_solve<double, double>(int, int, const double*, int, double*, int, void*, DevStatus*, int,
                                             cudaStream_t);
template void run_orth<float, float>(int, int, float*, int, double*, __nv_bfloat16*, int, void*, DevStatus*,
                                     int, cudaStream_t, const int*);
template void run_orth<double, double>(int, int, double*, int, double*, __nv_bfloat16*, int, void*,
                                       DevStatus*, int, cudaStream_t, const int*);
template void launch_gram<float>(int, int, const float*, int, double*, double*, float*, int, const int*,
                                 cudaStream_t, const int*, __nv_bfloat16*, __nv_bfloat16*, int);
template void launch_gram<double>(int, int, const double*, int, double*, double*, float*, int, const int*,
                                  cudaStream_t, const int*, __nv_bfloat16*, __nv_bfloat16*, int);

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
  if (sizeof(T) == 4 && l % 4 == 0 && ldy % 4 == 0 && lb % 4 == 0 && (((uintptr_t)Y & 15) == 0) &&
      (((uintptr_t)Yb & 7) == 0)) {
    // binary32: the vectorized conversion (four 16-byte loads in flight per
    // thread), hi part only; its grid is capped at 8 x 256 CTAs
    launch_split_bf16(rows, l, reinterpret_cast<const float*>(Y), ldy, Yb, nullptr, lb, 256, s);
    return;
  }
  copy_bf16_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(rows, l, Y, ldy, Yb, lb);
  note_launch();
}
template void launch_copy_bf16<float>(int, int, const float*, int, __nv_bfloat16*, int, cudaStream_t);
template void launch_copy_bf16<double>(int, int, const double*, int, __nv_bfloat16*, int, cudaStream_t);

}  // namespace rsvd
