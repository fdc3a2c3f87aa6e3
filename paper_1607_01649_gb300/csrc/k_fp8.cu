// Conversions for the e4m3 (FP8) sketch: the sample products of Fig.
// RSVDP_stabilized (A G, A^T Q, A W) taken with 8-bit operands.
//
//   rows:  A (fp32) -> A8 = e4m3(A_ij r_i), r_i = 448 / max_j |A_ij| (binary32),
//          s_i = 1 / r_i, so A ~ diag(s) A8; one pass over A (a warp owns a
//          row: the maximum first, then the conversion, which reads the row
//          again from L2).  The same pass can write the bf16 pair Ah + Al that
//          the split-bf16 projection B^T = A^T Q reads.
//   transpose: A8^T for the transposed product (both tcgen05 operands of an
//          e4m3 MMA are taken K-major).
//   cols:  a thin operand X (K x N), optionally row-scaled in binary32 by s
//          (X' = diag(s) X for A^T Q = A8^T (S Q)), converted per column and
//          stored transposed: X8t = e4m3(X'^T diag(r)), c_j = 1 / r_j.
// Conversion to e4m3 rounds to nearest (ties to even) and saturates at +-448.
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

namespace {

__device__ __forceinline__ uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void split_store(__nv_bfloat16* Ah, __nv_bfloat16* Al, size_t idx, float a) {
  const __nv_bfloat16 h = __float2bfloat16_rn(a);
  Ah[idx] = h;
  Al[idx] = __float2bfloat16_rn(a - __bfloat162float(h));
}

}  // namespace

// One warp per row (grid-stride).  vec: cols, lda multiples of 4 and A 16-byte
// aligned, ld8 a multiple of 4, ldb a multiple of 4.
template <bool VEC>
__global__ void __launch_bounds__(256)
    fp8_rows_kernel(int rows, int cols, const float* __restrict__ A, int lda, uint8_t* __restrict__ A8, int ld8,
                    float* __restrict__ s, __nv_bfloat16* __restrict__ Ah, __nv_bfloat16* __restrict__ Al, int ldb,
                    const float* __restrict__ amax) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < rows; i += gridDim.x * wpb) {
    const float* a = A + (size_t)i * lda;
    float mx = 0.f;
    if (VEC) {
      for (int j = 4 * lane; j < cols; j += 128) {
        const float4 v = *reinterpret_cast<const float4*>(a + j);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
    } else {
      for (int j = lane; j < cols; j += 32) mx = fmaxf(mx, fabsf(a[j]));
    }
    mx = warp_max(mx);
    if (amax) mx = amax[i];  // a maximum over a block of rows, given
    const float r = mx > 0.f ? 448.0f / mx : 1.0f;
    if (lane == 0) s[i] = 1.0f / r;
    uint8_t* q = A8 + (size_t)i * ld8;
    if (VEC) {
      for (int j = 4 * lane; j < cols; j += 128) {
        const float4 v = *reinterpret_cast<const float4*>(a + j);
        const uint32_t packed = (uint32_t)to_e4m3(v.x * r) | ((uint32_t)to_e4m3(v.y * r) << 8) |
                                ((uint32_t)to_e4m3(v.z * r) << 16) | ((uint32_t)to_e4m3(v.w * r) << 24);
        *reinterpret_cast<uint32_t*>(q + j) = packed;
        if (Ah) {
          __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
          const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
          __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
          __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
          uint2 hv, lv;
          hv.x = *reinterpret_cast<uint32_t*>(&h01);
          hv.y = *reinterpret_cast<uint32_t*>(&h23);
          lv.x = *reinterpret_cast<uint32_t*>(&l01);
          lv.y = *reinterpret_cast<uint32_t*>(&l23);
          *reinterpret_cast<uint2*>(Ah + (size_t)i * ldb + j) = hv;
          *reinterpret_cast<uint2*>(Al + (size_t)i * ldb + j) = lv;
        }
      }
    } else {
      for (int j = lane; j < cols; j += 32) {
        const float v = a[j];
        q[j] = to_e4m3(v * r);
        if (Ah) split_store(Ah, Al, (size_t)i * ldb + j, v);
      }
    }
  }
}

// The same conversion with a CTA per row for rows of at most 1024 NV
// columns: the row is read once into registers (NV 16-byte vectors per
// thread), the next row's loads are issued before this row is converted, and
// the row maximum meets in shared memory.  Same values as fp8_rows_kernel.
template <int NV>
__global__ void __launch_bounds__(256)
    fp8_rows_block_kernel(int rows, int cols, const float* __restrict__ A, int lda, uint8_t* __restrict__ A8,
                          int ld8, float* __restrict__ s, __nv_bfloat16* __restrict__ Ah,
                          __nv_bfloat16* __restrict__ Al, int ldb, const float* __restrict__ amax) {
  __shared__ float red[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4 nxt[NV];
  auto load = [&](int i, float4(&v)[NV]) {
    const float* a = A + (size_t)i * lda;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int j = 4 * (tid + 256 * u);
      v[u] = j < cols ? *reinterpret_cast<const float4*>(a + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  int i = blockIdx.x;
  if (i < rows) load(i, nxt);
  for (; i < rows; i += gridDim.x) {
    float4 cur[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) cur[u] = nxt[u];
    if (i + (int)gridDim.x < rows) load(i + gridDim.x, nxt);
    float mx = 0.f;
#pragma unroll
    for (int u = 0; u < NV; ++u)
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(cur[u].x), fabsf(cur[u].y)), fmaxf(fabsf(cur[u].z), fabsf(cur[u].w))));
    mx = warp_max(mx);
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    float m = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
    __syncthreads();  // red is rewritten for the next row
    if (amax) m = amax[i];  // a maximum over a block of rows, given
    const float r = m > 0.f ? 448.0f / m : 1.0f;
    if (tid == 0) s[i] = 1.0f / r;
    uint8_t* q = A8 + (size_t)i * ld8;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int j = 4 * (tid + 256 * u);
      if (j < cols) {
        const float4 v = cur[u];
        const uint32_t packed = (uint32_t)to_e4m3(v.x * r) | ((uint32_t)to_e4m3(v.y * r) << 8) |
                                ((uint32_t)to_e4m3(v.z * r) << 16) | ((uint32_t)to_e4m3(v.w * r) << 24);
        *reinterpret_cast<uint32_t*>(q + j) = packed;
        if (Ah) {
          __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
          const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
          __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
          __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
          uint2 hv, lv;
          hv.x = *reinterpret_cast<uint32_t*>(&h01);
          hv.y = *reinterpret_cast<uint32_t*>(&h23);
          lv.x = *reinterpret_cast<uint32_t*>(&l01);
          lv.y = *reinterpret_cast<uint32_t*>(&l23);
          *reinterpret_cast<uint2*>(Ah + (size_t)i * ldb + j) = hv;
          *reinterpret_cast<uint2*>(Al + (size_t)i * ldb + j) = lv;
        }
      }
    }
  }
}

// amax[i] = max |A| over the rows of i's block of `block` rows (and all
// columns): one CTA per block, 16-byte loads where the rows allow them.
__global__ void __launch_bounds__(256) fp8_block_max_kernel(int rows, int cols, const float* __restrict__ A, int lda,
                                                            int block, bool vec, float* __restrict__ amax) {
  __shared__ float red[8];
  const int r0 = blockIdx.x * block, r1 = min(rows, r0 + block);
  float mx = 0.f;
  if (vec) {
    const int c4 = cols / 4;
    for (int i = r0; i < r1; ++i) {
      const float4* a = reinterpret_cast<const float4*>(A + (size_t)i * lda);
      for (int j = threadIdx.x; j < c4; j += blockDim.x) {
        const float4 v = a[j];
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
    }
  } else {
    for (int i = r0; i < r1; ++i)
      for (int j = threadIdx.x; j < cols; j += blockDim.x) mx = fmaxf(mx, fabsf(A[(size_t)i * lda + j]));
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  float m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) amax[i] = m;
}

void launch_fp8_block_max(int rows, int cols, const float* A, int lda, int block, float* amax, cudaStream_t st) {
  if (rows == 0 || cols == 0) return;
  const bool vec = (cols % 4 == 0) && (lda % 4 == 0) && (((uintptr_t)A & 15) == 0);
  fp8_block_max_kernel<<<ceil_div(rows, block), 256, 0, st>>>(rows, cols, A, lda, block, vec, amax);
  note_launch();
}

void launch_fp8_rows(int rows, int cols, const float* A, int lda, uint8_t* A8, int ld8, float* s, __nv_bfloat16* Ah,
                     __nv_bfloat16* Al, int ldb, int sms, cudaStream_t st, const float* amax) {
  if (rows == 0 || cols == 0) return;
  const bool vec = (cols % 4 == 0) && (lda % 4 == 0) && (ld8 % 4 == 0) && (((uintptr_t)A & 15) == 0) &&
                   (((uintptr_t)A8 & 3) == 0) && (!Ah || (ldb % 4 == 0 && ((uintptr_t)Ah & 7) == 0 &&
                                                         ((uintptr_t)Al & 7) == 0));
  if (vec && cols <= 4096) {
    const int blocks = rows < sms * 4 ? rows : sms * 4;
    fp8_rows_block_kernel<4><<<blocks, 256, 0, st>>>(rows, cols, A, lda, A8, ld8, s, Ah, Al, ldb, amax);
    note_launch();
    return;
  }
  int blocks = ceil_div(rows, 8);
  if (blocks > sms * 16) blocks = sms * 16;
  if (vec)
    fp8_rows_kernel<true><<<blocks, 256, 0, st>>>(rows, cols, A, lda, A8, ld8, s, Ah, Al, ldb, amax);
  else
    fp8_rows_kernel<false><<<blocks, 256, 0, st>>>(rows, cols, A, lda, A8, ld8, s, Ah, Al, ldb, amax);
  note_launch();
}

// 64 x 256 byte tiles through shared memory (lda and ldt are multiples of
// 16: the padding columns of a row may be read, and bytes past `rows` in an
// output row land in its padding).  Loads: four 16-byte vectors per thread,
// all issued before any is stored.  Transpose: thread (column group g, row
// group v) reads 16 rows x 4 columns as 32-bit words, transposes each 4 x 4
// byte block with byte permutes, and writes 16 bytes of each of its 4
// output rows; the 4 threads of a column group sit in adjacent lanes, so a
// warp writes 64 contiguous bytes of 8 output rows per store.  Row r keeps
// its words rotated by 8 (r / 16) positions, which puts the 32 words a warp
// reads in 32 distinct banks.
constexpr int TR_R = 64, TR_C = 256, TR_LDW = TR_C / 4 + 4;  // row stride in 32-bit words

__device__ __forceinline__ void transpose4x4(const uint32_t (&w)[4], uint32_t (&c)[4]) {
  // word i holds row i's bytes of 4 columns; c[k] receives column k's bytes of the 4 rows
  const uint32_t t0 = __byte_perm(w[0], w[1], 0x5140), t1 = __byte_perm(w[0], w[1], 0x7362);
  const uint32_t t2 = __byte_perm(w[2], w[3], 0x5140), t3 = __byte_perm(w[2], w[3], 0x7362);
  c[0] = __byte_perm(t0, t2, 0x5410);
  c[1] = __byte_perm(t0, t2, 0x7632);
  c[2] = __byte_perm(t1, t3, 0x5410);
  c[3] = __byte_perm(t1, t3, 0x7632);
}

__global__ void __launch_bounds__(256)
    u8_transpose_kernel(int rows, int cols, const uint8_t* __restrict__ A, int lda, uint8_t* __restrict__ B, int ldt) {
  __shared__ __align__(16) uint32_t t[TR_R * TR_LDW];
  const int r0 = blockIdx.y * TR_R, c0 = blockIdx.x * TR_C;
  uint4 x[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = threadIdx.x + 256 * u;
    const int r = e >> 4, v = e & 15;  // row r, bytes 16 v .. 16 v + 15
    x[u] = make_uint4(0u, 0u, 0u, 0u);
    if (r0 + r < rows && c0 + 16 * v < lda)
      x[u] = *reinterpret_cast<const uint4*>(A + (size_t)(r0 + r) * lda + c0 + 16 * v);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = threadIdx.x + 256 * u;
    const int r = e >> 4, v = e & 15;
    *reinterpret_cast<uint4*>(&t[r * TR_LDW + ((4 * v + 8 * (r >> 4)) & 63)]) = x[u];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int g = 8 * (threadIdx.x >> 5) + (lane >> 2), v = lane & 3;  // columns 4 g .., rows 16 v ..
  const int wg = (g + 8 * v) & 63;                                    // rotated word of column group g
  uint32_t out[4][4];  // out[k][h]: column 4 g + k, rows 16 v + 4 h .. 16 v + 4 h + 3
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    uint32_t w[4], c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = t[(16 * v + 4 * h + i) * TR_LDW + wg];
    transpose4x4(w, c);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k][h] = c[k];
  }
  if (r0 + 16 * v < ldt) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = c0 + 4 * g + k;
      if (c < cols)
        *reinterpret_cast<uint4*>(B + (size_t)c * ldt + r0 + 16 * v) =
            make_uint4(out[k][0], out[k][1], out[k][2], out[k][3]);
    }
  }
}

void launch_u8_transpose(int rows, int cols, const uint8_t* A, int lda, uint8_t* B, int ldt, cudaStream_t st) {
  if (rows == 0 || cols == 0) return;
  u8_transpose_kernel<<<dim3(ceil_div(cols, TR_C), ceil_div(rows, TR_R)), 256, 0, st>>>(rows, cols, A, lda, B, ldt);
  note_launch();
}

constexpr int FC_ROWS = 1024;  // rows per partial column maximum

// Partial column maxima of X' = diag(rsc) X over FC_ROWS-row blocks.
__global__ void __launch_bounds__(256)
    fp8_colmax_kernel(int rows, int cols, const float* __restrict__ X, int ldx, const float* __restrict__ rsc,
                      float* __restrict__ part) {
  const int i0 = blockIdx.x * FC_ROWS, i1 = min(rows, i0 + FC_ROWS);
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    float mx = 0.f;
    for (int i = i0; i < i1; ++i) {
      const float v = rsc ? X[(size_t)i * ldx + c] * rsc[i] : X[(size_t)i * ldx + c];
      mx = fmaxf(mx, fabsf(v));
    }
    part[(size_t)blockIdx.x * cols + c] = mx;
  }
}

// r_j = 448 / amax_j (1 for a zero column), c_j = 1 / r_j.
__global__ void fp8_colscale_kernel(int nblk, int cols, const float* __restrict__ part, float* __restrict__ r,
                                    float* __restrict__ c) {
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    float mx = 0.f;
    for (int b = 0; b < nblk; ++b) mx = fmaxf(mx, part[(size_t)b * cols + j]);
    const float rr = mx > 0.f ? 448.0f / mx : 1.0f;
    r[j] = rr;
    c[j] = 1.0f / rr;
  }
}

// X8t (cols x rows) = e4m3(X'^T diag(r)), 64 x 64 tiles through shared memory;
// output rows are written as 16-byte vectors (ldt is a multiple of 16, so
// bytes past `rows` land in the row's padding).
__global__ void __launch_bounds__(256)
    fp8_cols_convert_kernel(int rows, int cols, const float* __restrict__ X, int ldx, const float* __restrict__ rsc,
                            const float* __restrict__ r, uint8_t* __restrict__ X8t, int ldt) {
  __shared__ __align__(16) uint8_t t[64][64 + 16];
  const int i0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int ii = e / 64, cc = e % 64;
    const int i = i0 + ii, c = c0 + cc;
    uint8_t q = 0;
    if (i < rows && c < cols) {
      const float v = rsc ? X[(size_t)i * ldx + c] * rsc[i] : X[(size_t)i * ldx + c];
      q = to_e4m3(v * r[c]);
    }
    t[ii][cc] = q;
  }
  __syncthreads();
  const int cc = threadIdx.x >> 2, v = threadIdx.x & 3;
  if (c0 + cc < cols && i0 + 16 * v < ldt) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      w[q] = (uint32_t)t[16 * v + 4 * q][cc] | ((uint32_t)t[16 * v + 4 * q + 1][cc] << 8) |
             ((uint32_t)t[16 * v + 4 * q + 2][cc] << 16) | ((uint32_t)t[16 * v + 4 * q + 3][cc] << 24);
    *reinterpret_cast<uint4*>(X8t + (size_t)(c0 + cc) * ldt + i0 + 16 * v) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

size_t fp8_cols_workspace(int rows, int cols) {
  Carver c(nullptr);
  c.take<float>((size_t)ceil_div(rows > 0 ? rows : 1, FC_ROWS) * cols);
  c.take<float>((size_t)cols);
  return c.size();
}

void launch_fp8_cols(int rows, int cols, const float* X, int ldx, const float* rsc, uint8_t* X8t, int ldt, float* c,
                     void* ws, cudaStream_t st) {
  if (rows == 0 || cols == 0) return;
  Carver cv(ws);
  const int nblk = ceil_div(rows, FC_ROWS);
  float* part = cv.take<float>((size_t)nblk * cols);
  float* r = cv.take<float>((size_t)cols);
  fp8_colmax_kernel<<<nblk, 256, 0, st>>>(rows, cols, X, ldx, rsc, part);
  fp8_colscale_kernel<<<1, 256, 0, st>>>(nblk, cols, part, r, c);
  fp8_cols_convert_kernel<<<dim3(ceil_div(cols, 64), ceil_div(rows, 64)), 256, 0, st>>>(rows, cols, X, ldx, rsc, r,
                                                                                         X8t, ldt);
  note_launch(3);
}

}  // namespace rsvd
