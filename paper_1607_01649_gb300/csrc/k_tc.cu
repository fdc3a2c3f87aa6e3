// tcgen05 sketch products for the mixed-precision path (the products A G, A^T Q,
// A W and Q^T A of Fig. RSVDP_stabilized, on tensor cores):
//
//   NN:  Y[M x N] = A[M x K] X[K x N]      A bf16 row-major (K-major operand)
//   TN:  Y[M x N] = A^T[M x K] X[K x N]    A bf16 K x M row-major (MN-major operand)
//   split3:  Y = Ah^T Xh + Ah^T Xl + Al^T Xh (TN; B^T = A^T Q with A = Ah + Al,
//            Q = Xh + Xl) or Yh Mh + Yh Ml + Yl Mh (NN; the orthonormalization's
//            Q = Y R^-1), the three-term split-bf16 products.
//
// X is bf16 K x N row-major (MN-major operand), Y fp32.  N <= 256 is one MMA
// tile wide (M = 128 rows per tile, K = 64 per pipeline stage, K = 16 per MMA).
//
//   e4m3 (NN only):  Y = diag(rs) (A8 X8t^T) diag(cs), A8 M x K and X8t N x K,
//                    both e4m3 row-major (K-major operands), K = 128 bytes per
//                    stage, K = 32 per MMA (kind::f8f6f4); the row and column
//                    scales are applied in the epilogue.
//
// Persistent stream-K schedule: the T x KB (tile, k-block) units are cut into
// G equal contiguous ranges, one per CTA (G <= #SMs), so every SM streams the
// same number of bytes of A.  A tile whose k-blocks span two or more CTAs is
// written as partial sums and added in CTA order by a fix-up kernel, which
// keeps the result bitwise reproducible.
//
// Roles: warp 0 issues TMA loads into a STAGES-deep ring; warp 1 owns the
// tensor memory (two accumulators, so one tile's epilogue overlaps the next
// tile's MMAs) and issues tcgen05.mma; warps 2-5 drain TMEM to global memory.
// All waits are bounded; a timeout sets RSVD_E_TIMEOUT and the CTA winds down.
#include "common.cuh"
#include "kernels.cuh"
#include "sm100.cuh"

#include <cudaTypedefs.h>

namespace rsvd {

using namespace sm100;

struct TcArgs {
  int M, N, K;
  int KB;        // k-blocks per tile
  int T;         // tiles
  long long W;   // T * KB units
  int G;         // CTAs
  int Npad;      // MMA N (multiple of 16)
  int NA;        // TMEM columns per accumulator (power of 2 >= 32)
  int nchunk;    // 64-column TMA boxes per B tile
  int nbuf;      // TMEM accumulator sets (2: one tile's epilogue overlaps the next tile's MMAs)
  int seg;       // k-blocks per TMEM accumulation segment (see seg_end)
  float* Y;
  int ldy;
  float* part;   // [G][2][BM][Npad]
  DevStatus* st;
  const float* rs;  // e4m3: per-row scale of Y (or null)
  const float* cs;  // e4m3: per-column scale of Y
  const int* gate;  // if non-null and *gate == 0 the product is skipped (device-side control)
};

__host__ __device__ inline long long su0(long long c, long long W, int G) { return (c * W) / G; }

// The tensor core adds each MMA's products into its fp32 accumulator with
// truncation, not round-to-nearest, so a sum over many k-blocks kept in TMEM
// drifts toward zero by about half an ulp per MMA (measured: 7.9e-4 relative
// on the 2^20-row projection B^T = A^T Q, about 41k accumulating MMAs per
// CTA).  The k-blocks of a tile are therefore cut into segments that end at
// multiples of g.seg; each segment starts a fresh accumulator, and the
// epilogue adds the segments together in fp32 with round-to-nearest.
__device__ __forceinline__ int seg_end(int kb, int kb_hi, int seg) {
  const int e = (kb / seg + 1) * seg;
  return e < kb_hi ? e : kb_hi;
}

constexpr int TC_THREADS = 192;
constexpr int TC_MAX_CTAS = 256;  // persistent grid cap (>= #SMs of the part)
constexpr uint32_t A_TILE = 16384;   // 128 x 64 bf16
constexpr uint32_t B_CHUNK = 8192;   // 64 x 64 bf16

template <bool TRANS, bool SPLIT3, int SUB, bool F8 = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmX2, TcArgs g,
                   int stages) {
  static_assert(!SPLIT3 || SUB == 1, "the split-bf16 projection uses 128-row tiles");
  static_assert(!F8 || (!TRANS && !SPLIT3), "e4m3 products take K-major operands only");
  if (g.gate && *g.gate == 0) return;  // uniform over the grid, before any resource is taken
  constexpr int BM = 128 * SUB;       // rows per tile: SUB sub-tiles of 128 share each X tile
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  constexpr int NT = SPLIT3 ? 2 : 1;  // operand copies per stage
  const uint32_t b_bytes = F8 ? (uint32_t)g.Npad * 128u : (uint32_t)g.nchunk * B_CHUNK;
  const uint32_t stage_bytes = NT * (SUB * A_TILE + b_bytes);
  __shared__ uint64_t full[8], empty[8], tfull[2], tempty[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int c = blockIdx.x;
  const long long u0 = su0(c, g.W, g.G), u1 = su0(c + 1, g.W, g.G);
  const int t_first = (int)(u0 / g.KB);
  const int t_last = (int)((u1 - 1) / g.KB);

  const uint32_t tcols = (uint32_t)(g.nbuf * SUB * g.NA);  // a power of 2 <= 512
  if (warp == 1) {
    tmem_alloc(&tslot, tcols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < g.nbuf; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 128);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmX);
    if (SPLIT3) {
      tma_prefetch_desc(&tmA2);
      tma_prefetch_desc(&tmX2);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    int it = 0;
    for (int t = t_first; t <= t_last && !abort_flag; ++t) {
      const int kb_lo = (int)((t == t_first) ? u0 - (long long)t * g.KB : 0);
      const int kb_hi = (int)((t == t_last) ? u1 - (long long)t * g.KB : g.KB);
      const int m0 = t * BM;
      for (int kb = kb_lo; kb < kb_hi; ++kb, ++it) {
        const int s = it % stages;
        const uint32_t ph = (uint32_t)(it / stages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u)) {
          set_status(g.st, RSVD_E_TIMEOUT);
          abort_flag = 1;
          break;
        }
        unsigned char* sA = sm + (size_t)s * stage_bytes;
        unsigned char* sB = sA + NT * SUB * A_TILE;
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        const int k0 = kb * (F8 ? 128 : 64);
#pragma unroll
        for (int sb = 0; sb < SUB; ++sb) {
          unsigned char* sAs = sA + sb * A_TILE;
          const int ms = m0 + 128 * sb;
          if (!TRANS) {
            tma_load_2d(sAs, &tmA, k0, ms, &full[s]);
            if (SPLIT3) tma_load_2d(sAs + A_TILE, &tmA2, k0, ms, &full[s]);
          } else {
            tma_load_2d(sAs, &tmA, ms, k0, &full[s]);
            tma_load_2d(sAs + 8192, &tmA, ms + 64, k0, &full[s]);
            if (SPLIT3) {
              tma_load_2d(sAs + A_TILE, &tmA2, ms, k0, &full[s]);
              tma_load_2d(sAs + A_TILE + 8192, &tmA2, ms + 64, k0, &full[s]);
            }
          }
        }
        if (F8) {
          tma_load_2d(sB, &tmX, k0, 0, &full[s]);  // Npad rows x 128 bytes of K
        } else {
          for (int ch = 0; ch < g.nchunk; ++ch) {
            tma_load_2d(sB + ch * B_CHUNK, &tmX, 64 * ch, k0, &full[s]);
            if (SPLIT3) tma_load_2d(sB + b_bytes + ch * B_CHUNK, &tmX2, 64 * ch, k0, &full[s]);
          }
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    const uint32_t idesc = F8 ? idesc_e4m3(128, g.Npad) : idesc_bf16(128, g.Npad, TRANS ? 1 : 0, 1);
    int it = 0, j = 0;
    bool ok = true;
    for (int t = t_first; t <= t_last && ok; ++t) {
      const int kb_lo = (int)((t == t_first) ? u0 - (long long)t * g.KB : 0);
      const int kb_hi = (int)((t == t_last) ? u1 - (long long)t * g.KB : g.KB);
      for (int sg = kb_lo; sg < kb_hi && ok; ++j) {
        const int se = seg_end(sg, kb_hi, g.seg);
        const int acc = j % g.nbuf;
        const uint32_t aph = (uint32_t)(j / g.nbuf) & 1u;
        if (!mbar_wait(&tempty[acc], aph ^ 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dtm = tbase + (uint32_t)(acc * SUB * g.NA);
        for (int kb = sg; kb < se; ++kb, ++it) {
          const int s = it % stages;
          const uint32_t ph = (uint32_t)(it / stages) & 1u;
          if (!mbar_wait(&full[s], ph)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aA = smem_u32(sm + (size_t)s * stage_bytes);
          const uint32_t aB = aA + NT * SUB * A_TILE;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            // bf16: 16 K-elements (32 bytes) per MMA; e4m3: 32 K-elements (32 bytes)
            const uint64_t bd = F8 ? umma_desc(aB + 32 * k, 16, 1024) : umma_desc(aB + 2048 * k, 8192, 1024);
            const uint32_t accum = (kb > sg || k > 0) ? 1u : 0u;
#pragma unroll
            for (int sb = 0; sb < SUB; ++sb) {
              const uint32_t aAs = aA + sb * A_TILE;
              const uint64_t ad = TRANS ? umma_desc(aAs + 2048 * k, 8192, 1024) : umma_desc(aAs + 32 * k, 16, 1024);
              if (F8)
                mma_e4m3(dtm + (uint32_t)(sb * g.NA), ad, bd, idesc, accum);
              else
                mma_bf16(dtm + (uint32_t)(sb * g.NA), ad, bd, idesc, accum);
              if (SPLIT3) {
                const uint64_t ad2 = TRANS ? umma_desc(aAs + A_TILE + 2048 * k, 8192, 1024)
                                           : umma_desc(aAs + A_TILE + 32 * k, 16, 1024);
                const uint64_t bd2 = umma_desc(aB + b_bytes + 2048 * k, 8192, 1024);
                mma_bf16(dtm, ad, bd2, idesc, 1u);   // Ah^T Xl
                mma_bf16(dtm, ad2, bd, idesc, 1u);   // Al^T Xh
              }
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[acc]);
        sg = se;
      }
    }
    if (!ok) {
      set_status(g.st, RSVD_E_TIMEOUT);
      abort_flag = 1;
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp % 4;
    const int r = 32 * q + lane;
    const bool yvec = (g.ldy % 4) == 0 && (((uintptr_t)g.Y) & 15) == 0;
    int j = 0;
    bool alive = true;
    for (int t = t_first; t <= t_last && alive; ++t) {
      const int kb_lo = (int)((t == t_first) ? u0 - (long long)t * g.KB : 0);
      const int kb_hi = (int)((t == t_last) ? u1 - (long long)t * g.KB : g.KB);
      const bool whole = (kb_lo == 0 && kb_hi == g.KB);
      for (int sg = kb_lo; sg < kb_hi; ++j) {
        const int se = seg_end(sg, kb_hi, g.seg);
        const bool first = (sg == kb_lo);  // later segments add to what the earlier ones stored
        const int acc = j % g.nbuf;
        const uint32_t aph = (uint32_t)(j / g.nbuf) & 1u;
        if (!mbar_wait(&tfull[acc], aph)) {
          set_status(g.st, RSVD_E_TIMEOUT);
          abort_flag = 1;
          alive = false;
          break;
        }
        tc_fence_after();
#pragma unroll 1
        for (int sb = 0; sb < SUB; ++sb) {
          const int row = t * BM + 128 * sb + r;
          float* dst;
          bool store = true;
          if (whole) {
            dst = g.Y + (size_t)row * g.ldy;
            store = row < g.M;
          } else {
            const int slot = (t == t_first) ? 0 : 1;
            dst = g.part + (((size_t)c * 2 + slot) * BM + 128 * sb + r) * g.Npad;
          }
          const uint32_t taddr = tbase + (uint32_t)((acc * SUB + sb) * g.NA) + ((uint32_t)(32 * q) << 16);
          const float rsc = (F8 && g.rs && row < g.M) ? g.rs[row] : 1.0f;
          // columns this thread may write: Y's N, or the partial row's Npad
          const int lim = whole ? g.N : g.Npad;
          const bool v4 = !whole || yvec;  // 16-byte accesses allowed where 4 columns fit
#pragma unroll 1
          for (int c0 = 0; c0 < g.Npad; c0 += 64) {
            // what the earlier segments stored, loaded for 64 columns at once
            // before the TMEM reads, so one L2 latency covers the group
            float old[64];
            if (!first && store) {
#pragma unroll
              for (int e = 0; e < 64; e += 4) {
                const int cc = c0 + e;
                if (v4 && cc + 4 <= lim) {
                  const float4 p = *reinterpret_cast<const float4*>(dst + cc);
                  old[e] = p.x;
                  old[e + 1] = p.y;
                  old[e + 2] = p.z;
                  old[e + 3] = p.w;
                } else {
#pragma unroll
                  for (int x = 0; x < 4; ++x) old[e + x] = (cc + x < lim) ? dst[cc + x] : 0.0f;
                }
              }
            } else {
#pragma unroll
              for (int e = 0; e < 64; ++e) old[e] = 0.0f;
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int c16 = c0 + 16 * h;
              if (c16 >= g.Npad) break;  // uniform over the warp
              uint32_t v[16];
              tmem_ld16(taddr + c16, v);
              tmem_wait_ld();
              float o[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                float x = __uint_as_float(v[e]);
                if (F8) {
                  // scales are linear, so partial tiles can be scaled before the fix-up adds them
                  const float cv = (c16 + e < g.N) ? g.cs[c16 + e] : 0.0f;
                  x = x * rsc * cv;
                }
                o[e] = x + old[16 * h + e];
              }
              if (store) {
#pragma unroll
                for (int e = 0; e < 16; e += 4) {
                  const int cc = c16 + e;
                  if (v4 && cc + 4 <= lim) {
                    // 16-byte stores (each instruction still touches the 32 rows of the warp)
                    *reinterpret_cast<float4*>(dst + cc) = make_float4(o[e], o[e + 1], o[e + 2], o[e + 3]);
                  } else {
#pragma unroll
                    for (int x = 0; x < 4; ++x)
                      if (cc + x < lim) dst[cc + x] = o[e + x];
                  }
                }
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[acc]);
        sg = se;
      }
    }
  }
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) {
    // best effort: let copies and MMAs already issued land before freeing smem/TMEM
    for (int s = 0; s < stages; ++s) {
      mbar_wait(&full[s], 0, 100000000ull);
      mbar_wait(&full[s], 1, 100000000ull);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, tcols);
  }
}

// Adds the partial tiles of tiles whose k-blocks were split between CTAs, in
// CTA order.  Grid: (tile, 16-row chunk); tiles computed whole by one CTA
// return at once.  Partial rows are Npad floats (a multiple of 16), read as
// float4.
constexpr int FIX_ROWS = 16;
__global__ void __launch_bounds__(256) tc_fixup_kernel(TcArgs g, int BM) {
  if (g.gate && *g.gate == 0) return;
  const int t = blockIdx.x;
  const int r0 = blockIdx.y * FIX_ROWS;
  __shared__ int s_cf, s_cl, s_slot[TC_MAX_CTAS + 1];
  if (threadIdx.x == 0) {
    const long long ub = (long long)t * g.KB, ue = ub + g.KB - 1;
    auto cta_of = [&](long long u) {
      long long c = (u * g.G) / g.W;
      while (c + 1 < g.G && su0(c + 1, g.W, g.G) <= u) ++c;
      while (c > 0 && su0(c, g.W, g.G) > u) --c;
      return (int)c;
    };
    s_cf = cta_of(ub);
    s_cl = cta_of(ue);  // s_cl - s_cf < G <= TC_MAX_CTAS
    for (int cc = s_cf; cc <= s_cl; ++cc) s_slot[cc - s_cf] = ((int)(su0(cc, g.W, g.G) / g.KB) == t) ? 0 : 1;
  }
  __syncthreads();
  const int cf = s_cf, cl = s_cl;
  if (cf == cl) return;
  const int rows = min(FIX_ROWS, g.M - t * BM - r0);
  if (rows <= 0) return;
  const int nv = g.Npad / 4;  // float4 per partial row
  for (int e = threadIdx.x; e < rows * nv; e += blockDim.x) {
    const int r = r0 + e / nv, c4 = (e % nv) * 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int cc = cf; cc <= cl; ++cc) {
      const float4 v =
          *reinterpret_cast<const float4*>(g.part + (((size_t)cc * 2 + s_slot[cc - cf]) * BM + r) * g.Npad + c4);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    float* y = g.Y + (size_t)(t * BM + r) * g.ldy + c4;
    if (c4 + 0 < g.N) y[0] = acc.x;
    if (c4 + 1 < g.N) y[1] = acc.y;
    if (c4 + 2 < g.N) y[2] = acc.z;
    if (c4 + 3 < g.N) y[3] = acc.w;
  }
}

// -------------------------------------------------------------- host side --
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool get_encode() {
  if (g_encode) return true;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return true;
}

// bf16 row-major matrix (rows x cols, ld elements) as a 2-D map with a
// (box_in x box_out) box and 128-byte swizzle.
static bool make_map(CUtensorMap* m, const void* ptr, int cols, int rows, int ld, int box_in, int box_out) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_in, (cuuint32_t)box_out};
  cuuint32_t es[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int pow2_at_least(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

// Rows per tile the launcher picks: 256 (two sub-tiles sharing X) for the
// plain sketch when M spans at least two 256-row tiles, else 128.
int tc_rows_per_tile(int M, bool split3) { return (!split3 && M >= 512) ? 256 : 128; }

size_t tc_gemm_workspace(int M, int N, int K, int sms) {
  const int KB = ceil_div(K, 64), T = ceil_div(M, 128);  // sized for 128-row tiles: enough for 256 too
  const long long W = (long long)T * KB;
  int G = (int)(W < sms ? W : sms);
  if (G > TC_MAX_CTAS) G = TC_MAX_CTAS;
  const int Npad = ceil_div(N, 16) * 16;
  return (size_t)G * 2 * 256 * Npad * sizeof(float);
}

bool tc_supported(int N) { return N >= 1 && N <= 256; }

cudaError_t launch_tc_gemm(bool trans, bool split3, int M, int N, int K, const __nv_bfloat16* A, int lda,
                           const __nv_bfloat16* A2, const __nv_bfloat16* X, int ldx, const __nv_bfloat16* X2, float* Y,
                           int ldy, float* part, int sms, DevStatus* st, cudaStream_t s, int bm, const int* gate) {
  if (M == 0 || N == 0) return cudaSuccess;
  if (!get_encode()) return cudaErrorNotSupported;
  if ((lda % 8) || (ldx % 8) || (((uintptr_t)A | (uintptr_t)X) & 15)) return cudaErrorInvalidValue;
  if (bm <= 0) bm = tc_rows_per_tile(M, split3);
  if (split3) bm = 128;
  const int SUBT = bm / 128;
  TcArgs g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.KB = ceil_div(K, 64);
  g.T = ceil_div(M, bm);
  g.W = (long long)g.T * g.KB;
  g.G = (int)(g.W < sms ? g.W : sms);
  if (g.G > TC_MAX_CTAS) g.G = TC_MAX_CTAS;
  // short reductions (K <= 512): whole tiles per CTA when a divisor of the tile
  // count keeps at least 3/4 of the SMs busy -- no split tiles, no fix-up
  bool whole_tiles = false;
  if (g.KB <= 8 && g.T >= sms) {
    for (int gg = sms; gg * 4 >= sms * 3; --gg)
      if (g.T % gg == 0) {
        g.G = gg;
        whole_tiles = true;
        break;
      }
  }
  g.Npad = ceil_div(N, 16) * 16;
  g.NA = pow2_at_least(g.Npad);
  g.nchunk = ceil_div(N, 64);
  g.nbuf = (2 * SUBT * g.NA <= 512) ? 2 : 1;
  // TMEM segments: 1024 K for the three-term projection (192 accumulating
  // MMAs, truncation drift about 4e-6 relative); 65536 K for the plain
  // sketches, whose bf16 inputs carry 2^-9 relative rounding anyway (one
  // segment per tile up to K = 65536, drift under 1e-4 beyond)
  g.seg = split3 ? 16 : 1024;
  g.Y = Y;
  g.ldy = ldy;
  g.part = part;
  g.st = st;
  g.rs = nullptr;
  g.cs = nullptr;
  g.gate = gate;
  CUtensorMap mA, mA2, mX, mX2;
  bool ok = true;
  if (!trans)
    ok &= make_map(&mA, A, K, M, lda, 64, 128);  // A: M x K row-major
  else
    ok &= make_map(&mA, A, M, K, lda, 64, 64);   // A: K x M row-major
  ok &= make_map(&mX, X, N, K, ldx, 64, 64);     // X: K x N row-major
  if (split3) {
    if (!trans)
      ok &= make_map(&mA2, A2, K, M, lda, 64, 128);
    else
      ok &= make_map(&mA2, A2, M, K, lda, 64, 64);
    ok &= make_map(&mX2, X2, N, K, ldx, 64, 64);
  } else {
    mA2 = mA;
    mX2 = mX;
  }
  if (!ok) return cudaErrorInvalidValue;
  const int NT = split3 ? 2 : 1;
  const size_t stage_bytes = (size_t)NT * (SUBT * A_TILE + (size_t)g.nchunk * B_CHUNK);
  int stages = (int)((200 * 1024) / stage_bytes);
  if (stages > 8) stages = 8;
  if (stages < 2) return cudaErrorInvalidValue;
  const size_t smem = stages * stage_bytes + 1024;
  cudaError_t e;
#define RSVD_TC_LAUNCH(TR, SP, SB)                                                                           \
  do {                                                                                                       \
    e = cudaFuncSetAttribute(tc_gemm_kernel<TR, SP, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                          \
    tc_gemm_kernel<TR, SP, SB><<<g.G, TC_THREADS, smem, s>>>(mA, mA2, mX, mX2, g, stages);                   \
  } while (0)
  if (split3 && trans)
    RSVD_TC_LAUNCH(true, true, 1);
  else if (split3)
    RSVD_TC_LAUNCH(false, true, 1);
  else if (!trans && SUBT == 1)
    RSVD_TC_LAUNCH(false, false, 1);
  else if (!trans)
    RSVD_TC_LAUNCH(false, false, 2);
  else if (SUBT == 1)
    RSVD_TC_LAUNCH(true, false, 1);
  else
    RSVD_TC_LAUNCH(true, false, 2);
#undef RSVD_TC_LAUNCH
  note_launch();
  if (!whole_tiles) {
    tc_fixup_kernel<<<dim3(g.T, bm / FIX_ROWS), 256, 0, s>>>(g, bm);
    note_launch();
  }
  return cudaGetLastError();
}

// e4m3 matrix (rows x cols bytes, ld bytes) as a 2-D map with a
// (box_in x box_out) box and 128-byte swizzle.
static bool make_map_u8(CUtensorMap* m, const void* ptr, int cols, int rows, int ld, int box_in, int box_out) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld};
  cuuint32_t box[2] = {(cuuint32_t)box_in, (cuuint32_t)box_out};
  cuuint32_t es[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tc_gemm_e4m3_workspace(int M, int N, int K, int sms) {
  const int KB = ceil_div(K, 128), T = ceil_div(M, 128);
  const long long W = (long long)T * KB;
  int G = (int)(W < sms ? W : sms);
  if (G > TC_MAX_CTAS) G = TC_MAX_CTAS;
  const int Npad = ceil_div(N, 16) * 16;
  return (size_t)G * 2 * 256 * Npad * sizeof(float);
}

cudaError_t launch_tc_gemm_e4m3(int M, int N, int K, const uint8_t* A8, int lda, const uint8_t* X8t, int ldx,
                                const float* rs, const float* cs, float* Y, int ldy, float* part, int sms,
                                DevStatus* st, cudaStream_t s) {
  if (M == 0 || N == 0) return cudaSuccess;
  if (!get_encode()) return cudaErrorNotSupported;
  if ((lda % 16) || (ldx % 16) || (((uintptr_t)A8 | (uintptr_t)X8t) & 15) || !cs || N > 256)
    return cudaErrorInvalidValue;
  const int bm = tc_rows_per_tile(M, false);
  const int SUBT = bm / 128;
  TcArgs g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.KB = ceil_div(K, 128);
  g.T = ceil_div(M, bm);
  g.W = (long long)g.T * g.KB;
  g.G = (int)(g.W < sms ? g.W : sms);
  if (g.G > TC_MAX_CTAS) g.G = TC_MAX_CTAS;
  g.Npad = ceil_div(N, 16) * 16;
  g.NA = pow2_at_least(g.Npad);
  g.nchunk = 1;
  g.nbuf = (2 * SUBT * g.NA <= 512) ? 2 : 1;
  g.seg = 512;  // 65536 K per TMEM segment, as for the bf16 sketches
  g.Y = Y;
  g.ldy = ldy;
  g.part = part;
  g.st = st;
  g.rs = rs;
  g.cs = cs;
  g.gate = nullptr;
  CUtensorMap mA, mX;
  bool ok = make_map_u8(&mA, A8, K, M, lda, 128, 128);   // A8: M x K bytes
  ok &= make_map_u8(&mX, X8t, K, N, ldx, 128, g.Npad);     // X8t: N x K bytes
  if (!ok) return cudaErrorInvalidValue;
  const size_t stage_bytes = (size_t)SUBT * A_TILE + (size_t)g.Npad * 128;
  int stages = (int)((200 * 1024) / stage_bytes);
  if (stages > 8) stages = 8;
  if (stages < 2) return cudaErrorInvalidValue;
  const size_t smem = stages * stage_bytes + 1024;
  cudaError_t e;
  if (SUBT == 1) {
    e = cudaFuncSetAttribute(tc_gemm_kernel<false, false, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<false, false, 1, true><<<g.G, TC_THREADS, smem, s>>>(mA, mA, mX, mX, g, stages);
  } else {
    e = cudaFuncSetAttribute(tc_gemm_kernel<false, false, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<false, false, 2, true><<<g.G, TC_THREADS, smem, s>>>(mA, mA, mX, mX, g, stages);
  }
  note_launch();
  tc_fixup_kernel<<<dim3(g.T, bm / FIX_ROWS), 256, 0, s>>>(g, bm);
  note_launch();
  return cudaGetLastError();
}

// --------------------------------------------------------------- converts --
// A (fp32, rows x cols, lda) -> Ah = bf16(A), Al = bf16(A - Ah) (ld = ldb).
__global__ void split_bf16_kernel(int rows, int cols, const float* __restrict__ A, int lda,
                                  __nv_bfloat16* __restrict__ Ah, __nv_bfloat16* __restrict__ Al, int ldb) {
  const long long total = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    const float a = A[(size_t)r * lda + c];
    const __nv_bfloat16 h = __float2bfloat16_rn(a);
    Ah[(size_t)r * ldb + c] = h;
    if (Al) Al[(size_t)r * ldb + c] = __float2bfloat16_rn(a - __bfloat162float(h));
  }
}

// Vectorized variant for cols % 4 == 0, lda % 4 == 0, ldb % 4 == 0.  Each
// thread walks four interleaved grid-stride streams of float4 groups, so four
// 16-byte loads are in flight per thread; a stream's (row, column) advances by
// whole rows per stride, so no 64-bit division runs per element.
__device__ __forceinline__ void split4_store(float4 a, __nv_bfloat16* Ah, __nv_bfloat16* Al, size_t off) {
  __nv_bfloat162 h01 = __floats2bfloat162_rn(a.x, a.y), h23 = __floats2bfloat162_rn(a.z, a.w);
  uint2 hv;
  hv.x = *reinterpret_cast<uint32_t*>(&h01);
  hv.y = *reinterpret_cast<uint32_t*>(&h23);
  *reinterpret_cast<uint2*>(Ah + off) = hv;
  if (Al) {
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    __nv_bfloat162 l01 = __floats2bfloat162_rn(a.x - f01.x, a.y - f01.y);
    __nv_bfloat162 l23 = __floats2bfloat162_rn(a.z - f23.x, a.w - f23.y);
    uint2 lv;
    lv.x = *reinterpret_cast<uint32_t*>(&l01);
    lv.y = *reinterpret_cast<uint32_t*>(&l23);
    *reinterpret_cast<uint2*>(Al + off) = lv;
  }
}

__global__ void split_bf16_vec_kernel(int rows, int cols, const float* __restrict__ A, int lda,
                                      __nv_bfloat16* __restrict__ Ah, __nv_bfloat16* __restrict__ Al, int ldb) {
  constexpr int U = 4;
  const int c4 = cols / 4;
  const long long total = (long long)rows * c4;
  const long long stride = (long long)gridDim.x * blockDim.x;  // one stream's step is U strides
  const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int r[U], c[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long long e = e0 + u * stride;
    r[u] = (int)(e / c4);
    c[u] = (int)(e % c4);
  }
  const long long step = U * stride;
  const int dr = (int)(step / c4), dc = (int)(step % c4);
  for (long long e = e0; e < total; e += step) {
    float4 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e + u * stride < total) a[u] = *reinterpret_cast<const float4*>(A + (size_t)r[u] * lda + 4 * c[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e + u * stride < total) split4_store(a[u], Ah, Al, (size_t)r[u] * ldb + 4 * c[u]);
      r[u] += dr;
      c[u] += dc;
      if (c[u] >= c4) {
        c[u] -= c4;
        ++r[u];
      }
    }
  }
}

void launch_split_bf16(int rows, int cols, const float* A, int lda, __nv_bfloat16* Ah, __nv_bfloat16* Al, int ldb,
                       int sms, cudaStream_t s) {
  if ((long long)rows * cols == 0) return;
  const bool vec = (cols % 4 == 0) && (lda % 4 == 0) && (ldb % 4 == 0) && (((uintptr_t)A & 15) == 0);
  const long long units = vec ? (long long)rows * (cols / 4) : (long long)rows * cols;
  long long want = (units + 4 * 256 - 1) / (4 * 256);  // about four units per thread
  if (want < 1) want = 1;
  const int blocks = (int)(want < sms * 8 ? want : sms * 8);
  if (vec)
    split_bf16_vec_kernel<<<blocks, 256, 0, s>>>(rows, cols, A, lda, Ah, Al, ldb);
  else
    split_bf16_kernel<<<blocks, 256, 0, s>>>(rows, cols, A, lda, Ah, Al, ldb);
  note_launch();
}

}  // namespace rsvd
