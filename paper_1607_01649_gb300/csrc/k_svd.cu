// Small SVD of B (Fig. RSVDP_stabilized; Sec. 3, Stage B: svd of the small matrix B).
//
// B (l x n) enters as B^T = A^T Q (n x l).  B^T is orthonormalized with the
// same CholeskyQR2 as Stage A: B^T = Q_B R_B.  Then B = R_B^T Q_B^T and the
// SVD of the l x l matrix M = R_B^T is computed by one-sided (Hestenes)
// Jacobi: M J = X with mutually orthogonal columns, X = W Sigma, so
//   B = W Sigma (Q_B J)^T,  Uhat = W,  V = Q_B J.
// Rotations on the QR factor's transpose converge in few sweeps (Drmac and
// Veselic, SIMAX 29 (2008)).
//
// The Jacobi runs in one thread-block cluster of NC CTAs.  The 2 NC column
// blocks (w columns each) follow a round-robin tournament; in every round a
// CTA sweeps all column pairs of the two blocks it holds (one warp per pair),
// then each CTA pushes its two blocks to the CTAs that need them next: one
// bulk copy per block from its shared memory into the receiver's, signalled
// on the receiver's mbarrier (one barrier per buffer parity), and one cluster
// barrier per round.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"
#include "sm100.cuh"

namespace cg = cooperative_groups;

namespace rsvd {

template <typename C>
struct JacobiTol;
template <>
struct JacobiTol<float> {
  static constexpr double u = 5.9604644775390625e-08;
};
template <>
struct JacobiTol<double> {
  static constexpr double u = 1.1102230246251565e-16;
};

// position of player i (0 <= i < P) in round r of the circle method
__device__ __forceinline__ int rr_pos(int i, int r, int P) {
  return i == 0 ? 0 : 1 + ((i - 1 + r) % (P - 1));
}
// which position holds player x in round r
__device__ __forceinline__ int rr_where(int x, int r, int P) {
  if (x == 0) return 0;
  int v = (x - 1 - r) % (P - 1);
  if (v < 0) v += P - 1;
  return 1 + v;
}

// 16-byte vectors of the working type.
template <typename C>
struct JVec;
template <>
struct JVec<float> {
  using T = float4;
  static constexpr int W = 4;
  static __device__ __forceinline__ float dot(const float4& a, const float4& b, float s) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
  }
  static __device__ __forceinline__ void rot(float4& a, float4& b, float c, float s) {
    const float4 x = a, y = b;
    a = make_float4(c * x.x - s * y.x, c * x.y - s * y.y, c * x.z - s * y.z, c * x.w - s * y.w);
    b = make_float4(s * x.x + c * y.x, s * x.y + c * y.y, s * x.z + c * y.z, s * x.w + c * y.w);
  }
};
template <>
struct JVec<double> {
  using T = double2;
  static constexpr int W = 2;
  static __device__ __forceinline__ double dot(const double2& a, const double2& b, double s) {
    return fma(a.y, b.y, fma(a.x, b.x, s));
  }
  static __device__ __forceinline__ void rot(double2& a, double2& b, double c, double s) {
    const double2 x = a, y = b;
    a = make_double2(c * x.x - s * y.x, c * x.y - s * y.y);
    b = make_double2(s * x.x + c * y.x, s * x.y + c * y.y);
  }
};

// Rotation of the pair with squared norms al, be and inner product ga
// (Rutishauser): zeta = (be - al) / (2 ga), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2).  binary32: the angle needs no
// correctly rounded division or square root (any angle near it still gives an
// orthogonal rotation; the sweep's convergence test measures what is left),
// so the hardware reciprocal square root and fast division are used.
template <typename C>
__device__ __forceinline__ void jac_rotation(C al, C be, C ga, C& t, C& c);
template <>
__device__ __forceinline__ void jac_rotation<float>(float al, float be, float ga, float& t, float& c) {
  const float zeta = __fdividef(be - al, 2.0f * ga);
  const float az = fabsf(zeta);
  const float q = 1.0f + zeta * zeta;
  const float tt = az > 1e15f ? __fdividef(0.5f, az) : __fdividef(1.0f, az + q * rsqrtf(q));
  t = zeta >= 0.0f ? tt : -tt;
  c = rsqrtf(1.0f + t * t);
}
template <>
__device__ __forceinline__ void jac_rotation<double>(double al, double be, double ga, double& t, double& c) {
  const double zeta = (be - al) / (2.0 * ga);
  const double az = fabs(zeta);
  const double tt = az > 1e15 ? 0.5 / az : 1.0 / (az + sqrt(1.0 + zeta * zeta));
  t = zeta >= 0.0 ? tt : -tt;
  c = 1.0 / sqrt(1.0 + t * t);
}

// Padded column length: a multiple of 32 lanes x one 16-byte vector.  A
// column occupies lp + W entries; entry lp holds its squared norm.
__host__ __device__ inline int jac_lp(int l, int vw) { return (l + 32 * vw - 1) / (32 * vw) * (32 * vw); }

// Buffers: four slots (two current blocks, two being received), each w
// columns of X then w columns of J.  The squared column norms are carried
// with the columns and updated by the rotation formulas (Rutishauser:
// alpha' = alpha - t gamma, beta' = beta + t gamma); they are recomputed at
// the start of every sweep.
template <typename C>
__global__ void __launch_bounds__(512)
    jacobi_cluster_kernel(int l, int w, const double* __restrict__ Rb, C* __restrict__ Wt,
                          C* __restrict__ Jt, double* __restrict__ sigma, DevStatus* st, int max_sweeps) {
  using V = typename JVec<C>::T;
  constexpr int VW = JVec<C>::W;
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int me = (int)cluster.block_rank();
  const int P = 2 * NC;
  const int lp = jac_lp(l, VW), cs = lp + VW, nv = lp / (32 * VW);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const size_t blk = (size_t)2 * w * cs;  // X then J, w columns each
  __shared__ int s_rot;
  __shared__ int s_total;
  __shared__ int s_bad;
  __shared__ __align__(8) uint64_t in_bar[2];  // incoming blocks, by buffer parity
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int nwarps = blockDim.x / 32;
  const double tol = 16.0 * sqrt((double)l) * JacobiTol<C>::u;
  const C tol2 = (C)(tol * tol);
  // pairs of the full round (circle method on 2w players), step-major
  __shared__ unsigned char s_pair[64 * 32 * 2];
  for (int e = tid; e < (2 * w - 1) * w; e += blockDim.x) {
    const int step = e / w, pr = e % w;
    s_pair[2 * e] = (unsigned char)rr_pos(pr, step, 2 * w);
    s_pair[2 * e + 1] = (unsigned char)rr_pos(2 * w - 1 - pr, step, 2 * w);
  }

  // round 0: CTA me holds players rr_pos(me, 0), rr_pos(P-1-me, 0)
  auto load_block = [&](C* dst, int bid) {
    C* X = dst;
    C* J = dst + (size_t)w * cs;
    const int total = w * cs;
    for (int e0 = tid; e0 < total; e0 += 8 * blockDim.x) {
      C v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = C(0);
        if (e < total) {
          const int cc = e / cs, r = e % cs, col = bid * w + cc;
          if (col < l && r < l) v[u] = (C)Rb[(size_t)col * l + r];  // column col of M = row col of R_B
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total) {
          const int cc = e / cs, r = e % cs, col = bid * w + cc;
          X[e] = v[u];
          J[e] = (col < l && r == col) ? C(1) : C(0);
        }
      }
    }
  };
  load_block(buf + 0 * blk, rr_pos(me, 0, P));
  load_block(buf + 1 * blk, rr_pos(P - 1 - me, 0, P));
  if (tid == 0) {
    s_total = 0;
    s_bad = 0;
    sm100::mbar_init(&in_bar[0], 1);
    sm100::mbar_init(&in_bar[1], 1);
    sm100::fence_mbar_init();
  }
  uint32_t in_phase = 0u;  // bit b: phase parity of in_bar[b]
  bool timed_out = false;
  const uint32_t blk_bytes = (uint32_t)(blk * sizeof(C));
  // every CTA's barriers exist before any block is pushed
  if (P > 2) cluster.sync();
  else __syncthreads();

  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    {  // fresh squared norms of the 2w columns this CTA holds
      const int par = (sweep * (P - 1)) & 1;
      for (int cc = warp; cc < 2 * w; cc += nwarps) {
        C* x = buf + (size_t)(2 * par + cc / w) * blk + (size_t)(cc % w) * cs;
        const V* xv = reinterpret_cast<const V*>(x);
        C a = C(0);
        for (int v = 0; v < nv; ++v) a = JVec<C>::dot(xv[v * 32 + lane], xv[v * 32 + lane], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) x[lp] = a;
      }
    }
    __syncthreads();
    for (int r = 0; r < P - 1; ++r) {
      const int par = (sweep * (P - 1) + r) & 1;
      C* top = buf + (size_t)(2 * par) * blk;
      C* bot = buf + (size_t)(2 * par + 1) * blk;
      // ---- local sweep.  Round 0 of a sweep visits every pair of the 2w
      // columns (circle method on 2w players), which covers the pairs inside
      // each block once per sweep; the other rounds visit only the w*w pairs
      // across the two blocks (step s pairs top i with bottom (i + s) mod w).
      const int Q2 = 2 * w;
      const bool full_round = (r == 0);
      const int nsteps = full_round ? Q2 - 1 : w;
      for (int step = 0; step < nsteps; ++step) {
        for (int pr = warp; pr < w; pr += nwarps) {
          int ia, ib;
          if (full_round) {
            ia = s_pair[2 * (step * w + pr)];
            ib = s_pair[2 * (step * w + pr) + 1];
          } else {
            ia = pr;
            ib = pr + step;
            if (ib >= w) ib -= w;
            ib += w;
          }
          C* xa = (ia < w ? top + (size_t)ia * cs : bot + (size_t)(ia - w) * cs);
          C* xb = (ib < w ? top + (size_t)ib * cs : bot + (size_t)(ib - w) * cs);
          V* va = reinterpret_cast<V*>(xa) + lane;
          V* vb = reinterpret_cast<V*>(xb) + lane;
          V* ja = reinterpret_cast<V*>(xa + (size_t)w * cs) + lane;
          V* jb = reinterpret_cast<V*>(xb + (size_t)w * cs) + lane;
          // the pair's X and J entries of this lane, loaded once (at most two
          // 16-byte vectors per column: l <= 256 in binary32, 128 in binary64);
          // the J loads and the carried norms are in flight during the dot product
          V a[2], b[2], pa[2], pb[2];
#pragma unroll
          for (int v = 0; v < 2; ++v)
            if (v < nv) {
              a[v] = va[32 * v];
              b[v] = vb[32 * v];
            }
#pragma unroll
          for (int v = 0; v < 2; ++v)
            if (v < nv) {
              pa[v] = ja[32 * v];
              pb[v] = jb[32 * v];
            }
          const C al = xa[lp], be = xb[lp];
          // two independent accumulation chains
          C g0 = C(0), g1 = C(0);
          g0 = JVec<C>::dot(a[0], b[0], g0);
          if (nv > 1) g1 = JVec<C>::dot(a[1], b[1], g1);
          C ga = g0 + g1;
          // xor butterflies leave the identical sum in every lane, so the
          // rotation decision below is warp-uniform without a broadcast
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
          if (al > C(0) && be > C(0) && ga * ga > tol2 * al * be) {
            // Rutishauser's formulas: zeta = (beta - alpha) / (2 gamma),
            // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t
            C t, c;
            jac_rotation<C>(al, be, ga, t, c);
            const C sn = c * t;
#pragma unroll
            for (int v = 0; v < 2; ++v)
              if (v < nv) {
                JVec<C>::rot(a[v], b[v], c, sn);
                JVec<C>::rot(pa[v], pb[v], c, sn);
                va[32 * v] = a[v];
                vb[32 * v] = b[v];
                ja[32 * v] = pa[v];
                jb[32 * v] = pb[v];
              }
            __syncwarp();
            if (lane == 0) {
              xa[lp] = al - t * ga;
              xb[lp] = be + t * ga;
              atomicAdd(&s_rot, 1);
            }
          }
        }
        __syncthreads();
      }
      // ---- exchange: push both blocks to the CTAs that hold them in the
      // next round (buffer parity par ^ 1 there).  Receivers' buffers of that
      // parity are free: their previous contents went out in the last round,
      // whose reads completed before the last cluster barrier.
      if (P > 2) {
        const int npar = par ^ 1;
        if (tid == 0) {
          sm100::fence_proxy_async_smem();  // the steps' stores, visible to the copy engine
          const int rn = (r + 1) % (P - 1);
          for (int half = 0; half < 2; ++half) {
            const int player = rr_pos(half == 0 ? me : P - 1 - me, r, P);
            const int pos_next = rr_where(player, rn, P);
            const int holder = pos_next < NC ? pos_next : P - 1 - pos_next;
            const int slot = pos_next < NC ? 0 : 1;
            const uint32_t src = sm100::smem_u32(buf + (size_t)(2 * par + half) * blk);
            const uint32_t dst_l = sm100::smem_u32(buf + (size_t)(2 * npar + slot) * blk);
            const uint32_t bar_l = sm100::smem_u32(&in_bar[npar]);
            uint32_t dst, bar;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(dst) : "r"(dst_l), "r"(holder));
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(bar) : "r"(bar_l), "r"(holder));
            asm volatile(
                "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"(dst), "r"(src), "r"(blk_bytes), "r"(bar) : "memory");
          }
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          // two blocks arrive here for the next round
          sm100::mbar_arrive_expect_tx(&in_bar[npar], 2u * blk_bytes);
          // this round's blocks may be overwritten once read
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        cluster.sync();
        // bounded wait (2 s); after a timeout the kernel runs on without
        // waiting again and reports RSVD_E_TIMEOUT
        if (!timed_out && !sm100::mbar_wait(&in_bar[npar], (in_phase >> npar) & 1u)) timed_out = true;
        in_phase ^= 1u << npar;
      } else {
        // single CTA: same two blocks; move them to the other buffer pair
        const int npar = par ^ 1;
        for (size_t e = tid; e < 2 * blk; e += blockDim.x)
          buf[(size_t)(2 * npar) * blk + e] = buf[(size_t)(2 * par) * blk + e];
        __syncthreads();
      }
    }
    // ---- convergence: total rotations of this sweep over the cluster
    if (tid == 0) {
      int* tot0 = cluster.map_shared_rank(&s_total, 0);
      atomicAdd(tot0, s_rot);
    }
    cluster.sync();
    const int total = *cluster.map_shared_rank(&s_total, 0);
    cluster.sync();
    if (me == 0 && tid == 0) s_total = 0;
    cluster.sync();
    converged = (total == 0);
    // Once a sweep rotates at most l pairs, test every pair of the current
    // columns at once instead of sweeping again to find none to rotate: the
    // fresh norms and the same dot product, summed in the same order, and the
    // same test a sweep applies (with no rotation the columns do not change
    // within a sweep, so the decision is the one a rotation-free sweep would
    // take); if no pair fails, the next sweep is skipped.
    if (!converged && total <= l) {
      const int pn = ((sweep + 1) * (P - 1)) & 1;  // the next sweep's round-0 buffers
      for (int cc = warp; cc < 2 * w; cc += nwarps) {
        C* x = buf + (size_t)(2 * pn + cc / w) * blk + (size_t)(cc % w) * cs;
        const V* xv = reinterpret_cast<const V*>(x);
        C a = C(0);
        for (int v = 0; v < nv; ++v) a = JVec<C>::dot(xv[v * 32 + lane], xv[v * 32 + lane], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) x[lp] = a;
      }
      cluster.sync();
      bool bad = false;
      // each warp takes remote columns (every CTA's two blocks) and tests
      // them against this CTA's 2w columns
      for (int rb = warp; rb < NC * 2 * w; rb += nwarps) {
        const int h = rb / (2 * w), sl = (rb % (2 * w)) / w, cb = rb % w;
        const C* xb = cluster.map_shared_rank(buf + (size_t)(2 * pn + sl) * blk + (size_t)cb * cs, h);
        const V* vb = reinterpret_cast<const V*>(xb) + lane;
        V b[2];
#pragma unroll
        for (int v = 0; v < 2; ++v)
          if (v < nv) b[v] = vb[32 * v];
        const C be = xb[lp];
        for (int oc = 0; oc < 2 * w; ++oc) {
          if (h == me && sl == oc / w && cb == oc % w) continue;  // the column itself
          const C* xa = buf + (size_t)(2 * pn + oc / w) * blk + (size_t)(oc % w) * cs;
          const V* va = reinterpret_cast<const V*>(xa) + lane;
          V a[2];
#pragma unroll
          for (int v = 0; v < 2; ++v)
            if (v < nv) a[v] = va[32 * v];
          const C al = xa[lp];
          C g0 = C(0), g1 = C(0);
          g0 = JVec<C>::dot(a[0], b[0], g0);
          if (nv > 1) g1 = JVec<C>::dot(a[1], b[1], g1);
          C ga = g0 + g1;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
          if (al > C(0) && be > C(0) && ga * ga > tol2 * al * be) bad = true;
        }
      }
      if (bad && lane == 0) atomicOr(cluster.map_shared_rank(&s_bad, 0), 1);
      cluster.sync();
      const int nbad = *cluster.map_shared_rank(&s_bad, 0);
      cluster.sync();
      if (me == 0 && tid == 0) s_bad = 0;
      cluster.sync();
      converged = (nbad == 0);
    }
  }
  if (me == 0 && tid == 0) st->jacobi_sweeps = sweep;
  if (timed_out && lane == 0) set_status(st, RSVD_E_TIMEOUT);

  // ---- outputs: after the last round the blocks sit in the buffer pair of
  // parity (sweeps * (P-1)) & 1, at round 0 positions of the tournament
  const int par = (sweep * (P - 1)) & 1;
  for (int half = 0; half < 2; ++half) {
    const int player = rr_pos(half == 0 ? me : P - 1 - me, (sweep * (P - 1)) % (P - 1), P);
    const C* X = buf + (size_t)(2 * par + half) * blk;
    const C* J = X + (size_t)w * cs;
    for (int cc = warp; cc < w; cc += nwarps) {
      const int col = player * w + cc;
      if (col >= l) continue;
      const C* x = X + (size_t)cc * cs;
      const C* jv = J + (size_t)cc * cs;
      double ss = 0.0;
      C part = C(0);
      for (int i = lane; i < l; i += 32) part = fma(x[i], x[i], part);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      ss = (double)part;
      const double sg = sqrt(ss);
      const double inv = sg > 0.0 ? 1.0 / sg : 0.0;
      // J is orthogonal in exact arithmetic; each binary32 rotation scales its
      // two columns by 1 + O(u) (the hardware reciprocal square root is not
      // correctly rounded), and over a few thousand rotations per column the
      // norms drift by up to ~1e-4 while the columns stay orthogonal, so each
      // column is rescaled to unit norm
      C jp = C(0);
      for (int i = lane; i < l; i += 32) jp = fma(jv[i], jv[i], jp);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) jp += __shfl_xor_sync(0xffffffffu, jp, o);
      const double jinv = jp > C(0) ? 1.0 / sqrt((double)jp) : 1.0;
      for (int i = lane; i < l; i += 32) {
        Wt[(size_t)col * l + i] = (C)((double)x[i] * inv);
        Jt[(size_t)col * l + i] = (C)((double)jv[i] * jinv);
      }
      if (lane == 0) sigma[col] = sg;
    }
  }
}

// Cluster size: 2 nc column blocks of w = l / (2 nc) columns.  Up to l = 256
// the portable maximum of 8 CTAs; for l >= 192 a 16-CTA cluster (a
// non-portable size) halves the warps each SM runs per step (the kernel is
// bound by instruction issue on its SMs) at the cost of twice the block
// exchanges per sweep.
static int g_jacobi_max_cluster = 16;  // lowered to 8 if a 16-CTA cluster cannot launch

int jacobi_cluster_size(int l) {
  int nc = (l + 31) / 32;
  if (l >= 192 && g_jacobi_max_cluster >= 16) nc = 16;
  else if (nc > 8) nc = 8;
  if (nc < 1) nc = 1;
  return nc;
}

size_t jacobi_smem_bytes(int l, size_t csize) {
  const int nc = jacobi_cluster_size(l);
  const int w = (l + 2 * nc - 1) / (2 * nc);
  const int vw = (int)(16 / csize);
  return (size_t)4 * 2 * w * (jac_lp(l, vw) + vw) * csize;
}

template <typename C>
cudaError_t launch_jacobi(int l, const double* Rb, C* Wt, C* Jt, double* sigma, DevStatus* st, cudaStream_t s) {
  // the kernel keeps a lane's share of a column pair in registers: at most two
  // 16-byte vectors per column (l <= 256 in binary32, l <= 128 in binary64)
  const int vw = (int)(16 / sizeof(C));
  if (l < 1 || jac_lp(l, vw) / (32 * vw) > 2) return cudaErrorInvalidValue;
  const int nc = jacobi_cluster_size(l);
  const int w = (l + 2 * nc - 1) / (2 * nc);
  const size_t smem = jacobi_smem_bytes(l, sizeof(C));
  auto kfn = jacobi_cluster_kernel<C>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc, 1, 1);
  cfg.blockDim = dim3(32 * (w < 1 ? 1 : w), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (nc > 8) {
    // a 16-CTA cluster must be allowed explicitly and must fit the part
    int ncl = 0;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&ncl, kfn, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      g_jacobi_max_cluster = 8;
      return launch_jacobi<C>(l, Rb, Wt, Jt, sigma, st, s);
    }
  }
  note_launch();
  return cudaLaunchKernelEx(&cfg, kfn, l, w, Rb, Wt, Jt, sigma, st, 40);
}

template cudaError_t launch_jacobi<float>(int, const double*, float*, float*, double*, DevStatus*, cudaStream_t);
template cudaError_t launch_jacobi<double>(int, const double*, double*, double*, double*, DevStatus*,
                                           cudaStream_t);

// ------------------------------------------------------------ sort + gather --
// perm[rank] = column with the rank-th largest sigma (ties: lower index
// first); D[rank] = sigma for rank < kk; Wsel, Jsel (l x kk row-major) hold the
// selected columns.
template <typename C>
__global__ void __launch_bounds__(256)
    sort_gather_kernel(int l, int kk, const double* __restrict__ sigma, const C* __restrict__ Wt,
                       const C* __restrict__ Jt, double* __restrict__ D, C* __restrict__ Wsel,
                       C* __restrict__ Jsel, int* __restrict__ perm) {
  // One CTA per selected column c: every CTA ranks all l values (l <= 512,
  // l^2 integer compares over the CTA), then moves its column: row src of Wt
  // and Jt (contiguous reads) into column c of Wsel and Jsel.
  __shared__ int sperm[512];
  // Keys: the IEEE bit patterns of the (non-negative) sigmas order like the
  // values; NaN maps to -1, so (key desc, index asc) is a strict total order
  // and the ranks form a permutation of 0..l-1.  Integer compares avoid
  // binary64 arithmetic.
  __shared__ long long key[512];
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double v = sigma[i];
    key[i] = (v >= 0.0) ? __double_as_longlong(v) : -1LL;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const long long ki = key[i];
    int rank = 0;
    for (int j = 0; j < l; ++j) {
      const long long kj = key[j];
      rank += (kj > ki) || (kj == ki && j < i);
    }
    sperm[rank] = i;
  }
  __syncthreads();
  const int c = blockIdx.x;
  const int src = min(max(sperm[c], 0), l - 1);
  if (threadIdx.x == 0) {
    D[c] = sigma[src];
    if (perm) perm[c] = src;
  }
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    Wsel[(size_t)i * kk + c] = Wt[(size_t)src * l + i];
    Jsel[(size_t)i * kk + c] = Jt[(size_t)src * l + i];
  }
}

template <typename C>
void launch_sort_gather(int l, int kk, const double* sigma, const C* Wt, const C* Jt, double* D, C* Wsel, C* Jsel,
                        cudaStream_t s) {
  if (kk < 1) return;
  sort_gather_kernel<C><<<kk, 256, 0, s>>>(l, kk, sigma, Wt, Jt, D, Wsel, Jsel, nullptr);
  note_launch();
}
template void launch_sort_gather<float>(int, int, const double*, const float*, const float*, double*, float*,
                                        float*, cudaStream_t);
template void launch_sort_gather<double>(int, int, const double*, const double*, const double*, double*, double*,
                                         double*, cudaStream_t);

// ------------------------------------------------------------------ signs --
// Sign convention: for column c of V (n x kk, ldv) the entry of largest
// magnitude (lowest row index on ties) is made positive, and U's column c gets
// the same sign.  Pass 1: each CTA scans a chunk of rows (coalesced along the
// row) and writes the per-column (|v|, row) maximum of its chunk.  Pass 2:
// per column, reduce the chunks, flip V's column if needed and record the
// sign, which pass 3 (the U lift) applies by scaling the selected Uhat columns.
template <typename T>
__global__ void colmax_partial_kernel(int n, int kk, const T* __restrict__ V, int ldv, int rows_per,
                                      float* __restrict__ pmax, int* __restrict__ pidx) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= kk) return;
  const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
  float best = -1.f;
  int bi = 0x7fffffff;
  for (int r = r0; r < r1; ++r) {
    const float a = fabsf((float)V[(size_t)r * ldv + c]);
    if (a > best) {
      best = a;
      bi = r;
    }
  }
  pmax[(size_t)blockIdx.x * kk + c] = best;
  pidx[(size_t)blockIdx.x * kk + c] = bi;
}

// Pass 2, one CTA per column: the CTA reduces the chunk maxima in parallel
// (ties to the lowest row), decides the column's sign, flips Wsel's column and
// records the decision in flip[c]; colflip_kernel then flips V with row-wise
// (coalesced) accesses.
template <typename T, typename C>
__global__ void __launch_bounds__(256)
    colsign_kernel(int n, int kk, int chunks, const float* __restrict__ pmax, const int* __restrict__ pidx,
                   const T* __restrict__ V, int ldv, C* __restrict__ Wsel, int l, int* __restrict__ flip) {
  const int c = blockIdx.x;
  __shared__ float s_b[8];
  __shared__ int s_i[8];
  __shared__ int s_flip;
  float best = -1.f;
  int bi = 0x7fffffff;
  for (int z = threadIdx.x; z < chunks; z += blockDim.x) {
    const float b = pmax[(size_t)z * kk + c];
    const int i = pidx[(size_t)z * kk + c];
    if (b > best || (b == best && i < bi)) {
      best = b;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float b = __shfl_down_sync(0xffffffffu, best, o);
    const int i = __shfl_down_sync(0xffffffffu, bi, o);
    if (b > best || (b == best && i < bi)) {
      best = b;
      bi = i;
    }
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    s_b[warp] = best;
    s_i[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x / 32); ++w)
      if (s_b[w] > best || (s_b[w] == best && s_i[w] < bi)) {
        best = s_b[w];
        bi = s_i[w];
      }
    s_flip = (bi < n && V[(size_t)bi * ldv + c] < T(0)) ? 1 : 0;
    flip[c] = s_flip;
  }
  __syncthreads();
  if (!s_flip) return;
  for (int i = threadIdx.x; i < l; i += blockDim.x) Wsel[(size_t)i * kk + c] = -Wsel[(size_t)i * kk + c];
}

// Pass 2b: V(i, c) = -V(i, c) for the flipped columns, rows walked with the
// columns fastest.
template <typename T>
__global__ void colflip_kernel(int n, int kk, T* __restrict__ V, int ldv, const int* __restrict__ flip) {
  const long long total = (long long)n * kk;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / kk), c = (int)(e % kk);
    if (flip[c]) V[(size_t)i * ldv + c] = -V[(size_t)i * ldv + c];
  }
}

size_t sign_workspace_bytes(int n, int kk) {
  const int chunks = (n + 255) / 256;
  return (size_t)chunks * kk * (sizeof(float) + sizeof(int)) + (size_t)kk * sizeof(int) + 1024;
}

template <typename T, typename C>
void launch_sign_fix(int n, int kk, int l, T* V, int ldv, C* Wsel, void* ws, cudaStream_t s) {
  if (kk == 0 || n == 0) return;
  const int rows_per = 256;
  const int chunks = (n + rows_per - 1) / rows_per;
  float* pmax = (float*)ws;
  const size_t off_i = ((size_t)chunks * kk * sizeof(float) + 255) & ~(size_t)255;
  int* pidx = (int*)((char*)ws + off_i);
  int* flip = (int*)((char*)ws + ((off_i + (size_t)chunks * kk * sizeof(int) + 255) & ~(size_t)255));
  const int tx = kk >= 128 ? 128 : 64;
  dim3 grid(chunks, (kk + tx - 1) / tx);
  colmax_partial_kernel<T><<<grid, tx, 0, s>>>(n, kk, V, ldv, rows_per, pmax, pidx);
  note_launch();
  colsign_kernel<T, C><<<kk, 256, 0, s>>>(n, kk, chunks, pmax, pidx, V, ldv, Wsel, l, flip);
  note_launch();
  const long long total = (long long)n * kk;
  const long long want = (total + 4 * 256 - 1) / (4 * 256);
  const int blocks = (int)(want < 4096 ? want : 4096);
  colflip_kernel<T><<<blocks, 256, 0, s>>>(n, kk, V, ldv, flip);
  note_launch();
}
template void launch_sign_fix<float, float>(int, int, int, float*, int, float*, void*, cudaStream_t);
template void launch_sign_fix<double, double>(int, int, int, double*, int, double*, void*, cudaStream_t);

}  // namespace rsvd
