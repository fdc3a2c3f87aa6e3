// Learned (l, q) controller: the probe sketch, its features, the small MLP
// (inference and training: forward, backward, Adam) and the residual judge.
//
// The paper has no learned component; what the controller is wrapped in is
// the paper's:
//   probe   Y = A G with 16 Gaussian columns (Sec. 4, Fig. RSVD with l = 16;
//           G is the first 16 columns of the Omega stream), singular values
//           of Y from its binary64 Gram matrix by cyclic Jacobi;
//   judge   E = (A - U D V^T) G with 16 columns of the certificate stream
//           (Sec. 13-14): E||E(:, i)||^2 = ||A - U D V^T||_F^2 (eq. infomm)
//           and ||A - U D V^T|| <= 10 sqrt(2/pi) max_i ||E(:, i)||
//           (Lemma thm:aposteriori, alpha = 1/10).
//
// Network: 17 -> Linear -> ReLU -> 128 -> Linear -> ReLU -> 128 -> Linear ->
// 20 logits (16 for l = 16 (c + 1), 4 for q).  Parameters in one flat binary32
// array: W1 [128][17], b1, W2 [128][128], b2, W3 [20][128], b3.
// Loss per sample: -log p_l[c*] - log p_q[q*] + lam sum_{c < c*} p_l[c].
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

constexpr int NC = 16;  // probe / judge columns
constexpr int D_IN = RSVD_CTRL_D_IN, HID = RSVD_CTRL_HIDDEN, N_OUT = RSVD_CTRL_OUT, N_L = 16, N_Q = 4;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * D_IN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + N_OUT * HID, NPARAM = OFF_B3 + N_OUT;
static_assert(NPARAM == RSVD_CTRL_PARAMS, "parameter count");
constexpr float FEAT_FLOOR = -3.0f;

// ------------------------------------------------------- thin sketch ------
// Yp[split] (m x 16) = A(:, k-range of split) G(k-range, :), and per-CTA
// partial sums of A's squares (binary32 within a thread, binary64 across
// threads).  CTA tile: 128 rows x 16 columns, k-step 32; thread (r, h) owns
// row r, columns 8h .. 8h + 7.
constexpr int TS_R = 128, TS_K = 32;

__global__ void __launch_bounds__(256)
    thin_sketch_kernel(int m, int n, const float* __restrict__ A, int lda, const float* __restrict__ G,
                       float* __restrict__ Yp, int kchunk, double* __restrict__ fro2p) {
  __shared__ float As[TS_R][TS_K + 1];
  __shared__ __align__(16) float Gs[TS_K][NC];
  __shared__ double red[8];
  const int tid = threadIdx.x, r = tid >> 1, h = tid & 1;
  const int r0 = blockIdx.x * TS_R;
  const int k0 = blockIdx.y * kchunk, k1 = min(n, k0 + kchunk);
  float acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.f;
  float sq = 0.f;
  for (int kb = k0; kb < k1; kb += TS_K) {
#pragma unroll
    for (int t = 0; t < (TS_R * TS_K) / 256; ++t) {
      const int e = tid + 256 * t;
      const int rr = e / TS_K, kk = e % TS_K;
      const int gr = r0 + rr, gk = kb + kk;
      const float v = (gr < m && gk < k1) ? A[(size_t)gr * lda + gk] : 0.f;
      As[rr][kk] = v;
      sq = fmaf(v, v, sq);
    }
#pragma unroll
    for (int t = 0; t < (TS_K * NC) / 256; ++t) {
      const int e = tid + 256 * t;
      const int kk = e / NC, c = e % NC;
      Gs[kk][c] = (kb + kk < k1) ? G[(size_t)(kb + kk) * NC + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TS_K; ++kk) {
      const float a = As[r][kk];
      const float4 g0 = *reinterpret_cast<const float4*>(&Gs[kk][8 * h]);
      const float4 g1 = *reinterpret_cast<const float4*>(&Gs[kk][8 * h + 4]);
      acc[0] = fmaf(a, g0.x, acc[0]);
      acc[1] = fmaf(a, g0.y, acc[1]);
      acc[2] = fmaf(a, g0.z, acc[2]);
      acc[3] = fmaf(a, g0.w, acc[3]);
      acc[4] = fmaf(a, g1.x, acc[4]);
      acc[5] = fmaf(a, g1.y, acc[5]);
      acc[6] = fmaf(a, g1.z, acc[6]);
      acc[7] = fmaf(a, g1.w, acc[7]);
    }
    __syncthreads();
  }
  if (r0 + r < m) {
    float* out = Yp + ((size_t)blockIdx.y * m + r0 + r) * NC + 8 * h;
#pragma unroll
    for (int c = 0; c < 8; ++c) out[c] = acc[c];
  }
  if (fro2p) {
    double v = (double)sq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w];
      fro2p[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
  }
}

// Y(i, c) = sum over splits (fixed order) of Yp.
__global__ void thin_reduce_kernel(int m, int splits, const float* __restrict__ Yp, float* __restrict__ Y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * NC) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += Yp[(size_t)z * m * NC + e];
  Y[e] = s;
}

int thin_splits(int m, int n, int sms) {
  const int tiles = ceil_div(m, TS_R);
  int s = ceil_div(4 * sms, tiles);
  const int smax = ceil_div(n, 8 * TS_K);
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  return s;
}

// Y (m x 16) = A G; fro2p (may be NULL) receives ceil(m/128) * splits partial
// sums of squares of A.  Yp: thin_splits(...) * m * 16 floats.
int launch_thin_sketch(int m, int n, const float* A, int lda, const float* G, float* Yp, float* Y, double* fro2p,
                       int sms, cudaStream_t s) {
  const int splits = thin_splits(m, n, sms);
  const int kchunk = ceil_div(ceil_div(n, splits), TS_K) * TS_K;
  const int used = ceil_div(n, kchunk);
  thin_sketch_kernel<<<dim3(ceil_div(m, TS_R), used), 256, 0, s>>>(m, n, A, lda, G, Yp, kchunk, fro2p);
  note_launch();
  thin_reduce_kernel<<<ceil_div(m * NC, 256), 256, 0, s>>>(m, used, Yp, Y);
  note_launch();
  return ceil_div(m, TS_R) * used;
}

// ------------------------------------------------------------ features ----
// One warp: cyclic Jacobi (Golub and Van Loan, Matrix Computations, Sec. 8.5,
// the two-by-two symmetric Schur step) on the 16 x 16 binary64 Gram matrix of
// the probe in the round-robin parallel order (8 disjoint rotations per
// round, 15 rounds per sweep); sigma_i = sqrt(max(lambda_i, 0)) sorted
// descending; features f_i = max(log10(sigma_{i+1} / sigma_1), -3),
// i = 0..14, f_15 = log2(m) / 16, f_16 = log2(n) / 16.
__device__ __forceinline__ void rr_pair(int round, int k, int& p, int& q) {
  // circle method on 16 players: player 15 fixed, the rest rotate
  if (k == 0) {
    p = round;
    q = 15;
  } else {
    p = (round + k) % 15;
    q = (round + 15 - k) % 15;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

__global__ void ctrl_features_kernel(int m, int n, const double* __restrict__ Gram, int nfro,
                                     const double* __restrict__ fro2p, RsvdCtrlBlock* blk) {
  __shared__ double S[NC][NC + 1];
  __shared__ double cs[8][2];
  __shared__ int pq[8][2];
  __shared__ double off;
  const int lane = threadIdx.x;
  for (int e = lane; e < NC * NC; e += 32) S[e / NC][e % NC] = Gram[e];
  __syncwarp();
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (lane == 0) {
      double o = 0.0, d = 0.0;
      for (int i = 0; i < NC; ++i) {
        d += S[i][i] * S[i][i];
        for (int j = i + 1; j < NC; ++j) o += S[i][j] * S[i][j];
      }
      off = o;
      blk->jacobi_sweeps = sweep;
      // converged when the off-diagonal mass is negligible against the diagonal
      if (!(o > 1e-30 * d)) off = -1.0;
    }
    __syncwarp();
    if (off < 0.0) break;
    for (int round = 0; round < 15; ++round) {
      if (lane < 8) {
        int p, q;
        rr_pair(round, lane, p, q);
        const double apq = S[p][q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double tau = (S[q][q] - S[p][p]) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        cs[lane][0] = c;
        cs[lane][1] = s;
        pq[lane][0] = p;
        pq[lane][1] = q;
      }
      __syncwarp();
      // rows: S <- J^T S
      for (int e = lane; e < 8 * NC; e += 32) {
        const int k = e / NC, j = e % NC;
        const int p = pq[k][0], q = pq[k][1];
        const double c = cs[k][0], s = cs[k][1];
        const double a = S[p][j], b = S[q][j];
        S[p][j] = c * a - s * b;
        S[q][j] = s * a + c * b;
      }
      __syncwarp();
      // columns: S <- S J
      for (int e = lane; e < 8 * NC; e += 32) {
        const int k = e / NC, i = e % NC;
        const int p = pq[k][0], q = pq[k][1];
        const double c = cs[k][0], s = cs[k][1];
        const double a = S[i][p], b = S[i][q];
        S[i][p] = c * a - s * b;
        S[i][q] = s * a + c * b;
      }
      __syncwarp();
    }
  }
  if (lane == 0) {
    double sig[NC];
    for (int i = 0; i < NC; ++i) sig[i] = S[i][i] > 0.0 ? sqrt(S[i][i]) : 0.0;
    for (int i = 1; i < NC; ++i) {  // insertion sort, descending
      const double v = sig[i];
      int j = i - 1;
      while (j >= 0 && sig[j] < v) {
        sig[j + 1] = sig[j];
        --j;
      }
      sig[j + 1] = v;
    }
    for (int i = 0; i < NC; ++i) blk->sigma[i] = sig[i];
    for (int i = 0; i < NC - 1; ++i) {
      float f = FEAT_FLOOR;
      if (sig[0] > 0.0 && sig[i + 1] > 0.0) f = fmaxf((float)log10(sig[i + 1] / sig[0]), FEAT_FLOOR);
      blk->feat[i] = f;
    }
    blk->feat[NC - 1] = (float)(log2((double)m) / 16.0);
    blk->feat[NC] = (float)(log2((double)n) / 16.0);
    if (fro2p) {
      double f2 = 0.0;
      for (int p = 0; p < nfro; ++p) f2 += fro2p[p];
      blk->fro2 = f2;
    }
  }
}

// ------------------------------------------------------------------ MLP ---
// One CTA of 128 threads handles up to 32 samples.  MODE 0: logits only.
// MODE 1: logits, loss and this CTA's gradient partial sums (already divided
// by the batch size), written to part[blockIdx.x][NPARAM] and lossp[blockIdx.x].
constexpr int MS = 32;  // samples per CTA

struct MlpSmem {
  float X[MS][D_IN + 1];
  float H1[MS][HID];
  float H2[MS][HID];
  float Z[MS][N_OUT];
  float dH2[MS][HID];
  float dH1[MS][HID];
  double lossv[MS];
};

template <int MODE>
__global__ void __launch_bounds__(128)
    mlp_kernel(int batch, const float* __restrict__ X, const int* __restrict__ yl, const int* __restrict__ yq,
               float lam, const float* __restrict__ th, float* __restrict__ logits, float* __restrict__ part,
               double* __restrict__ lossp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * MS;
  const int ns = min(MS, batch - s0);
  for (int e = tid; e < MS * D_IN; e += blockDim.x) {
    const int s = e / D_IN, i = e % D_IN;
    S.X[s][i] = (s < ns) ? X[(size_t)(s0 + s) * D_IN + i] : 0.f;
  }
  __syncthreads();
  // H1 = relu(W1 x + b1): thread j owns hidden unit j
  {
    const int j = tid;
    float w[D_IN];
#pragma unroll
    for (int i = 0; i < D_IN; ++i) w[i] = th[OFF_W1 + j * D_IN + i];
    const float b = th[OFF_B1 + j];
    for (int s = 0; s < MS; ++s) {
      float a = b;
#pragma unroll
      for (int i = 0; i < D_IN; ++i) a = fmaf(w[i], S.X[s][i], a);
      S.H1[s][j] = fmaxf(a, 0.f);
    }
  }
  __syncthreads();
  // H2 = relu(W2 h1 + b2)
  {
    const int j = tid;
    float acc[MS];
    const float b = th[OFF_B2 + j];
#pragma unroll
    for (int s = 0; s < MS; ++s) acc[s] = b;
    for (int k = 0; k < HID; ++k) {
      const float w = th[OFF_W2 + j * HID + k];
#pragma unroll
      for (int s = 0; s < MS; ++s) acc[s] = fmaf(w, S.H1[s][k], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < MS; ++s) S.H2[s][j] = fmaxf(acc[s], 0.f);
  }
  __syncthreads();
  // Z = W3 h2 + b3: thread t -> output o = t % 20, samples s = t / 20, + 6, ...
  if (tid < 120) {
    const int o = tid % N_OUT;
    for (int s = tid / N_OUT; s < MS; s += 6) {
      float a = th[OFF_B3 + o];
      for (int j = 0; j < HID; ++j) a = fmaf(th[OFF_W3 + o * HID + j], S.H2[s][j], a);
      S.Z[s][o] = a;
    }
  }
  __syncthreads();
  if (logits)
    for (int e = tid; e < ns * N_OUT; e += blockDim.x) logits[(size_t)(s0 + e / N_OUT) * N_OUT + e % N_OUT] =
        S.Z[e / N_OUT][e % N_OUT];
  if (MODE == 0) return;

  // softmax of both heads, the loss and dL/dZ (divided by the batch size)
  const float inv_b = 1.0f / (float)batch;
  if (tid < MS) {
    const int s = tid;
    if (s < ns) {
      // labels outside their ranges are clamped into them
      const int cl = min(max(yl[s0 + s], 0), N_L - 1), cq = min(max(yq[s0 + s], 0), N_Q - 1);
      float mx = -INFINITY;
      for (int c = 0; c < N_L; ++c) mx = fmaxf(mx, S.Z[s][c]);
      float p[N_L], sum = 0.f;
      for (int c = 0; c < N_L; ++c) {
        p[c] = expf(S.Z[s][c] - mx);
        sum += p[c];
      }
      float under = 0.f;
      for (int c = 0; c < N_L; ++c) {
        p[c] /= sum;
        if (c < cl) under += p[c];
      }
      float mq = -INFINITY;
      for (int c = 0; c < N_Q; ++c) mq = fmaxf(mq, S.Z[s][N_L + c]);
      float pqv[N_Q], sq = 0.f;
      for (int c = 0; c < N_Q; ++c) {
        pqv[c] = expf(S.Z[s][N_L + c] - mq);
        sq += pqv[c];
      }
      for (int c = 0; c < N_Q; ++c) pqv[c] /= sq;
      S.lossv[s] = -(double)logf(p[cl]) - (double)logf(pqv[cq]) + (double)lam * (double)under;
      for (int c = 0; c < N_L; ++c) {
        float d = p[c] - (c == cl ? 1.f : 0.f) + lam * p[c] * ((c < cl ? 1.f : 0.f) - under);
        S.Z[s][c] = d * inv_b;
      }
      for (int c = 0; c < N_Q; ++c) S.Z[s][N_L + c] = (pqv[c] - (c == cq ? 1.f : 0.f)) * inv_b;
    } else {
      S.lossv[s] = 0.0;
      for (int c = 0; c < N_OUT; ++c) S.Z[s][c] = 0.f;
    }
  }
  __syncthreads();
  // dH2 = (W3^T dZ) * [H2 > 0]
  {
    const int j = tid;
    float acc[MS];
#pragma unroll
    for (int s = 0; s < MS; ++s) acc[s] = 0.f;
    for (int o = 0; o < N_OUT; ++o) {
      const float w = th[OFF_W3 + o * HID + j];
#pragma unroll
      for (int s = 0; s < MS; ++s) acc[s] = fmaf(w, S.Z[s][o], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < MS; ++s) S.dH2[s][j] = S.H2[s][j] > 0.f ? acc[s] : 0.f;
  }
  __syncthreads();
  // dH1 = (W2^T dH2) * [H1 > 0]: thread k owns input unit k of layer 2
  {
    const int k = tid;
    float acc[MS];
#pragma unroll
    for (int s = 0; s < MS; ++s) acc[s] = 0.f;
    for (int j = 0; j < HID; ++j) {
      const float w = th[OFF_W2 + j * HID + k];
#pragma unroll
      for (int s = 0; s < MS; ++s) acc[s] = fmaf(w, S.dH2[s][j], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < MS; ++s) S.dH1[s][k] = S.H1[s][k] > 0.f ? acc[s] : 0.f;
  }
  __syncthreads();
  float* g = part + (size_t)blockIdx.x * NPARAM;
  {
    const int j = tid;
    // W3 and b3: gW3[o][j] = sum_s dZ[s][o] H2[s][j]
    for (int o = 0; o < N_OUT; ++o) {
      float a = 0.f;
      for (int s = 0; s < MS; ++s) a = fmaf(S.Z[s][o], S.H2[s][j], a);
      g[OFF_W3 + o * HID + j] = a;
    }
    if (j < N_OUT) {
      float a = 0.f;
      for (int s = 0; s < MS; ++s) a += S.Z[s][j];
      g[OFF_B3 + j] = a;
    }
    // W2 (row jj, column j) and b2
    for (int jj = 0; jj < HID; ++jj) {
      float a = 0.f;
#pragma unroll 8
      for (int s = 0; s < MS; ++s) a = fmaf(S.dH2[s][jj], S.H1[s][j], a);
      g[OFF_W2 + jj * HID + j] = a;
    }
    {
      float a = 0.f;
      for (int s = 0; s < MS; ++s) a += S.dH2[s][j];
      g[OFF_B2 + j] = a;
    }
    // W1 (row j) and b1
    for (int i = 0; i < D_IN; ++i) {
      float a = 0.f;
      for (int s = 0; s < MS; ++s) a = fmaf(S.dH1[s][j], S.X[s][i], a);
      g[OFF_W1 + j * D_IN + i] = a;
    }
    float a = 0.f;
    for (int s = 0; s < MS; ++s) a += S.dH1[s][j];
    g[OFF_B1 + j] = a;
  }
  if (tid == 0) {
    double l = 0.0;
    for (int s = 0; s < MS; ++s) l += S.lossv[s];
    lossp[blockIdx.x] = l;
  }
}

// Gradient = sum of the CTA partials in a fixed order (binary64).  mode 0:
// write it to grad; mode 1: one Adam step (Kingma and Ba, Algorithm 1) on th
// with moments m1, m2 at step t >= 1.  Block 0, thread 0 also sums the loss.
__global__ void mlp_reduce_kernel(int nblk, int batch, const float* __restrict__ part,
                                  const double* __restrict__ lossp, int mode, float* __restrict__ grad,
                                  float* __restrict__ th, float* __restrict__ m1, float* __restrict__ m2, int t,
                                  float lr, double* loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    double l = 0.0;
    for (int b = 0; b < nblk; ++b) l += lossp[b];
    *loss_out = l / (double)batch;
  }
  if (p >= NPARAM) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += (double)part[(size_t)b * NPARAM + p];
  const float gv = (float)s;
  if (mode == 0) {
    grad[p] = gv;
    return;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float a1 = b1 * m1[p] + (1.f - b1) * gv;
  const float a2 = b2 * m2[p] + (1.f - b2) * gv * gv;
  m1[p] = a1;
  m2[p] = a2;
  const float mh = a1 / (1.f - powf(b1, (float)t));
  const float vh = a2 / (1.f - powf(b2, (float)t));
  th[p] -= lr * mh / (sqrtf(vh) + eps);
}

size_t mlp_smem_bytes() { return sizeof(MlpSmem); }

int mlp_blocks(int batch) { return ceil_div(batch, MS); }

size_t mlp_workspace_bytes(int batch) {
  Carver c(nullptr);
  c.take<float>((size_t)mlp_blocks(batch) * NPARAM);
  c.take<double>((size_t)mlp_blocks(batch));
  return c.size();
}

cudaError_t launch_mlp(int mode, int batch, const float* X, const int* yl, const int* yq, float lam,
                       const float* th, float* logits, float* grad, float* m1, float* m2, int t, float lr,
                       double* loss_out, void* ws, cudaStream_t s) {
  // the opt-in for > 48 KB of dynamic shared memory is per device
  static std::atomic<unsigned long long> done_mask{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done_mask.load() & bit)) {
    e = cudaFuncSetAttribute(mlp_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(mlp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    if (e != cudaSuccess) return e;
    done_mask.fetch_or(bit);
  }
  const int nblk = mlp_blocks(batch);
  if (mode < 0) {  // inference only
    mlp_kernel<0><<<nblk, 128, sizeof(MlpSmem), s>>>(batch, X, nullptr, nullptr, 0.f, th, logits, nullptr,
                                                     nullptr);
    note_launch();
    return cudaGetLastError();
  }
  Carver c(ws);
  float* part = c.take<float>((size_t)nblk * NPARAM);
  double* lossp = c.take<double>((size_t)nblk);
  mlp_kernel<1><<<nblk, 128, sizeof(MlpSmem), s>>>(batch, X, yl, yq, lam, th, logits, part, lossp);
  note_launch();
  mlp_reduce_kernel<<<ceil_div(NPARAM, 256), 256, 0, s>>>(nblk, batch, part, lossp, mode, grad,
                                                           const_cast<float*>(th), m1, m2, t, lr, loss_out);
  note_launch();
  return cudaGetLastError();
}

// Decision from the logits of one sample: q = argmax of the q head (lowest
// index on ties); l = 16 (c + 1) with c the smallest class whose cumulative
// probability reaches `quantile`; clamped to [16, lmax] (a multiple of 16
// not required for lmax).
__global__ void ctrl_decide_kernel(RsvdCtrlBlock* blk, float quantile, int lmax) {
  if (threadIdx.x != 0) return;
  const float* z = blk->logits;
  float mx = -INFINITY;
  for (int c = 0; c < N_L; ++c) mx = fmaxf(mx, z[c]);
  float p[N_L], sum = 0.f;
  for (int c = 0; c < N_L; ++c) {
    p[c] = expf(z[c] - mx);
    sum += p[c];
  }
  float cum = 0.f;
  int cls = N_L - 1;
  for (int c = 0; c < N_L; ++c) {
    cum += p[c] / sum;
    if (cum >= quantile - 1e-6f) {
      cls = c;
      break;
    }
  }
  int q = 0;
  for (int c = 1; c < N_Q; ++c)
    if (z[N_L + c] > z[N_L + q]) q = c;
  int l = 16 * (cls + 1);
  if (l > lmax) l = lmax;
  blk->l_hat = l;
  blk->q_hat = q;
}

// --------------------------------------------------------------- judge ----
// Per-CTA binary64 sums of squares of E(:, c) = Yc(:, c) - sum_k U(:, k) D_k
// T(k, c) over this CTA's rows; T = V^T G (l x 16) staged with D folded in.
__global__ void __launch_bounds__(256)
    resid_cols_kernel(int m, int l, const float* __restrict__ Yc, const float* __restrict__ U, int ldu,
                      const double* __restrict__ D, const float* __restrict__ T, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ts = reinterpret_cast<float*>(smem_raw);  // l x 16
  __shared__ double red[8][NC];
  for (int e = threadIdx.x; e < l * NC; e += blockDim.x) Ts[e] = (float)D[e / NC] * T[e];
  __syncthreads();
  double acc2[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc2[c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    float w[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = 0.f;
    for (int k = 0; k < l; ++k) {
      const float u = U[(size_t)i * ldu + k];
      const float4* t4 = reinterpret_cast<const float4*>(Ts + k * NC);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = t4[q];
        w[4 * q] = fmaf(u, t.x, w[4 * q]);
        w[4 * q + 1] = fmaf(u, t.y, w[4 * q + 1]);
        w[4 * q + 2] = fmaf(u, t.z, w[4 * q + 2]);
        w[4 * q + 3] = fmaf(u, t.w, w[4 * q + 3]);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double e = (double)(Yc[(size_t)i * NC + c] - w[c]);
      acc2[c] += e * e;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double v = acc2[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < NC) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    part[(size_t)blockIdx.x * NC + threadIdx.x] = s;
  }
}

// Column norms, the Frobenius estimate, the spectral bound, acceptance
// (estimate <= safety * tol * ||A||_F) and the truncation rank: the smallest
// r with est^2 + sum_{i >= r} D_i^2 <= (safety tol ||A||_F)^2.
__global__ void judge_finalize_kernel(int nblk, const double* __restrict__ part, int l, const double* __restrict__ D,
                                      double tol, double safety, RsvdCtrlBlock* blk) {
  if (threadIdx.x != 0) return;
  double est2 = 0.0, mx = 0.0;
  for (int c = 0; c < NC; ++c) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * NC + c];
    est2 += s;
    mx = fmax(mx, s);
  }
  est2 /= (double)NC;
  blk->est2 = est2;
  blk->spec_bound = 10.0 * sqrt(2.0 / 3.14159265358979323846) * sqrt(mx);
  const double thr2 = safety * safety * tol * tol * blk->fro2;
  const int ok = (est2 <= thr2) && isfinite(est2);
  blk->accepted = ok;
  int r = l;
  if (ok) {
    double tail = 0.0;
    r = l;
    while (r > 0 && est2 + tail + D[r - 1] * D[r - 1] <= thr2) {
      tail += D[r - 1] * D[r - 1];
      --r;
    }
  }
  blk->rank = r;
}

void launch_ctrl_features(int m, int n, const double* Gram, int nfro, const double* fro2p, RsvdCtrlBlock* blk,
                          cudaStream_t s) {
  ctrl_features_kernel<<<1, 32, 0, s>>>(m, n, Gram, nfro, fro2p, blk);
  note_launch();
}

// ||A||_F^2 from the thin sketch's partial sums, in a fixed order.
__global__ void fro2_reduce_kernel(int nfro, const double* __restrict__ fro2p, RsvdCtrlBlock* blk) {
  if (threadIdx.x != 0) return;
  double f2 = 0.0;
  for (int p = 0; p < nfro; ++p) f2 += fro2p[p];
  blk->fro2 = f2;
}

void launch_fro2_reduce(int nfro, const double* fro2p, RsvdCtrlBlock* blk, cudaStream_t s) {
  fro2_reduce_kernel<<<1, 32, 0, s>>>(nfro, fro2p, blk);
  note_launch();
}

void launch_ctrl_decide(RsvdCtrlBlock* blk, float quantile, int lmax, cudaStream_t s) {
  ctrl_decide_kernel<<<1, 32, 0, s>>>(blk, quantile, lmax);
  note_launch();
}

int resid_blocks(int m, int sms) {
  int b = ceil_div(m, 256);
  return b < 2 * sms ? b : 2 * sms;
}

void launch_judge(int m, int l, const float* Yc, const float* U, int ldu, const double* D, const float* T,
                  double* part, double tol, double safety, RsvdCtrlBlock* blk, int sms, cudaStream_t s) {
  const int nb = resid_blocks(m, sms);
  resid_cols_kernel<<<nb, 256, (size_t)l * NC * sizeof(float), s>>>(m, l, Yc, U, ldu, D, T, part);
  note_launch();
  judge_finalize_kernel<<<1, 32, 0, s>>>(nb, part, l, D, tol, safety, blk);
  note_launch();
}

}  // namespace rsvd
