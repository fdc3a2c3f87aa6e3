// Shared device/host helpers of the randomized-SVD library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/rsvd.h"

namespace rsvd {

// ----------------------------------------------------------------- status --
// The device status block lives at the start of every workspace.
struct DevStatus {
  int code;         // rsvd_status of the first device-side failure (0 = OK)
  int shifted;      // orth: the current CholeskyQR needed a shifted first pass
  int passes;       // orth: CholeskyQR passes still to run (device-driven)
  int jacobi_sweeps;
  int rank;         // adaptive: current rank
  int done;         // adaptive: tolerance met / loop finished
  int shift_count;  // Cholesky factorizations that needed a diagonal shift
  int run2;         // orth: an intermediate basis needs its second CholeskyQR pass
                    // (0: the first pass already gives a basis within the
                    // acceptance bound, which is kept)
  double fro2_a;    // adaptive: ||A||_Fro^2
  double fro2_res;  // adaptive: ||A_j||_Fro^2 of the current remainder
  double scratch[6];
};
static_assert(sizeof(DevStatus) <= 256, "status block fits its slot");

// Device-side record of one controller decision (probe, network, judge).
struct RsvdCtrlBlock {
  int l_hat, q_hat;       // the network's choice
  int accepted;           // judge: residual estimate within tolerance
  int rank;               // judge: truncation rank
  int jacobi_sweeps;      // probe: sweeps of the 16 x 16 eigen-solve
  int pad[3];
  double fro2;            // ||A||_F^2
  double est2;            // mean_i ||E(:, i)||^2 (Frobenius estimate, squared)
  double spec_bound;      // 10 sqrt(2/pi) max_i ||E(:, i)||
  double pad2;
  double sigma[16];       // probe singular values, descending
  float feat[RSVD_CTRL_D_IN];
  float logits[RSVD_CTRL_OUT];
};

__device__ __forceinline__ void set_status(DevStatus* st, int code) {
  atomicCAS(&st->code, 0, code);
}

// ----------------------------------------------------------------- philox --
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (c0..c3), key
// (k0, k1); a round maps (c0, c1, c2, c3) to
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// and the key advances by the Weyl increments after each round.
struct Philox4 {
  uint32_t x[4];
};

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                          uint32_t c3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c0;
    const uint64_t p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  Philox4 o;
  o.x[0] = c0;
  o.x[1] = c1;
  o.x[2] = c2;
  o.x[3] = c3;
  return o;
}

// 24-bit Box-Muller pair in binary32.
__device__ __forceinline__ void box_muller_f32(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float u1 = (float)((wa >> 8) + 1u) * 5.9604644775390625e-08f;  // 2^-24, exact
  const float u2 = (float)(wb >> 8) * 5.9604644775390625e-08f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);  // sin/cos of 2 pi u2; 2 u2 is exact
  z0 = r * c;
  z1 = r * s;
}

// 24-bit Box-Muller pair in binary64.
__device__ __forceinline__ void box_muller_f64(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  const double u1 = (double)((wa >> 8) + 1u) * 5.9604644775390625e-08;
  const double u2 = (double)(wb >> 8) * 5.9604644775390625e-08;
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// --------------------------------------------------------- launch counter --
// Number of kernels the library has enqueued since it was loaded.
inline std::atomic<long long>& launch_counter() {
  static std::atomic<long long> c{0};
  return c;
}
inline void note_launch(long long n = 1) { launch_counter().fetch_add(n, std::memory_order_relaxed); }

// ------------------------------------------------------------- workspace --
// Bump allocator over the caller's workspace; every slice is 256-byte aligned.
struct Carver {
  char* base;
  size_t off;
  explicit Carver(void* b) : base((char*)b), off(0) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return (off + 255) & ~(size_t)255; }
};

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

template <typename T>
struct TypeName;

}  // namespace rsvd
