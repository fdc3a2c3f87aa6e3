// Gaussian test matrices from the Philox4x32-10 counter stream
// (the paper's "randn" that draws G in Fig. RSVD and Fig. RSVDP_stabilized).
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

// out[(j * n_groups + g) * 4 + w] = word w of counter (g, col0 + j, stream, 0).
__global__ void philox_words_kernel(int n_groups, int l, uint32_t k0, uint32_t k1, uint32_t stream,
                                    int col0, uint32_t* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n_groups * l;
  if (idx >= total) return;
  const int j = (int)(idx / n_groups);
  const int g = (int)(idx % n_groups);
  const Philox4 r = philox4x32_10((uint32_t)g, (uint32_t)(col0 + j), stream, 0u, k0, k1);
  uint4 v = make_uint4(r.x[0], r.x[1], r.x[2], r.x[3]);
  reinterpret_cast<uint4*>(out)[idx] = v;
}

template <typename T>
__device__ __forceinline__ T to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// One thread per (row group g, column j); adjacent threads take adjacent columns
// so each of the four row writes is coalesced along the row.
template <typename T>
__global__ void gaussian_f32_kernel(int n, int l, uint32_t k0, uint32_t k1, uint32_t stream,
                                    int col0, T* __restrict__ out, int ldo) {
  const int jtiles = (l + blockDim.x - 1) / blockDim.x;
  const int g = blockIdx.x / jtiles;
  const int j = (blockIdx.x % jtiles) * blockDim.x + threadIdx.x;
  if (j >= l) return;
  const Philox4 r = philox4x32_10((uint32_t)g, (uint32_t)(col0 + j), stream, 0u, k0, k1);
  float z[4];
  box_muller_f32(r.x[0], r.x[1], z[0], z[1]);
  box_muller_f32(r.x[2], r.x[3], z[2], z[3]);
  const int i0 = 4 * g;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (i0 + t < n) out[(size_t)(i0 + t) * ldo + j] = to_out<T>(z[t]);
}

__global__ void gaussian_f64_kernel(int n, int l, uint32_t k0, uint32_t k1, uint32_t stream,
                                    int col0, double* __restrict__ out, int ldo) {
  const int jtiles = (l + blockDim.x - 1) / blockDim.x;
  const int g = blockIdx.x / jtiles;
  const int j = (blockIdx.x % jtiles) * blockDim.x + threadIdx.x;
  if (j >= l) return;
  const Philox4 r = philox4x32_10((uint32_t)g, (uint32_t)(col0 + j), stream, 0u, k0, k1);
  double z[4];
  box_muller_f64(r.x[0], r.x[1], z[0], z[1]);
  box_muller_f64(r.x[2], r.x[3], z[2], z[3]);
  const int i0 = 4 * g;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (i0 + t < n) out[(size_t)(i0 + t) * ldo + j] = z[t];
}

void launch_philox_words(int n_groups, int l, uint64_t seed, uint32_t stream_id, int col0,
                         uint32_t* out, cudaStream_t s) {
  const long long total = (long long)n_groups * l;
  if (total == 0) return;
  const int threads = 256;
  const int blocks = (int)((total + threads - 1) / threads);
  philox_words_kernel<<<blocks, threads, 0, s>>>(n_groups, l, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                 stream_id, col0, out);
  note_launch();
}

void launch_gaussian(int n, int l, uint64_t seed, uint32_t stream_id, int col0, int dtype, void* out,
                     int ldo, cudaStream_t s) {
  if (n == 0 || l == 0) return;
  const int groups = (n + 3) / 4;
  const int tx = l >= 128 ? 128 : (l >= 64 ? 64 : 32);
  const long long nblk = (long long)((l + tx - 1) / tx) * groups;
  dim3 grid((unsigned)nblk);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (dtype == RSVD_DT_F64)
    gaussian_f64_kernel<<<grid, tx, 0, s>>>(n, l, k0, k1, stream_id, col0, (double*)out, ldo);
  else if (dtype == RSVD_DT_F32)
    gaussian_f32_kernel<float><<<grid, tx, 0, s>>>(n, l, k0, k1, stream_id, col0, (float*)out, ldo);
  else
    gaussian_f32_kernel<__nv_bfloat16>
        <<<grid, tx, 0, s>>>(n, l, k0, k1, stream_id, col0, (__nv_bfloat16*)out, ldo);
  note_launch();
}

}  // namespace rsvd
