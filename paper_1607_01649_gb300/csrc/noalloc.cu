// rsvd_sketch_noalloc: the bf16 tensor-core sketch product (the same kernel
// rsvd_sketch runs for RSVD_MIXED_BF16) for callers that cannot allocate
// device memory -- for example code running inside another framework's
// memory pool, an allocation-free real-time loop, or a plugin that is handed
// only its input and output buffers.  The product's scratch (the stream-K
// partial tiles and the device status word) lives in a fixed array in this
// library's device image instead of a caller workspace.
//
// Limits: l <= 128 columns and at most 160 persistent CTAs (the scratch holds
// 160 x 2 x 128 x 128 fp32 partial tiles, 20 MiB, plus 256 bytes of status);
// every GPU that loads the library holds the array until the process exits.
// The array is shared by every call: calls that overlap on the GPU (on
// different streams, or from different host threads) race on it, status word
// included, and must be serialized by the caller.  The call runs on the
// current device, which must be the handle's.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int NOALLOC_MAX_L = 128;
constexpr int NOALLOC_MAX_CTAS = 160;
constexpr size_t NOALLOC_STATUS_BYTES = 256;
constexpr size_t NOALLOC_PART_FLOATS = (size_t)NOALLOC_MAX_CTAS * 2 * 128 * NOALLOC_MAX_L;
constexpr size_t NOALLOC_BYTES = NOALLOC_STATUS_BYTES + NOALLOC_PART_FLOATS * sizeof(float);

// The scratch: status block first, then the partial tiles.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_dev_ptr[MAX_DEVICES];  // device address of g_noalloc_scratch, per device

// Looks up (once per device, with that device current) the device address of
// the scratch array.  The host-side symbol is only a stand-in: its address
// must never reach a kernel.
rsvd_status scratch_for(int device, void** out) {
  if (device < 0 || device >= MAX_DEVICES) return RSVD_E_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[device]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return RSVD_E_CUDA;
    if (cur != device && cudaSetDevice(device) != cudaSuccess) return RSVD_E_CUDA;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess || p == nullptr) return RSVD_E_CUDA;
    g_dev_ptr[device] = p;
  }
  *out = g_dev_ptr[device];
  return RSVD_OK;
}

}  // namespace

int handle_device(rsvd_handle_t h);
int handle_sms(rsvd_handle_t h);
rsvd_status handle_fail(rsvd_handle_t h, rsvd_status code, const char* msg);

}  // namespace rsvd

using namespace rsvd;

extern "C" rsvd_status rsvd_sketch_noalloc(rsvd_handle_t handle, int trans, int m, int n, int l, const void* A,
                                           int lda, const void* X, int ldx, float* Y, int ldy, int* status_out,
                                           rsvd_stream_t stream) {
  if (!handle) return RSVD_E_INVALID;
  if (m < 0 || n < 0 || l < 0) return handle_fail(handle, RSVD_E_INVALID, "rsvd_sketch_noalloc: negative size");
  if (l > NOALLOC_MAX_L)
    return handle_fail(handle, RSVD_E_INVALID, "rsvd_sketch_noalloc: l exceeds the fixed scratch limit of 128 columns");
  if (lda < n || ldx < l || ldy < l)
    return handle_fail(handle, RSVD_E_INVALID, "rsvd_sketch_noalloc: leading dimension too small");
  const int M = trans ? n : m, K = trans ? m : n;
  if ((long long)M * l == 0) return RSVD_OK;
  if (!A || !X || !Y) return handle_fail(handle, RSVD_E_INVALID, "rsvd_sketch_noalloc: NULL matrix pointer");
  if ((lda % 8) || (ldx % 8) || (((uintptr_t)A | (uintptr_t)X) & 15))
    return handle_fail(handle, RSVD_E_INVALID,
                       "rsvd_sketch_noalloc: bf16 operands need 16-byte aligned rows (lda, ldx multiples of 8)");
  // the scratch array exists once per device; the kernel must run on the
  // device whose copy it writes
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return handle_fail(handle, RSVD_E_CUDA, "rsvd_sketch_noalloc: cudaGetDevice failed");
  if (cur != handle_device(handle))
    return handle_fail(handle, RSVD_E_INVALID, "rsvd_sketch_noalloc: the current device is not the handle's device");
  void* base = nullptr;
  rsvd_status st = scratch_for(handle_device(handle), &base);
  if (st != RSVD_OK) return handle_fail(handle, st, "rsvd_sketch_noalloc: cudaGetSymbolAddress failed");
  DevStatus* dst = reinterpret_cast<DevStatus*>(base);
  float* part = reinterpret_cast<float*>((unsigned char*)base + NOALLOC_STATUS_BYTES);
  cudaStream_t s = (cudaStream_t)stream;
  // the status word must start at zero; the partial tiles are written before
  // they are read within the same call
  if (cudaMemsetAsync(dst, 0, NOALLOC_STATUS_BYTES, s) != cudaSuccess)
    return handle_fail(handle, RSVD_E_CUDA, "rsvd_sketch_noalloc: status clear failed");
  int sms = handle_sms(handle);
  if (sms > NOALLOC_MAX_CTAS) sms = NOALLOC_MAX_CTAS;  // partial tiles for at most 160 CTAs
  // 128-row tiles: the fixed scratch holds two 128-row partial tiles per CTA
  const cudaError_t e = launch_tc_gemm(trans != 0, false, M, l, K, (const __nv_bfloat16*)A, lda, nullptr,
                                       (const __nv_bfloat16*)X, ldx, nullptr, Y, ldy, part, sms, dst, s, 128);
  if (e != cudaSuccess) return handle_fail(handle, RSVD_E_CUDA, "rsvd_sketch_noalloc: launch failed");
  if (cudaGetLastError() != cudaSuccess) return handle_fail(handle, RSVD_E_CUDA, "rsvd_sketch_noalloc: launch failed");
  // the device status word (RSVD_E_TIMEOUT if a bounded wait gave up) is
  // private to the library's array: copy it out for the caller, in stream order
  if (status_out && cudaMemcpyAsync(status_out, &dst->code, sizeof(int), cudaMemcpyDefault, s) != cudaSuccess)
    return handle_fail(handle, RSVD_E_CUDA, "rsvd_sketch_noalloc: status copy failed");
  return RSVD_OK;
}
