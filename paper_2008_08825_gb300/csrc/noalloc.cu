// bse_solve_chol_noalloc: the Cholesky method (Alg. 2) for one small
// problem, k lowest pairs, without any memory allocation.  The paper has no
// counterpart: this is an interface for callers that cannot allocate, e.g.
//   - code whose device memory is wholly reserved by another allocator (a
//     framework's caching pool), where a cudaMalloc would fail;
//   - latency-critical loops, where cudaMalloc/cudaFree would take a driver
//     lock and cudaFree would synchronise the whole device;
//   - services that must not meet an out-of-memory error after start-up.
// All of its device memory is one file-scope __device__ array (the scratch
// below); the host side uses fixed-size locals.  The array exists once this
// file's CUDA module is loaded on a device.  Under CUDA's default lazy module
// loading, the cudaGetSymbolAddress of the first call on a device is what
// loads it (and the solver kernel's module loads at its first launch), so the
// first call is the one that takes device memory: the 8 MiB scratch and the
// code.  Callers make it at start-up, before another allocator claims the
// memory; a call with n == 0 does only this set-up.
//
// Set-up, once per device: the first call made with a device current looks
// up the scratch's device address for that device (cudaGetSymbolAddress) and
// sets the kernel's shared-memory attribute; later calls reuse the address.
// Make that first call before any stream capture begins on the device.
//
// Calls that overlap on one device (other streams, other host threads) share
// the one scratch array and race: serialise them.
#include <atomic>

#include "kernels.cuh"

namespace {

constexpr int64_t kMaxN = BSE_NOALLOC_MAX_N;
constexpr size_t kScratchBytes = (size_t)BSE_NOALLOC_SCRATCH_BYTES;
constexpr size_t kStatusBytes = 256;  // two int64 status words, padded to keep the workspace aligned
constexpr int kMaxDevices = 64;

// layout: [status words | 256 B][instance workspace]
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::atomic<void*> g_scratch_ptr[kMaxDevices];

bse_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BSE_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return BSE_ERR_CUDA;
  void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (p) {
    *out = p;
    return BSE_OK;
  }
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return BSE_ERR_CUDA;
  }
  if (single_chol_prepare() != cudaSuccess) {
    cudaGetLastError();
    return BSE_ERR_CUDA;
  }
  g_scratch_ptr[dev].store(p, std::memory_order_release);
  *out = p;
  return BSE_OK;
}

}  // namespace

extern "C" bse_status bse_solve_chol_noalloc(int64_t n, int64_t k, const double* A, const double* B, double* omega,
                                             double* X, double* Y, bse_info* info, void* stream) {
  if (info) {
    info->info = 0;
    info->err_est = 0.0;
    info->refine_iters = 0;
    info->reserved = 0;
  }
  if (n < 0 || k < 0 || k > n) return BSE_ERR_ARG;
  if (n > kMaxN) return BSE_ERR_TOO_LARGE;
  void* base = nullptr;
  if (n == 0) return scratch_for_current_device(&base);  // set-up only
  if (k == 0) return BSE_OK;
  if (!A || !B || !omega || !X || !Y) return BSE_ERR_ARG;
  if (kStatusBytes + batched_inst_bytes(n, k) > kScratchBytes) return BSE_ERR_TOO_LARGE;
  const bse_status r = scratch_for_current_device(&base);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t* dstatus = (int64_t*)base;
  char* ws = (char*)base + kStatusBytes;
  if (single_chol_launch(s, n, k, A, B, omega, X, Y, ws, dstatus) != cudaSuccess) return BSE_ERR_CUDA;
  int64_t hstatus[2] = {0, 0};
  if (cudaMemcpyAsync(hstatus, dstatus, sizeof(hstatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return BSE_ERR_CUDA;
  }
  if (info) info->info = hstatus[1];
  return (bse_status)hstatus[0];
}
