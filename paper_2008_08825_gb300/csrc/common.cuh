// Shared device definitions for the BSE solver library (sm_103a).
//
// Storage convention everywhere: complex128 as double2 {re, im}, column-major,
// element (i, j) at p[i + j * ld].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bse.h"

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx mkc(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return mkc(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return mkc(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return mkc(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return mkc(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// acc += a * b  (4 DFMA)
__device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_cj(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  double d = b.x * b.x + b.y * b.y;
  return mkc((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

#define IDX2(i, j, ld) ((int64_t)(i) + (int64_t)(j) * (int64_t)(ld))

static inline unsigned ceil_div_u(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Host-side CUDA error check that returns a bse_status from the enclosing function.
#define BSE_CUDA(call)                                \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) {                          \
      bse_internal_set_error(cudaGetErrorString(e_)); \
      return BSE_ERR_CUDA;                            \
    }                                                 \
  } while (0)

#define BSE_LAUNCH_CHECK() BSE_CUDA(cudaGetLastError())

void bse_internal_set_error(const char* msg);

// Device status word layout (int64 array in workspace):
//   st[0]  error code (bse_status), 0 = OK; first writer wins
//   st[1]  info (failing column, 1-based, for NOT_PD)
struct DevStatus {
  int64_t* st;
};

__device__ __forceinline__ void dev_fail(int64_t* st, int64_t code, int64_t info) {
  if (atomicCAS((unsigned long long*)st, 0ull, (unsigned long long)code) == 0ull) st[1] = info;
}
