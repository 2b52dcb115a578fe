// tcgen05.mma throughput probe (the measurement behind the tile shape of the
// split-operand product engine): one CTA per SM (152 CTAs, 120 KB of shared
// memory each), operands already in shared memory, R MMAs of M = 128,
// N in {64, 128, 256}, K = 16, BF16 -> FP32 into one TMEM accumulator, with A
// from shared memory or from TMEM (copied there once by tcgen05.cp); clock64
// around the issue loop and the final commit.  Every wait is bounded.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O2 -std=c++17 -o tcgen05_mma_rate tcgen05_mma_rate.cu
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)4 << 61);
}

template <int N, bool TS>
__global__ void __launch_bounds__(128, 1) rate_kernel(int R, long long* out, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* base = (unsigned char*)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);
  // A: 128 rows x 64 B (8 KB), B: N rows x 64 B
  uint64_t* bar = (uint64_t*)(base + 8192 + N * 64);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  for (int i = threadIdx.x; i < (8192 + N * 64) / 4; i += blockDim.x) ((uint32_t*)base)[i] = 0;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t da = smem_u32(base), db = da + 8192;
    if (TS) {
      asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;\n" ::"r"(tmem + 256), "l"(sdesc(da)));
      asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;\n" ::"r"(tmem + 264), "l"(sdesc(da + 32)));
    }
    const long long t0 = clock64();
    for (int r = 0; r < R; ++r) {
      const uint64_t ad = sdesc(da + (r & 1) * 32), bd = sdesc(db + (r & 1) * 32);
      if (TS)
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                     ::"r"(tmem), "r"(tmem + 256 + (r & 1) * 8), "l"(bd), "r"(idesc), "r"((uint32_t)(r > 0)));
      else
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)(r > 0)));
    }
    const long long t1 = clock64();
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
    const long long tw = clock64();
    bool ok = false;
    for (;;) {
      uint32_t done;
      asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], 0;\n selp.b32 %0, 1, 0, P;\n}\n"
                   : "=r"(done) : "r"(smem_u32(bar)) : "memory");
      if (done) { ok = true; break; }
      if (clock64() - tw > 2000000000LL) break;
    }
    const long long t2 = clock64();
    if (!ok) atomicExch(err, 1);
    out[blockIdx.x * 2] = t1 - t0;
    out[blockIdx.x * 2 + 1] = t2 - t0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
  }
}

template <int N, bool TS>
int run(int R, long long* d_out, int* d_err) {
  const int smem = 120 * 1024;  // one CTA per SM
  cudaFuncSetAttribute(rate_kernel<N, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  rate_kernel<N, TS><<<152, 128, smem>>>(R, d_out, d_err);
  if (cudaDeviceSynchronize() != cudaSuccess) { printf("kernel failed\n"); return 1; }
  long long h[304];
  cudaMemcpy(h, d_out, sizeof(h), cudaMemcpyDeviceToHost);
  int herr; cudaMemcpy(&herr, d_err, 4, cudaMemcpyDeviceToHost);
  double issue = 0, total = 0;
  for (int b = 0; b < 152; ++b) { issue += h[2 * b]; total += h[2 * b + 1]; }
  issue /= 152; total /= 152;
  printf("%s N=%3d R=%d: issue %.1f clk/MMA, complete %.1f clk/MMA, %.0f MAC/clk/SM (err %d)\n", TS ? "A tmem" : "A smem", N, R, issue / R, total / R,
         128.0 * N * 16 * R / total, herr);
  return 0;
}

int main() {
  long long* d_out; int* d_err;
  cudaMalloc(&d_out, 304 * sizeof(long long)); cudaMalloc(&d_err, 4); cudaMemset(d_err, 0, 4);
  for (int R : {16384}) {
    if (run<64, false>(R, d_out, d_err) || run<64, true>(R, d_out, d_err) || run<128, false>(R, d_out, d_err) ||
        run<128, true>(R, d_out, d_err) || run<256, true>(R, d_out, d_err))
      return 1;
  }
  return 0;
}
