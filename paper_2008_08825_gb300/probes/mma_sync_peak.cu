// Throughput probe: mma.sync bf16 m16n8k16 (f32 accum), tf32 m16n8k8, f16 m16n8k16.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o mma_sync_peak mma_sync_peak.cu
#include <cstdio>
#include <cuda_runtime.h>
#define CHECK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

template <int CH>
__global__ void bf16_kernel(float* out, int iters) {
  unsigned a[4], b[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = 0x3f803f80u + threadIdx.x;
#pragma unroll
  for (int i = 0; i < 2; ++i) b[i] = 0x3f803f80u - threadIdx.x;
  float c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void tf32_kernel(float* out, int iters) {
  unsigned a[4], b[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = 0x3f800000u + threadIdx.x * 64;
#pragma unroll
  for (int i = 0; i < 2; ++i) b[i] = 0x3f800000u - threadIdx.x * 64;
  float c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void s8_kernel(int* out, int iters) {
  unsigned a[4], b[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = 0x01010101u + threadIdx.x;
#pragma unroll
  for (int i = 0; i < 2; ++i) b[i] = 0x01010101u - threadIdx.x;
  int c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                   : "+r"(c[i][0]), "+r"(c[i][1]), "+r"(c[i][2]), "+r"(c[i][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  int s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void f16_kernel(float* out, int iters) {
  unsigned a[4], b[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = 0x3c003c00u + threadIdx.x;
#pragma unroll
  for (int i = 0; i < 2; ++i) b[i] = 0x3c003c00u - threadIdx.x;
  float c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  cudaDeviceProp p;
  CHECK(cudaGetDeviceProperties(&p, 0));
  int sms = p.multiProcessorCount;
  const int threads = 256;
  int blocks = sms * 8;
  float* dout;
  CHECK(cudaMalloc(&dout, sizeof(float) * blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int warps = blocks * threads / 32;
  auto run = [&](const char* name, auto launch, double flops) -> int {
    for (int w = 0; w < 2; ++w) launch();
    CHECK(cudaDeviceSynchronize());
    float best = 1e30f, ms;
    for (int r = 0; r < 5; ++r) {
      cudaEventRecord(e0);
      launch();
      cudaEventRecord(e1);
      CHECK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    CHECK(cudaGetLastError());
    printf("%-14s %.3f ms  %.1f TFLOP/s\n", name, best, flops / (best * 1e-3) / 1e12);
    return 0;
  };
  int it = 4000;
  if (run("BF16 m16n8k16", [&] { bf16_kernel<4><<<blocks, threads>>>(dout, it); }, 4096.0 * 4 * it * warps)) return 1;
  if (run("TF32 m16n8k8", [&] { tf32_kernel<4><<<blocks, threads>>>(dout, it); }, 2048.0 * 4 * it * warps)) return 1;
  if (run("S8 m16n8k32", [&] { s8_kernel<4><<<blocks, threads>>>((int*)dout, it); }, 8192.0 * 4 * it * warps)) return 1;
  if (run("F16 m16n8k16", [&] { f16_kernel<4><<<blocks, threads>>>(dout, it); }, 4096.0 * 4 * it * warps)) return 1;
  printf("ok\n");
  return 0;
}
