// Throughput probe: FP64 DFMA, FP32 FFMA, FP64 mma.sync (m8n8k4, m16n8k4/k8/k16).
// Every thread writes exactly one element of `out` (sized grid*block), nothing else.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_fp32_peak fp64_fp32_peak.cu
#include <cstdio>
#include <cuda_runtime.h>

#define CHECK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

template <int CH>
__global__ void dfma_kernel(double* out, int iters, double a, double b) {
  double acc[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) acc[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i) acc[i] = fma(acc[i], a, b);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void ffma_kernel(float* out, int iters, float a, float b) {
  float acc[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) acc[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i) acc[i] = fmaf(acc[i], a, b);
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// m8n8k4 f64: A 1 reg, B 1 reg, C/D 2 regs per thread.
template <int CH>
__global__ void dmma884_kernel(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-6, b = 1.0 - threadIdx.x * 1e-6;
  double c[CH][2];
#pragma unroll
  for (int i = 0; i < CH; ++i) { c[i][0] = 0; c[i][1] = 0; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// m16n8k16 f64: A 8 regs, B 4 regs, C/D 4 regs.
template <int CH>
__global__ void dmma16816_kernel(double* out, int iters) {
  double a[8], b[4];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1.0 + (threadIdx.x + i) * 1e-6;
#pragma unroll
  for (int i = 0; i < 4; ++i) b[i] = 1.0 - (threadIdx.x + i) * 1e-6;
  double c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) { c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
                   : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
                   : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                     "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// m16n8k4 f64: A 2 regs, B 1 reg, C/D 4 regs.
template <int CH>
__global__ void dmma1684_kernel(double* out, int iters) {
  double a0 = 1.0 + threadIdx.x * 1e-6, a1 = 1.0 + threadIdx.x * 2e-6, b = 1.0 - threadIdx.x * 1e-6;
  double c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) { c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
                   : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
                   : "d"(a0), "d"(a1), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  cudaDeviceProp p;
  CHECK(cudaGetDeviceProperties(&p, 0));
  int sms = p.multiProcessorCount;
  printf("device %s sms=%d cc=%d.%d\n", p.name, sms, p.major, p.minor);
  const int threads = 256;
  int blocks = sms * 8;
  double* dout;
  CHECK(cudaMalloc(&dout, sizeof(double) * blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms;
  auto run = [&](const char* name, auto launch, double flops_per_launch) -> int {
    for (int w = 0; w < 2; ++w) launch();
    CHECK(cudaDeviceSynchronize());
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
      cudaEventRecord(e0);
      launch();
      cudaEventRecord(e1);
      CHECK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    CHECK(cudaGetLastError());
    printf("%-12s %.3f ms  %.2f TFLOP/s\n", name, best, flops_per_launch / (best * 1e-3) / 1e12);
    return 0;
  };
  int it_d = 2000;
  if (run("DFMA", [&] { dfma_kernel<8><<<blocks, threads>>>(dout, it_d, 0.999999, 1e-7); },
          2.0 * 8 * it_d * (double)blocks * threads)) return 1;
  int it_f = 20000;
  if (run("FFMA", [&] { ffma_kernel<8><<<blocks, threads>>>((float*)dout, it_f, 0.999999f, 1e-7f); },
          2.0 * 8 * it_f * (double)blocks * threads)) return 1;
  // per warp per mma m8n8k4: 8*8*4*2 = 512 flops
  int it_m = 1000;
  int warps = blocks * threads / 32;
  if (run("DMMA884", [&] { dmma884_kernel<4><<<blocks, threads>>>(dout, it_m); },
          512.0 * 4 * it_m * warps)) return 1;
  if (run("DMMA1684", [&] { dmma1684_kernel<4><<<blocks, threads>>>(dout, it_m); },
          1024.0 * 4 * it_m * warps)) return 1;
  if (run("DMMA16816", [&] { dmma16816_kernel<4><<<blocks, threads>>>(dout, it_m / 4); },
          4096.0 * 4 * (it_m / 4) * warps)) return 1;
  cudaFree(dout);
  printf("ok\n");
  return 0;
}
