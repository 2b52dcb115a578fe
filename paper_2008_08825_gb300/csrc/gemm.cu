// Tiled FP64 GEMM engine, real and complex:  C = alpha op(A) op(B) + beta C
// with triangular operand structure, lower-triangle-only output, a status
// early-out and the fused X/Y epilogue of the final setup (Alg. 2 and Alg. 3,
// last step).
//
// Tile 64 x 64 per CTA of 256 threads, each thread a 4 x 4 register tile
// (rows tx + 16a, columns ty + 16b, so that a warp's stores are contiguous in
// a column).  k-tiles of 8 (complex) or 16 (real) are double-buffered in
// shared memory with a register prefetch of the next tile.
#include <atomic>

#include <mutex>
#include <set>
#include <tuple>

#include "gemm_tile.cuh"
#include "kernels.cuh"
#include "prof.cuh"

static std::atomic<long long> g_launches{0};
void bse_count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// The dynamic shared-memory limit of a kernel is a per-device attribute: set
// it once per (device, kernel, size).
bse_status set_smem_attr(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<int, const void*, int>> done;
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(std::make_tuple(dev, func, bytes))) return BSE_OK;
  BSE_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert(std::make_tuple(dev, func, bytes));
  return BSE_OK;
}
long long bse_total_launches() { return g_launches.load(); }

// Useful (structurally nonzero) multiply-adds of a launch, for the profiler:
// the number of (i, j, kk) with i < m, j < n, kk < k allowed by the
// triangular structure of op(A), op(B) and the lower-only output.
static double sum_min(int64_t cnt, int64_t cap, int64_t off) {
  // sum_{i=0}^{cnt-1} clamp(i + off, 0, cap)
  double s = 0.0;
  for (int64_t i = 0; i < cnt; ++i) {
    int64_t v = i + off;
    s += (double)(v < 0 ? 0 : (v > cap ? cap : v));
  }
  return s;
}
template <typename T>
static double useful_macs(const GemmParams<T>& p) {
  const int64_t m = p.m, n = p.n, k = p.k;
  const bool lo = p.lowerC != 0;
  if (p.triA == TRI_NONE && p.triB == TRI_NONE) {
    if (!lo) return (double)m * n * k;
    double s = 0.0;  // pairs i >= j
    for (int64_t j = 0; j < n && j < m; ++j) s += (double)(m - j);
    return s * (double)k;
  }
  if (p.triA == TRI_LO && p.triB == TRI_NONE && !lo) return sum_min(m, k, 1) * (double)n;  // kk <= i
  if (p.triA == TRI_UP && p.triB == TRI_NONE) {                                            // kk >= i
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      const double kk = (double)(k - i > 0 ? k - i : 0);
      const double jj = lo ? (double)((i < n ? i : n - 1) + 1) : (double)n;
      s += kk * jj;
    }
    return s;
  }
  if (p.triB == TRI_LO && p.triA == TRI_NONE && !lo) {  // kk >= j
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += (double)(k - j > 0 ? k - j : 0);
    return s * (double)m;
  }
  if (p.triB == TRI_UP && p.triA == TRI_NONE && !lo) return sum_min(n, k, 1) * (double)m;  // kk <= j
  if (p.triA == TRI_UP && p.triB == TRI_LO && !lo) {  // kk >= max(i, j)
    double s = 0.0;
    const int64_t mx = m > n ? m : n;
    for (int64_t t = 0; t < mx && t < k; ++t) {
      const double a1 = (double)(t + 1 < m ? t + 1 : m) * (double)(t + 1 < n ? t + 1 : n);
      const double a0 = (double)(t < m ? t : m) * (double)(t < n ? t : n);
      s += (a1 - a0) * (double)(k - t);
    }
    return s;
  }
  return (double)m * n * k;  // not used by the pipelines: dense count
}

static bool beta_nz(cplx b) { return b.x != 0.0 || b.y != 0.0; }
static bool beta_nz(double b) { return b != 0.0; }
static bool beta_nz(float b) { return b != 0.0f; }

template <typename T, int BK>
static bse_status gemm_launch(cudaStream_t s, const GemmParams<T>& p) {
  if (p.m <= 0 || p.n <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(p.n, GBN), ceil_div_u(p.m, GBM), p.kchunk > 0 ? ceil_div_u(p.k, p.kchunk) : 1);
  if (p.kchunk > 0 && (p.kchunk % 64 != 0 || beta_nz(p.beta))) {
    bse_internal_set_error("gemm: split-K needs kchunk % 64 == 0 and beta == 0");
    return BSE_ERR_ARG;
  }
  if (grid.y > 65535) {
    bse_internal_set_error("gemm: m too large for one launch");
    return BSE_ERR_ARG;
  }
  const bool prof = prof_current() != nullptr;
  if (prof) prof_gemm_begin(s);
  prof_launch_begin(s);
  gemm_kernel<T, BK><<<grid, 256, 0, s>>>(p);
  prof_launch_end(s, sizeof(T) == sizeof(cplx) ? "gemm_kernel<cplx> (DFMA)" : "gemm_kernel<real>");
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  if (prof) prof_gemm_end(s, sizeof(T) == sizeof(float) ? 0.0 : useful_macs(p) * (sizeof(T) == sizeof(cplx) ? 8.0 : 2.0));
  return BSE_OK;
}

// split-K on the tensor-core engine: tcgen05 only, plain epilogue, beta 0
template <typename T>
static bool oz_split_ok(const OzWork& oz, const GemmParams<T>& p) {
  return p.kchunk == 0 ||
         (oz.engine == OZ_ENGINE_TCGEN05 && p.kchunk % 64 == 0 && !beta_nz(p.beta) && p.epi == EPI_NONE);
}

bse_status gemm_z(cudaStream_t s, const GemmParams<cplx>& p) {
  const OzWork oz = oz_current();
  if (oz.ptr && oz_split_ok(oz, p) && p.opA != OPT && p.opB != OPT && (double)p.m * p.n * p.k >= (double)oz.min_mnk) {
    const bool prof = prof_current() != nullptr;
    if (prof) prof_gemm_begin(s);
    const double flops = useful_macs(p) * 8.0;
    const bse_status r = gemm_z_oz_raw(s, p, flops);
    if (prof) prof_gemm_end(s, flops);
    return r;
  }
  return gemm_launch<cplx, 8>(s, p);
}
bse_status gemm_d(cudaStream_t s, const GemmParams<double>& p) {
  const OzWork oz = oz_current();
  if (oz.ptr && oz_split_ok(oz, p) && p.opA != OPC && p.opB != OPC && (double)p.m * p.n * p.k >= (double)oz.min_mnk) {
    const bool prof = prof_current() != nullptr;
    if (prof) prof_gemm_begin(s);
    const double flops = useful_macs(p) * 2.0;
    const bse_status r = gemm_d_oz_raw(s, p, flops);
    if (prof) prof_gemm_end(s, flops);
    return r;
  }
  return gemm_launch<double, 16>(s, p);
}
bse_status gemm_f(cudaStream_t s, const GemmParams<float>& p) { return gemm_launch<float, 32>(s, p); }
