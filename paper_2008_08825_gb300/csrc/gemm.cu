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

#include "gemm.cuh"
#include "prof.cuh"

static std::atomic<long long> g_launches{0};
void bse_count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long bse_total_launches() { return g_launches.load(); }

template <typename T>
struct Num;
template <>
struct Num<double> {
  __device__ __forceinline__ static double zero() { return 0.0; }
  __device__ __forceinline__ static double cj(double a) { return a; }
  __device__ __forceinline__ static void fma_(double& acc, double a, double b) { acc = fma(a, b, acc); }
  __device__ __forceinline__ static double mul(double a, double b) { return a * b; }
  __device__ __forceinline__ static double add(double a, double b) { return a + b; }
  __device__ __forceinline__ static bool nz(double a) { return a != 0.0; }
  __device__ __forceinline__ static double rs(double a, double s) { return a * s; }
};
template <>
struct Num<float> {
  __device__ __forceinline__ static float zero() { return 0.0f; }
  __device__ __forceinline__ static float cj(float a) { return a; }
  __device__ __forceinline__ static void fma_(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
  __device__ __forceinline__ static float mul(float a, float b) { return a * b; }
  __device__ __forceinline__ static float add(float a, float b) { return a + b; }
  __device__ __forceinline__ static bool nz(float a) { return a != 0.0f; }
  __device__ __forceinline__ static float rs(float a, double s) { return a * (float)s; }
};
template <>
struct Num<cplx> {
  __device__ __forceinline__ static cplx zero() { return mkc(0.0, 0.0); }
  __device__ __forceinline__ static cplx cj(cplx a) { return cconj(a); }
  __device__ __forceinline__ static void fma_(cplx& acc, cplx a, cplx b) { cfma(acc, a, b); }
  __device__ __forceinline__ static cplx mul(cplx a, cplx b) { return cmul(a, b); }
  __device__ __forceinline__ static cplx add(cplx a, cplx b) { return cadd(a, b); }
  __device__ __forceinline__ static bool nz(cplx a) { return a.x != 0.0 || a.y != 0.0; }
  __device__ __forceinline__ static cplx rs(cplx a, double s) { return cscale(a, s); }
};

constexpr int GBM = 64, GBN = 64;

template <typename T, int BK>
__global__ void __launch_bounds__(256, 2) gemm_kernel(const GemmParams<T> p) {
  using N_ = Num<T>;
  constexpr int LA = GBM * BK / 256;
  constexpr int LB = GBN * BK / 256;
  __shared__ T As[2][BK][GBM + 1];
  __shared__ T Bs[2][BK][GBN + 1];

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * GBM, j0 = (int64_t)blockIdx.x * GBN;
  if (i0 >= p.m || j0 >= p.n) return;
  if (p.lowerC && j0 > i0 + GBM - 1) return;
  if (p.status && *(volatile const int64_t*)p.status) return;

  int64_t kbeg = 0, kend = p.k;
  if (p.triA == TRI_LO) kend = min(kend, i0 + GBM);
  if (p.triA == TRI_UP) kbeg = max(kbeg, i0);
  if (p.triB == TRI_LO) kbeg = max(kbeg, j0);
  if (p.triB == TRI_UP) kend = min(kend, j0 + GBN);
  kbeg = (kbeg / BK) * BK;
  const int64_t nk = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;

  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = N_::zero();

  T ra[LA], rb[LB];
  auto load = [&](int64_t kt) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + 256 * r;
      int i, kk;
      if (p.opA == OPN) {
        i = e % GBM, kk = e / GBM;
      } else {
        kk = e % BK, i = e / BK;
      }
      const int64_t gi = i0 + i, gk = kt + kk;
      T v = N_::zero();
      bool ok = gi < p.m && gk < p.k;
      if (p.triA == TRI_LO && gk > gi) ok = false;
      if (p.triA == TRI_UP && gk < gi) ok = false;
      if (ok) {
        if (p.opA == OPN)
          v = p.A[gi + gk * p.lda];
        else if (p.opA == OPT)
          v = p.A[gk + gi * p.lda];
        else
          v = N_::cj(p.A[gk + gi * p.lda]);
      }
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + 256 * r;
      int j, kk;
      if (p.opB == OPN) {
        kk = e % BK, j = e / BK;
      } else {
        j = e % GBN, kk = e / GBN;
      }
      const int64_t gj = j0 + j, gk = kt + kk;
      T v = N_::zero();
      bool ok = gj < p.n && gk < p.k;
      if (p.triB == TRI_LO && gk < gj) ok = false;
      if (p.triB == TRI_UP && gk > gj) ok = false;
      if (ok) {
        if (p.opB == OPN)
          v = p.B[gk + gj * p.ldb];
        else if (p.opB == OPT)
          v = p.B[gj + gk * p.ldb];
        else
          v = N_::cj(p.B[gj + gk * p.ldb]);
      }
      rb[r] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + 256 * r;
      int i, kk;
      if (p.opA == OPN) {
        i = e % GBM, kk = e / GBM;
      } else {
        kk = e % BK, i = e / BK;
      }
      As[buf][kk][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + 256 * r;
      int j, kk;
      if (p.opB == OPN) {
        kk = e % BK, j = e / BK;
      } else {
        j = e % GBN, kk = e / GBN;
      }
      Bs[buf][kk][j] = rb[r];
    }
  };

  if (nk > 0) {
    load(kbeg);
    store(0);
    __syncthreads();
    for (int64_t t = 0; t < nk; ++t) {
      const int cur = (int)(t & 1);
      if (t + 1 < nk) load(kbeg + (t + 1) * BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[cur][kk][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[cur][kk][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) N_::fma_(acc[a][b], av[a], bv[b]);
      }
      if (t + 1 < nk) store(cur ^ 1);
      __syncthreads();
    }
  }

  const bool use_beta = N_::nz(p.beta);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int64_t j = j0 + ty + 16 * b;
    if (j >= p.n) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + tx + 16 * a;
      if (i >= p.m) continue;
      if (p.lowerC && i < j) continue;
      T v = N_::mul(p.alpha, acc[a][b]);
      if (p.epi == EPI_XY) {
        const T v1 = p.P[i + j * p.ldp];
        const double s1 = p.c1[j], s2 = p.c2[j];
        const T x1 = N_::rs(v1, 0.5 * s1), x2 = N_::rs(v, 0.5 * s2);
        p.C[i + j * p.ldc] = N_::add(x1, x2);
        p.Y[i + j * p.ldy] = N_::add(x2, N_::rs(x1, -1.0));
      } else {
        if (use_beta) v = N_::add(v, N_::mul(p.beta, p.C[i + j * p.ldc]));
        p.C[i + j * p.ldc] = v;
      }
    }
  }
}

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

template <typename T, int BK>
static bse_status gemm_launch(cudaStream_t s, const GemmParams<T>& p) {
  if (p.m <= 0 || p.n <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(p.n, GBN), ceil_div_u(p.m, GBM));
  if (grid.y > 65535) {
    bse_internal_set_error("gemm: m too large for one launch");
    return BSE_ERR_ARG;
  }
  const bool prof = prof_current() != nullptr;
  if (prof) prof_gemm_begin(s);
  gemm_kernel<T, BK><<<grid, 256, 0, s>>>(p);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  if (prof) prof_gemm_end(s, sizeof(T) == sizeof(float) ? 0.0 : useful_macs(p) * (sizeof(T) == sizeof(cplx) ? 8.0 : 2.0));
  return BSE_OK;
}

bse_status gemm_z(cudaStream_t s, const GemmParams<cplx>& p) { return gemm_launch<cplx, 8>(s, p); }
bse_status gemm_d(cudaStream_t s, const GemmParams<double>& p) { return gemm_launch<double, 16>(s, p); }
bse_status gemm_f(cudaStream_t s, const GemmParams<float>& p) { return gemm_launch<float, 32>(s, p); }
