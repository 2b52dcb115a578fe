// The tile body of the FP64 GEMM engine (see gemm.cu), shared by the grid
// launcher and by the batched per-instance solver.
#pragma once
#include "gemm.cuh"

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

// One 64 x 64 output tile (rows i0.., columns j0..) computed by the calling
// CTA of 256 threads.  Used by the grid kernel below (one tile per CTA) and by
// the batched per-instance solver (a CTA loops over the tiles of its own
// products).  The caller guarantees i0 < m, j0 < n; on return the shared
// staging buffers may be reused (the function ends with a barrier).
template <typename T, int BK>
__device__ __forceinline__ void gemm_tile(const GemmParams<T>& p, int64_t i0, int64_t j0, int64_t kz0 = 0,
                                          int64_t kz1 = INT64_MAX, T* Cz = nullptr) {
  using N_ = Num<T>;
  constexpr int LA = GBM * BK / 256;
  constexpr int LB = GBN * BK / 256;
  __shared__ T As[2][BK][GBM + 1];
  __shared__ T Bs[2][BK][GBN + 1];

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  int64_t kbeg = 0, kend = p.k;
  if (p.triA == TRI_LO) kend = min(kend, i0 + GBM);
  if (p.triA == TRI_UP) kbeg = max(kbeg, i0);
  if (p.triB == TRI_LO) kbeg = max(kbeg, j0);
  if (p.triB == TRI_UP) kend = min(kend, j0 + GBN);
  kbeg = max(kbeg, kz0);  // split-K layer (kz0, kz1 multiples of BK)
  kend = min(kend, kz1);
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
  T* const Cout = Cz ? Cz : p.C;
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
        if (use_beta) v = N_::add(v, N_::mul(p.beta, Cout[i + j * p.ldc]));
        Cout[i + j * p.ldc] = v;
      }
    }
  }
  __syncthreads();
}

template <typename T, int BK>
__global__ void __launch_bounds__(256, 2) gemm_kernel(const GemmParams<T> p) {
  // longest tiles first: with a lower-triangular A a tile's k range grows with
  // its row, with an upper-triangular B with its column, so those orders are
  // reversed (CTAs start in increasing block order; the last wave is then
  // made of the shortest tiles)
  const int64_t by = p.triA == TRI_LO ? (int64_t)gridDim.y - 1 - blockIdx.y : (int64_t)blockIdx.y;
  const int64_t bx = p.triB == TRI_UP ? (int64_t)gridDim.x - 1 - blockIdx.x : (int64_t)blockIdx.x;
  const int64_t i0 = by * GBM, j0 = bx * GBN;
  if (i0 >= p.m || j0 >= p.n) return;
  if (p.lowerC && j0 > i0 + GBM - 1) return;
  if (p.status && *(volatile const int64_t*)p.status) return;
  const bool split = p.kchunk > 0;
  const int64_t z = blockIdx.z;
  gemm_tile<T, BK>(p, i0, j0, split ? z * p.kchunk : 0, split ? (z + 1) * p.kchunk : INT64_MAX,
                   split ? p.C + z * p.cstride : p.C);
}

// All tiles of one product, computed by the calling CTA (batched solver).
template <typename T, int BK>
__device__ __forceinline__ void gemm_cta(const GemmParams<T>& p) {
  if (p.m <= 0 || p.n <= 0) return;
  for (int64_t i0 = 0; i0 < p.m; i0 += GBM)
    for (int64_t j0 = 0; j0 < p.n; j0 += GBN) {
      if (p.lowerC && j0 > i0 + GBM - 1) continue;
      gemm_tile<T, BK>(p, i0, j0);
    }
}

