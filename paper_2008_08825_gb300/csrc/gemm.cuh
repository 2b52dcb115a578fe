// Tiled FP64 GEMM engine (real and complex) used by every dense contraction
// of the solver: Cholesky panels and trailing updates, the congruence
// M = L^H (A+B) L, the product L1^H L2, Householder block updates, the
// back-transformations and the triangular solves / products of the
// post-processing.  On GB300 the FP64 pipe (measured ~1.2 TFLOP/s for DFMA,
// ~1.05 for FP64 mma.sync) is the bound for all of these, so the engine uses
// DFMA from registers with shared-memory staged tiles; it skips every k-tile
// that a triangular operand makes zero and every output tile outside a
// requested lower triangle, so no FP64 operation is spent on known zeros.
#pragma once
#include "common.cuh"

enum { OPN = 0, OPT = 1, OPC = 2 };
// Structure of the LOGICAL operand op(X): lower (entries with col > row are
// zero), upper (col < row zero) or full.  Masked entries are never read.
enum { TRI_NONE = 0, TRI_LO = 1, TRI_UP = 2 };
enum { EPI_NONE = 0, EPI_XY = 1 };

template <typename T>
struct GemmParams {
  int64_t m, n, k;
  int opA, opB, triA, triB;
  const T* A;
  int64_t lda;
  const T* B;
  int64_t ldb;
  T* C;
  int64_t ldc;
  T alpha, beta;
  int lowerC;               // write only entries with row >= col (and skip tiles above)
  const int64_t* status;    // if non-NULL and *status != 0, write nothing
  // EPI_XY (complex only): v2 = alpha*acc, v1 = P(i,j);
  //   C(i,j) = X = (c1[j] v1 + c2[j] v2)/2,  Y(i,j) = (c2[j] v2 - c1[j] v1)/2
  int epi;
  const T* P;
  int64_t ldp;
  const double* c1;
  const double* c2;
  T* Y;
  int64_t ldy;
  // split-K (DFMA engine only): when kchunk > 0, grid layer z computes the k
  // range [z kchunk, (z+1) kchunk) into C + z cstride (kchunk a multiple of
  // 64, beta 0); the caller adds the layers
  int64_t kchunk;
  int64_t cstride;
};

template <typename T>
__host__ __device__ inline GemmParams<T> gemm_params(int64_t m, int64_t n, int64_t k, int opA, const T* A, int64_t lda, int opB,
                          const T* B, int64_t ldb, T alpha, T beta, T* C, int64_t ldc) {
  GemmParams<T> p;
  p.m = m, p.n = n, p.k = k;
  p.opA = opA, p.opB = opB, p.triA = TRI_NONE, p.triB = TRI_NONE;
  p.A = A, p.lda = lda, p.B = B, p.ldb = ldb, p.C = C, p.ldc = ldc;
  p.alpha = alpha, p.beta = beta;
  p.lowerC = 0;
  p.status = nullptr;
  p.epi = EPI_NONE;
  p.P = nullptr, p.ldp = 0, p.c1 = nullptr, p.c2 = nullptr, p.Y = nullptr, p.ldy = 0;
  p.kchunk = 0, p.cstride = 0;
  return p;
}

bse_status gemm_z(cudaStream_t s, const GemmParams<cplx>& p);
bse_status gemm_d(cudaStream_t s, const GemmParams<double>& p);
bse_status gemm_f(cudaStream_t s, const GemmParams<float>& p);

// Launch counter shared by all translation units.
void bse_count_launch(int64_t k = 1);
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (device, kernel, size)
bse_status set_smem_attr(const void* func, int bytes);
