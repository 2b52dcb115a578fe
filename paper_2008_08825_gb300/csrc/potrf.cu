// Blocked Cholesky factorisation L L^H = M (Alg. 2 step 1; Alg. 3 steps 1-2)
// and the triangular solve with L^H used by Alg. 2 step 4.
//
// Right-looking, block size 64: for each diagonal block one CTA factors it
// in shared memory (FP64, pivot > 0 check) and writes both L_kk and
// L_kk^{-1}; the panel below is L21 = A21 L_kk^{-H} (a GEMM with the inverse,
// in place), and the trailing lower triangle takes A22 -= L21 L21^H.  A
// non-positive or NaN pivot sets the device status word (code, 1-based global
// column) and every later kernel of the pipeline returns at once.
#include "kernels.cuh"

constexpr int CHOL_NB = 64;
constexpr int DIAG_LD = CHOL_NB + 1;

__global__ void __launch_bounds__(256) potrf_diag_kernel(cplx* __restrict__ A, int64_t lda, int64_t k0,
                                                         int bs, cplx* __restrict__ Linv,
                                                         int64_t* __restrict__ status, int64_t err_code) {
  extern __shared__ cplx sm[];
  cplx* S = sm;                          // L block, column-major, ld DIAG_LD
  cplx* Iv = sm + CHOL_NB * DIAG_LD;     // inverse, column-major, ld DIAG_LD
  __shared__ int fail;
  const int tid = threadIdx.x;
  if (*(volatile int64_t*)status) return;
  if (tid == 0) fail = 0;
  for (int e = tid; e < CHOL_NB * CHOL_NB; e += blockDim.x) {
    const int i = e % CHOL_NB, j = e / CHOL_NB;
    cplx v = mkc(0.0, 0.0);
    if (i < bs && j < bs && i >= j) v = A[IDX2(k0 + i, k0 + j, lda)];
    S[i + j * DIAG_LD] = v;
    Iv[i + j * DIAG_LD] = mkc(0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < bs; ++j) {
    if (tid == 0) {
      const double d = S[j + j * DIAG_LD].x;
      if (!(d > 0.0)) {
        fail = 1;
        dev_fail(status, err_code, k0 + j + 1);
      } else {
        S[j + j * DIAG_LD] = mkc(sqrt(d), 0.0);
      }
    }
    __syncthreads();
    if (fail) return;
    const double rl = 1.0 / S[j + j * DIAG_LD].x;
    for (int i = j + 1 + tid; i < bs; i += blockDim.x) S[i + j * DIAG_LD] = cscale(S[i + j * DIAG_LD], rl);
    __syncthreads();
    const int m = bs - j - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int ii = e % m, kc = e / m;
      if (ii < kc) continue;
      const int i = j + 1 + ii, c = j + 1 + kc;
      cplx v = S[i + c * DIAG_LD];
      const cplx a = S[i + j * DIAG_LD], b = S[c + j * DIAG_LD];
      v.x -= a.x * b.x + a.y * b.y;  // v -= a * conj(b)
      v.y -= a.y * b.x - a.x * b.y;
      S[i + c * DIAG_LD] = v;
    }
    __syncthreads();
  }
  // inverse of the lower-triangular block, one column per thread
  if (tid < bs) {
    const int c = tid;
    Iv[c + c * DIAG_LD] = mkc(1.0 / S[c + c * DIAG_LD].x, 0.0);
    for (int i = c + 1; i < bs; ++i) {
      cplx s = mkc(0.0, 0.0);
      for (int k = c; k < i; ++k) cfma(s, S[i + k * DIAG_LD], Iv[k + c * DIAG_LD]);
      Iv[i + c * DIAG_LD] = cscale(s, -1.0 / S[i + i * DIAG_LD].x);
    }
  }
  __syncthreads();
  for (int e = tid; e < bs * bs; e += blockDim.x) {
    const int i = e % bs, j = e / bs;
    A[IDX2(k0 + i, k0 + j, lda)] = (i >= j) ? S[i + j * DIAG_LD] : mkc(0.0, 0.0);
    Linv[i + (int64_t)j * CHOL_NB] = (i >= j) ? Iv[i + j * DIAG_LD] : mkc(0.0, 0.0);
  }
}


int chol_block_size() { return CHOL_NB; }
size_t chol_linv_elems(int64_t n) { return (size_t)((n + CHOL_NB - 1) / CHOL_NB) * CHOL_NB * CHOL_NB; }

bse_status potrf_lower(cudaStream_t s, int64_t n, cplx* A, int64_t lda, cplx* Linv, int64_t* status,
                       int64_t err_code) {
  const size_t smem = sizeof(cplx) * 2 * CHOL_NB * DIAG_LD;
  {
    const bse_status r = set_smem_attr((const void*)potrf_diag_kernel, (int)smem);
    if (r) return r;
  }
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0), mone = mkc(-1.0, 0.0);
  for (int64_t k0 = 0; k0 < n; k0 += CHOL_NB) {
    const int bs = (int)((n - k0) < CHOL_NB ? (n - k0) : CHOL_NB);
    cplx* Li = Linv + (k0 / CHOL_NB) * CHOL_NB * CHOL_NB;
    potrf_diag_kernel<<<1, 256, smem, s>>>(A, lda, k0, bs, Li, status, err_code);
    bse_count_launch();
    BSE_LAUNCH_CHECK();
    const int64_t m2 = n - k0 - bs;
    if (m2 <= 0) continue;
    cplx* A21 = A + IDX2(k0 + bs, k0, lda);
    cplx* A22 = A + IDX2(k0 + bs, k0 + bs, lda);
    // L21 = A21 * Linv^H, in place: one CTA column (bs <= 64) and every CTA
    // reads all of its rows before its epilogue writes them.
    GemmParams<cplx> p = gemm_params<cplx>(m2, bs, bs, OPN, A21, lda, OPC, Li, CHOL_NB, one, zero, A21, lda);
    p.triB = TRI_UP;
    p.status = status;
    bse_status r = gemm_z(s, p);
    if (r) return r;
    GemmParams<cplx> q = gemm_params<cplx>(m2, m2, bs, OPN, A21, lda, OPC, A21, lda, mone, one, A22, lda);
    q.lowerC = 1;
    q.status = status;
    r = gemm_z(s, q);
    if (r) return r;
  }
  return BSE_OK;
}

// Solve L^H X = R in place (R: n x k, ld ldr) with L lower triangular from
// potrf_lower and its diagonal-block inverses.  Recursive: rows [off, off+n)
// split at n1 (a multiple of the block size); the bottom part is solved
// first, the top right-hand side takes one large update
//   R1 -= (L21)^H R2,   L21 = L(off+n1 : off+n, off : off+n1),
// then the top part is solved; a leaf (one diagonal block) is X = Linv^H R.
static bse_status trsm_rec(cudaStream_t s, int64_t off, int64_t n, int64_t k, const cplx* L, int64_t ldl,
                           const cplx* Linv, cplx* R, int64_t ldr, const int64_t* status) {
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0), mone = mkc(-1.0, 0.0);
  if (n <= CHOL_NB) {
    const cplx* Li = Linv + (off / CHOL_NB) * CHOL_NB * CHOL_NB;
    cplx* Rb = R + off;
    // in place: m = n <= 64 means one CTA row (DFMA engine) or a split that
    // reads all of Rb before the product writes it (tensor-core engine)
    GemmParams<cplx> p = gemm_params<cplx>(n, k, n, OPC, Li, CHOL_NB, OPN, Rb, ldr, one, zero, Rb, ldr);
    p.triA = TRI_UP;
    p.status = status;
    return gemm_z(s, p);
  }
  const int64_t half = (n + 1) / 2;
  const int64_t n1 = (half + CHOL_NB - 1) / CHOL_NB * CHOL_NB, n2 = n - n1;
  bse_status r = trsm_rec(s, off + n1, n2, k, L, ldl, Linv, R, ldr, status);
  if (r) return r;
  GemmParams<cplx> q = gemm_params<cplx>(n1, k, n2, OPC, L + IDX2(off + n1, off, ldl), ldl, OPN, R + off + n1, ldr,
                                         mone, one, R + off, ldr);
  q.status = status;
  if ((r = gemm_z(s, q))) return r;
  return trsm_rec(s, off, n1, k, L, ldl, Linv, R, ldr, status);
}

bse_status trsm_lower_conjtrans(cudaStream_t s, int64_t n, int64_t k, const cplx* L, int64_t ldl,
                                const cplx* Linv, cplx* R, int64_t ldr, const int64_t* status) {
  if (n <= 0 || k <= 0) return BSE_OK;
  return trsm_rec(s, 0, n, k, L, ldl, Linv, R, ldr, status);
}
