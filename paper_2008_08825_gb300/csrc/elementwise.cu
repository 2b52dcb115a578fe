// O(n^2) kernels of the solver pipeline: forming A +- B (Thm. ProdEig:
// M1 = A + B, M2 = A - B), Hermitian mirroring, type conversion, the
// omega / scaling vectors of the final setup, and the eigenvalue gradient.
#include "kernels.cuh"

// ---------------------------------------------------------------------------
// Tile-transposing Hermitian expansion.  Output tile (bi, bj) takes its data
// from the lower (or diagonal) source tile (max, min), loaded coalesced into
// shared memory; above-diagonal outputs are conjugate transposes.
constexpr int TT = 32;

__device__ __forceinline__ cplx herm_pick(const cplx (*S)[TT + 1], int r, int c, int64_t bi, int64_t bj) {
  if (bi > bj) return S[c][r];                 // S[col][row] layout, source = same tile
  if (bi < bj) return cconj(S[r][c]);          // source tile (bj, bi): element (j, i)
  if (r > c) return S[c][r];
  if (r < c) return cconj(S[r][c]);
  return mkc(S[r][r].x, 0.0);
}

__global__ void form_sum_kernel(int64_t n, const cplx* __restrict__ A, int64_t lda, const cplx* __restrict__ B,
                                int64_t ldb, double sgn, cplx* __restrict__ M, int64_t ldm, int full) {
  __shared__ cplx S[TT][TT + 1];  // S[col][row] of the source tile
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (!full && bi < bj) return;
  const int64_t si = bi > bj ? bi : bj, sj = bi > bj ? bj : bi;
  const int r = threadIdx.x;
  for (int c = threadIdx.y; c < TT; c += blockDim.y) {
    const int64_t gi = si * TT + r, gj = sj * TT + c;
    cplx v = mkc(0.0, 0.0);
    if (gi < n && gj < n && gi >= gj) {
      const cplx a = A[IDX2(gi, gj, lda)], b = B[IDX2(gi, gj, ldb)];
      v = mkc(a.x + sgn * b.x, a.y + sgn * b.y);
    }
    S[c][r] = v;
  }
  __syncthreads();
  for (int c = threadIdx.y; c < TT; c += blockDim.y) {
    const int64_t gi = bi * TT + r, gj = bj * TT + c;
    if (gi >= n || gj >= n) continue;
    if (!full && gi < gj) continue;
    M[IDX2(gi, gj, ldm)] = herm_pick(S, r, c, bi, bj);
  }
}

bse_status form_sum(cudaStream_t s, int64_t n, const cplx* A, int64_t lda, const cplx* B, int64_t ldb,
                    double sgn, cplx* M, int64_t ldm, int full) {
  if (n <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(n, TT), ceil_div_u(n, TT)), blk(TT, 8);
  form_sum_kernel<<<grid, blk, 0, s>>>(n, A, lda, B, ldb, sgn, M, ldm, full);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

__global__ void fill_upper_kernel(int64_t n, cplx* M, int64_t ldm) {
  __shared__ cplx S[TT][TT + 1];
  const int64_t bi = blockIdx.y, bj = blockIdx.x;  // output tile, bi <= bj
  if (bi > bj) return;
  const int r = threadIdx.x;
  for (int c = threadIdx.y; c < TT; c += blockDim.y) {
    const int64_t gi = bj * TT + r, gj = bi * TT + c;  // source tile (bj, bi), lower
    cplx v = mkc(0.0, 0.0);
    if (gi < n && gj < n && gi >= gj) v = M[IDX2(gi, gj, ldm)];
    S[c][r] = v;
  }
  __syncthreads();
  for (int c = threadIdx.y; c < TT; c += blockDim.y) {
    const int64_t gi = bi * TT + r, gj = bj * TT + c;
    if (gi >= n || gj >= n || gi > gj) continue;
    // element (gi, gj) with gi <= gj is conj of (gj, gi) = source S[col = gi - bi*TT][row = gj - bj*TT]
    const cplx v = S[r][c];
    M[IDX2(gi, gj, ldm)] = (gi == gj) ? mkc(v.x, 0.0) : cconj(v);
  }
}

bse_status hermitian_fill_upper(cudaStream_t s, int64_t n, cplx* M, int64_t ldm) {
  if (n <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(n, TT), ceil_div_u(n, TT)), blk(TT, 8);
  fill_upper_kernel<<<grid, blk, 0, s>>>(n, M, ldm);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

__global__ void real_to_complex_kernel(int64_t n, int64_t k, const double* Z, int64_t ldz, cplx* V, int64_t ldv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < n && j < k) V[IDX2(i, j, ldv)] = mkc(Z[IDX2(i, j, ldz)], 0.0);
}

bse_status real_to_complex(cudaStream_t s, int64_t n, int64_t k, const double* Z, int64_t ldz, cplx* V,
                           int64_t ldv) {
  if (n <= 0 || k <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(n, 256), (unsigned)k);
  real_to_complex_kernel<<<grid, 256, 0, s>>>(n, k, Z, ldz, V, ldv);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

__global__ void sub_identity_kernel(int64_t k, double* E, int64_t lde) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < k) E[IDX2(i, i, lde)] -= 1.0;
}

bse_status sub_identity(cudaStream_t s, int64_t k, double* E, int64_t lde) {
  if (k <= 0) return BSE_OK;
  sub_identity_kernel<<<ceil_div_u(k, 256), 256, 0, s>>>(k, E, lde);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

__global__ void finish_omega_kernel(int64_t k, const double* lam, int mode, double* omega, double* c1, double* c2,
                                    int64_t* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= k) return;
  const double l = lam[i];
  if (!(l > 0.0)) {
    // M = L^H (A+B) L (CHOL) or L1^H L2 (SVD) is nonsingular/PD exactly when
    // A + B is positive definite
    dev_fail(status, BSE_ERR_NOT_PD_APLUSB, 0);
    return;
  }
  const double om = (mode == 0) ? sqrt(l) : l;
  const double sq = sqrt(om);
  omega[i] = om;
  if (mode == 0) {
    c1[i] = sq;
    c2[i] = 1.0 / sq;
  } else {
    c1[i] = 1.0 / sq;
    c2[i] = 1.0 / sq;
  }
}

bse_status finish_omega(cudaStream_t s, int64_t k, const double* lam, int mode, double* omega_out, double* c1,
                        double* c2, const int64_t* status) {
  if (k <= 0) return BSE_OK;
  finish_omega_kernel<<<ceil_div_u(k, 256), 256, 0, s>>>(k, lam, mode, omega_out, c1, c2, (int64_t*)status);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

__global__ void zero_c_kernel(int64_t m, int64_t n, cplx* A, int64_t lda) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < m && j < n) A[IDX2(i, j, lda)] = mkc(0.0, 0.0);
}

bse_status zero_c(cudaStream_t s, int64_t m, int64_t n, cplx* A, int64_t lda) {
  if (m <= 0 || n <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(m, 256), (unsigned)n);
  zero_c_kernel<<<grid, 256, 0, s>>>(m, n, A, lda);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// ---------------------------------------------------------------------------
// Gradient (Thm. 3 item 3 with the Sigma-normalisation of Eq. (13)):
//   dA = sum_i w_i (x_i x_i^H + y_i y_i^H),  dB = sum_i w_i (x_i y_i^H + y_i x_i^H).
// Both are Hermitian: each CTA computes one 32 x 32 tile on or below the
// diagonal and stores it and its conjugate transpose (through shared memory,
// so both stores are coalesced).  The k columns are processed in chunks of
// GK; the column-b factors are pre-multiplied by w_i and conjugated.
constexpr int GK = 16;

__global__ void __launch_bounds__(256) grad_kernel(int64_t n, int64_t k, const cplx* __restrict__ X, int64_t ldx,
                                                   const cplx* __restrict__ Y, int64_t ldy,
                                                   const double* __restrict__ w, cplx* __restrict__ dA,
                                                   int64_t ldda, cplx* __restrict__ dB, int64_t lddb) {
  const int64_t ta = blockIdx.y, tb = blockIdx.x;
  if (tb > ta) return;
  __shared__ cplx Xa[GK][TT], Ya[GK][TT], Xb[GK][TT], Yb[GK][TT];  // Xb, Yb: w_i conj(.)
  __shared__ cplx TA[TT][TT + 1], TB[TT][TT + 1];
  const int r = threadIdx.x, cy = threadIdx.y;  // 32 x 8
  cplx ga[4], gb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) ga[q] = gb[q] = mkc(0.0, 0.0);
  for (int64_t i0 = 0; i0 < k; i0 += GK) {
    __syncthreads();
    for (int e = threadIdx.y; e < GK; e += blockDim.y) {
      const int64_t i = i0 + e;
      const int64_t ga_row = ta * TT + r, gb_row = tb * TT + r;
      cplx xa = mkc(0, 0), ya = mkc(0, 0), xb = mkc(0, 0), yb = mkc(0, 0);
      if (i < k) {
        const double wi = w[i];
        if (ga_row < n) xa = X[IDX2(ga_row, i, ldx)], ya = Y[IDX2(ga_row, i, ldy)];
        if (gb_row < n) {
          xb = cscale(cconj(X[IDX2(gb_row, i, ldx)]), wi);
          yb = cscale(cconj(Y[IDX2(gb_row, i, ldy)]), wi);
        }
      }
      Xa[e][r] = xa, Ya[e][r] = ya, Xb[e][r] = xb, Yb[e][r] = yb;
    }
    __syncthreads();
#pragma unroll 4
    for (int e = 0; e < GK; ++e) {
      const cplx xa = Xa[e][r], ya = Ya[e][r];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = cy + 8 * q;
        const cplx xb = Xb[e][c], yb = Yb[e][c];
        cfma(ga[q], xa, xb);
        cfma(ga[q], ya, yb);
        cfma(gb[q], xa, yb);
        cfma(gb[q], ya, xb);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = cy + 8 * q;
    const int64_t gi = ta * TT + r, gj = tb * TT + c;
    if (gi < n && gj < n) {
      dA[IDX2(gi, gj, ldda)] = ga[q];
      dB[IDX2(gi, gj, lddb)] = gb[q];
    }
    TA[c][r] = ga[q];
    TB[c][r] = gb[q];
  }
  if (ta == tb) return;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = cy + 8 * q;
    // element (tb*TT + r, ta*TT + c) = conj of (ta*TT + c, tb*TT + r) = TA[r][c]
    const int64_t gi = tb * TT + r, gj = ta * TT + c;
    if (gi < n && gj < n) {
      dA[IDX2(gi, gj, ldda)] = cconj(TA[r][c]);
      dB[IDX2(gi, gj, lddb)] = cconj(TB[r][c]);
    }
  }
}

bse_status grad_outer(cudaStream_t s, int64_t n, int64_t k, const cplx* X, int64_t ldx, const cplx* Y,
                      int64_t ldy, const double* w, cplx* dA, int64_t ldda, cplx* dB, int64_t lddb) {
  if (n <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(n, TT), ceil_div_u(n, TT)), blk(TT, 8);
  grad_kernel<<<grid, blk, 0, s>>>(n, k, X, ldx, Y, ldy, w, dA, ldda, dB, lddb);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// ---------------------------------------------------------------------------
// Refinement of omega against the original A, B (mixed form).  With
// V1 = X - Y, V2 = X + Y and A = (M1 + M2)/2, B = (M1 - M2)/2:
//   v^H Hcal1 v = (v2^H M1 v2 + v1^H M2 v1)/2,   v^H Sigma v = Re(v1^H v2),
//   Hcal1 v - omega Sigma v = [ (M1 v2 + M2 v1)/2 - omega x ; (M1 v2 - M2 v1)/2 + omega y ].
// omega_i is replaced by the Rayleigh quotient of the pencil (Hcal1, Sigma)
// (second-order accurate in the eigenvector error) and est_i = ||r_i|| /
// (omega_i ||v_i||) is the relative residual.
__global__ void sum_diff_kernel(int64_t n, int64_t k, const cplx* X, int64_t ldx, const cplx* Y, int64_t ldy,
                                cplx* V1, cplx* V2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n || j >= k) return;
  const cplx x = X[IDX2(i, j, ldx)], y = Y[IDX2(i, j, ldy)];
  V1[IDX2(i, j, n)] = csub(x, y);
  V2[IDX2(i, j, n)] = cadd(x, y);
}

__global__ void __launch_bounds__(256) refine_omega_kernel(int64_t n, const cplx* X, int64_t ldx, const cplx* Y,
                                                           int64_t ldy, const cplx* V1, const cplx* V2,
                                                           const cplx* P1, const cplx* P2, double* omega,
                                                           double* est, int replace, const int64_t* status) {
  __shared__ double red[8][8];
  if (*(volatile const int64_t*)status) return;
  const int64_t j = blockIdx.x;
  const double om = omega[j];
  double s[6] = {0, 0, 0, 0, 0, 0};  // Re a, Re b, Re(v1^H v2), ||r||^2, ||v||^2, unused
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const cplx v1 = V1[IDX2(i, j, n)], v2 = V2[IDX2(i, j, n)];
    const cplx p1 = P1[IDX2(i, j, n)], p2 = P2[IDX2(i, j, n)];
    const cplx x = X[IDX2(i, j, ldx)], y = Y[IDX2(i, j, ldy)];
    s[0] += v2.x * p1.x + v2.y * p1.y;
    s[1] += v1.x * p2.x + v1.y * p2.y;
    s[2] += v1.x * v2.x + v1.y * v2.y;
    const cplx top = csub(cscale(cadd(p1, p2), 0.5), cscale(x, om));
    const cplx bot = cadd(cscale(csub(p1, p2), 0.5), cscale(y, om));
    s[3] += cabs2(top) + cabs2(bot);
    s[4] += cabs2(x) + cabs2(y);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int q = 0; q < 5; ++q) {
    double v = s[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[q][w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[5];
    for (int q = 0; q < 5; ++q) {
      t[q] = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t[q] += red[q][ww];
    }
    est[j] = sqrt(t[3]) / (om * sqrt(t[4]));
    if (replace) omega[j] = 0.5 * (t[0] + t[1]) / t[2];
  }
}

__global__ void max_kernel(int64_t k, const double* v, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) m = fmax(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    *out = r;
  }
}

bse_status refine_omega(cudaStream_t s, int64_t n, int64_t k, const cplx* M1, const cplx* M2, const cplx* X,
                        int64_t ldx, const cplx* Y, int64_t ldy, cplx* work, double* omega, double* est,
                        double* est_max, const int64_t* status, int replace) {
  if (n <= 0 || k <= 0) return BSE_OK;
  cplx* V1 = work;
  cplx* V2 = V1 + n * k;
  cplx* P1 = V2 + n * k;
  cplx* P2 = P1 + n * k;
  dim3 g(ceil_div_u(n, 256), (unsigned)k);
  sum_diff_kernel<<<g, 256, 0, s>>>(n, k, X, ldx, Y, ldy, V1, V2);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  GemmParams<cplx> a = gemm_params<cplx>(n, k, n, OPN, M1, n, OPN, V2, n, one, zero, P1, n);
  a.status = status;
  bse_status r = gemm_z(s, a);
  if (r) return r;
  GemmParams<cplx> b = gemm_params<cplx>(n, k, n, OPN, M2, n, OPN, V1, n, one, zero, P2, n);
  b.status = status;
  if ((r = gemm_z(s, b))) return r;
  refine_omega_kernel<<<(unsigned)k, 256, 0, s>>>(n, X, ldx, Y, ldy, V1, V2, P1, P2, omega, est, replace, status);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  max_kernel<<<1, 256, 0, s>>>(k, est, est_max);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// ---- square-root method (Alg. 1) -----------------------------------------------
// For the eigenvalues d of A - B: q+ = d^{1/4}, q- = d^{-1/4}, so that with
// W+- = Q diag(q+-) the principal square root is S = W+ W+^H = Q diag(d^{1/2}) Q^H
// and its inverse S^{-1} = W- W-^H.  A non-positive eigenvalue means A - B is
// not positive definite: status (BSE_ERR_NOT_PD_AMINUSB, 1-based index of one
// such eigenvalue in ascending order).
__global__ void sqrt_factors_kernel(int64_t n, const double* __restrict__ d, double* __restrict__ qp,
                                    double* __restrict__ qm, int64_t* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = d[i];
  if (!(di > 0.0)) {
    dev_fail(status, BSE_ERR_NOT_PD_AMINUSB, i + 1);
    return;
  }
  const double r = sqrt(sqrt(di));
  qp[i] = r;
  qm[i] = 1.0 / r;
}

bse_status sqrt_factors(cudaStream_t s, int64_t n, const double* d, double* qp, double* qm, int64_t* status) {
  if (n <= 0) return BSE_OK;
  sqrt_factors_kernel<<<ceil_div_u(n, 256), 256, 0, s>>>(n, d, qp, qm, status);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// W(:, j) = Q(:, j) * q[j]
__global__ void scale_columns_kernel(int64_t n, int64_t k, const cplx* __restrict__ Q, int64_t ldq,
                                     const double* __restrict__ q, cplx* __restrict__ W, int64_t ldw) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < n && j < k) W[IDX2(i, j, ldw)] = cscale(Q[IDX2(i, j, ldq)], q[j]);
}

bse_status scale_columns(cudaStream_t s, int64_t n, int64_t k, const cplx* Q, int64_t ldq, const double* q, cplx* W,
                         int64_t ldw) {
  if (n <= 0 || k <= 0) return BSE_OK;
  dim3 grid(ceil_div_u(n, 256), (unsigned)k);
  scale_columns_kernel<<<grid, 256, 0, s>>>(n, k, Q, ldq, q, W, ldw);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}
