// Householder bidiagonalisation G = Q_L B Q_R^H of the n x n product
// G = L1^H L2 of Alg. 3, with B real upper bidiagonal (diagonal d, super-
// diagonal e), and the back-transformations U = Q_L U_B, V = Q_R V_B.
//
// Blocked in panels of NBB columns.  Inside a panel the matrix is kept as
// the panel-start A plus the correction -U Y^H - X V^H, where u_q / v_q are
// the left / right reflectors of the panel's processed columns and
// y_q = tauq A_cur^H u_q, x_q = taup A_cur v_q.  Step i:
//   1. column i receives the correction; left reflector H_L with
//      H_L^H c = d_i e_1 (d_i real); y = tauq (A^H u - Y (U^H u) - V (X^H u));
//   2. row i receives the correction (now including u_i, y_i); right
//      reflector H_R with r H_R = e_i e_1^T (e_i real);
//      x = taup (A v - U (Y^H v) - X (V^H v));
// so that H_L^H A_cur H_R = A_cur - u y^H - x v^H.  The trailing matrix then
// takes A22 -= U Y^H + X V^H through the GEMM engine.  The two matvecs per
// step (A^H u by column sums, A v by row sums) run over 64 x 64 tiles of the
// trailing matrix (one CTA per tile, coalesced loads) and are bound by the
// FP64 pipe on GB300.
#include "kernels.cuh"
#include "prof.cuh"

constexpr int NBB = 32;
constexpr int BRB = 256;

static inline int64_t bchunks(int64_t m) { return (m + 63) / 64; }  // partial slots (64-wide tiles)
size_t gebrd_part_elems(int64_t n) { return (size_t)(bchunks(n) + 1) * (size_t)(n + 1) + 4 * (n / BRB + 2) + 64; }

__device__ __forceinline__ double bsum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < (blockDim.x >> 5)) t = red[threadIdx.x];
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

struct BHouse {
  cplx tau, scal;
  double beta;
};
__device__ __forceinline__ BHouse bmake_house(cplx alpha, double xnorm2) {
  BHouse h;
  if (xnorm2 == 0.0 && alpha.y == 0.0) {
    h.tau = mkc(0.0, 0.0);
    h.beta = alpha.x;
    h.scal = mkc(0.0, 0.0);
  } else {
    const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
    const double beta = (alpha.x >= 0.0) ? -nrm : nrm;
    h.beta = beta;
    h.tau = mkc((beta - alpha.x) / beta, -alpha.y / beta);
    h.scal = cdiv(mkc(1.0, 0.0), mkc(alpha.x - beta, alpha.y));
  }
  return h;
}

struct BdArgs {
  int64_t n, p, i;
  cplx* A;
  int64_t lda;
  cplx* U;   // ld n
  cplx* Vr;  // ld n
  cplx* X;   // ld n
  cplx* Y;   // ld n
  cplx* tauq;
  cplx* taup;
  double* d;
  double* e;
  cplx* part;       // chunk partials, ld n+1
  double* npart;    // norm partials
  cplx* s;          // small dots: [0..NBB) first set, [NBB..2NBB) second set
  const int64_t* status;
};

#define BD_GUARD() \
  if (*(volatile const int64_t*)a.status) return

// 1a. column update, partial norms of rows > i
__global__ void __launch_bounds__(BRB) bd_col_update(BdArgs a) {
  __shared__ cplx yi[NBB], vi[NBB];
  __shared__ double red[32];
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n;
  const int ii = (int)(i - a.p);
  if (threadIdx.x < ii) {
    yi[threadIdx.x] = a.Y[IDX2(i, threadIdx.x, ld)];
    vi[threadIdx.x] = a.Vr[IDX2(i, a.p + threadIdx.x, ld)];
  }
  __syncthreads();
  const int64_t r = i + (int64_t)blockIdx.x * BRB + threadIdx.x;
  double nrm = 0.0;
  if (r < n) {
    cplx c = a.A[IDX2(r, i, a.lda)];
    for (int q = 0; q < ii; ++q) {
      c = csub(c, cmul(a.U[IDX2(r, a.p + q, ld)], cconj(yi[q])));
      c = csub(c, cmul(a.X[IDX2(r, q, ld)], cconj(vi[q])));
    }
    a.A[IDX2(r, i, a.lda)] = c;
    if (r > i) nrm = cabs2(c);
  }
  const double s = bsum(nrm, red);
  if (threadIdx.x == 0) a.npart[blockIdx.x] = s;
}

// 1b. left reflector, u into U(:, i) (rows >= i)
__global__ void __launch_bounds__(BRB) bd_house_left(BdArgs a, int nparts) {
  __shared__ BHouse hs;
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n;
  if (threadIdx.x == 0) {
    double x2 = 0.0;
    for (int k = 0; k < nparts; ++k) x2 += a.npart[k];
    hs = bmake_house(a.A[IDX2(i, i, a.lda)], x2);
    if (blockIdx.x == 0) {
      a.tauq[i] = hs.tau;
      a.d[i] = hs.beta;
    }
  }
  __syncthreads();
  const int64_t r = i + (int64_t)blockIdx.x * BRB + threadIdx.x;
  if (r < n) a.U[IDX2(r, i, ld)] = (r == i) ? mkc(1.0, 0.0) : cmul(a.A[IDX2(r, i, a.lda)], hs.scal);
}

// 1c. column partials of A^H u over rows >= i, columns > i: 64 x 64 tiles,
// slot = row block.  Thread (row r, column quarter q) holds 16 entries.
constexpr int BT64 = 64;

// the small panel dots out[q] = sum_{r in [r0, n)} conj(colA_q(r)) vec(r) (q < nA)
// and out[NBB + q] likewise over colB, done by the extra row of CTAs of a
// matrix-vector launch (outputs first, first + stride, ...): they run beside
// the matvec instead of as a launch of their own
__device__ void bd_dots_role(int64_t n, int64_t r0, int nA, const cplx* colA, int64_t offA, int nB,
                             const cplx* colB, int64_t offB, const cplx* vec, cplx* out, int first, int stride,
                             double* red) {
  for (int d = first; d < nA + nB; d += stride) {
    const int which = d < nA ? 0 : 1;
    const int q = which == 0 ? d : d - nA;
    const cplx* col = which == 0 ? colA + (offA + q) * n : colB + (offB + q) * n;
    cplx acc = mkc(0.0, 0.0);
    for (int64_t r = r0 + threadIdx.x; r < n; r += blockDim.x) cfma_cj(acc, col[r], vec[r]);
    const double sx = bsum(acc.x, red);
    const double sy = bsum(acc.y, red);
    if (threadIdx.x == 0) out[which * NBB + q] = mkc(sx, sy);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(BRB) bd_gemv_c(BdArgs a, int dots) {
  __shared__ cplx us[BT64];
  __shared__ cplx cs[4][BT64];
  __shared__ double red[32];
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n, ldp = n + 1;
  if (dots && blockIdx.y == gridDim.y - 1) {  // U^H u and X^H u of the panel so far
    const int ii = (int)(i - a.p);
    bd_dots_role(n, i, ii, a.U, a.p, ii, a.X, 0, a.U + i * ld, a.s, blockIdx.x, gridDim.x, red);
    return;
  }
  const int64_t r0 = i + (int64_t)blockIdx.y * BT64, c0 = i + 1 + (int64_t)blockIdx.x * BT64;
  const int tid = threadIdx.x;
  if (tid < BT64) us[tid] = (r0 + tid < n) ? a.U[IDX2(r0 + tid, i, ld)] : mkc(0.0, 0.0);
  __syncthreads();
  // thread (column c, row quarter q): 16 consecutive rows of one column
  // (two 128-byte lines, served from L1 after the first touch)
  const int c = tid & 63, q = tid >> 6;
  const int64_t gc = c0 + c, rb = r0 + q * 16;
  cplx av[16];
#pragma unroll
  for (int u = 0; u < 16; ++u)
    av[u] = (gc < n && rb + u < n) ? __ldg(a.A + IDX2(rb + u, gc, a.lda)) : mkc(0.0, 0.0);
  cplx acc = mkc(0.0, 0.0);
#pragma unroll
  for (int u = 0; u < 16; ++u) cfma_cj(acc, av[u], us[q * 16 + u]);
  cs[q][c] = acc;
  __syncthreads();
  if (tid < BT64) {
    const int64_t cc = c0 + tid;
    if (cc < n) a.part[(cc - i - 1) + blockIdx.y * ldp] = cadd(cadd(cs[0][tid], cs[1][tid]), cadd(cs[2][tid], cs[3][tid]));
  }
}


// 1d. y(c) = tauq (sum parts - Y s_U - V s_X), c > i -> Y(c, ii); 64 entries
// per CTA, 4 threads per entry
constexpr int AR = 64;

__global__ void __launch_bounds__(BRB) bd_y_assemble(BdArgs a, int nch) {
  __shared__ cplx su[NBB], sx[NBB];
  __shared__ cplx red4[4][AR];
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n, ldp = n + 1;
  const int ii = (int)(i - a.p);
  if (threadIdx.x < ii) su[threadIdx.x] = a.s[threadIdx.x], sx[threadIdx.x] = a.s[NBB + threadIdx.x];
  __syncthreads();
  const int rl = threadIdx.x & (AR - 1), qq = threadIdx.x / AR;
  const int64_t c = i + 1 + (int64_t)blockIdx.x * AR + rl;
  cplx y = mkc(0.0, 0.0);
  if (c < n) {
    for (int k = qq; k < nch; k += 4) y = cadd(y, a.part[(c - i - 1) + k * ldp]);
    for (int q = qq; q < ii; q += 4) {
      y = csub(y, cmul(a.Y[IDX2(c, q, ld)], su[q]));
      y = csub(y, cmul(a.Vr[IDX2(c, a.p + q, ld)], sx[q]));
    }
  }
  red4[qq][rl] = y;
  __syncthreads();
  if (qq == 0 && c < n) {
    y = cadd(cadd(red4[0][rl], red4[1][rl]), cadd(red4[2][rl], red4[3][rl]));
    a.Y[IDX2(c, ii, ld)] = cmul(a.tauq[i], y);
  }
}

// 2a. row update (c > i), partial norms of c >= i+2
__global__ void __launch_bounds__(BRB) bd_row_update(BdArgs a) {
  __shared__ cplx ui[NBB], xi[NBB];
  __shared__ double red[32];
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n;
  const int ii = (int)(i - a.p);
  if (threadIdx.x <= ii) ui[threadIdx.x] = a.U[IDX2(i, a.p + threadIdx.x, ld)];
  if (threadIdx.x < ii) xi[threadIdx.x] = a.X[IDX2(i, threadIdx.x, ld)];
  __syncthreads();
  const int64_t c = i + 1 + (int64_t)blockIdx.x * BRB + threadIdx.x;
  double nrm = 0.0;
  if (c < n) {
    cplx r = a.A[IDX2(i, c, a.lda)];
    for (int q = 0; q <= ii; ++q) r = csub(r, cmul(ui[q], cconj(a.Y[IDX2(c, q, ld)])));
    for (int q = 0; q < ii; ++q) r = csub(r, cmul(xi[q], cconj(a.Vr[IDX2(c, a.p + q, ld)])));
    a.A[IDX2(i, c, a.lda)] = r;
    if (c >= i + 2) nrm = cabs2(r);
  }
  const double s = bsum(nrm, red);
  if (threadIdx.x == 0) a.npart[blockIdx.x] = s;
}

// 2b. right reflector from x = conj(row), v into Vr(:, i) (rows >= i+1)
__global__ void __launch_bounds__(BRB) bd_house_right(BdArgs a, int nparts) {
  __shared__ BHouse hs;
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n;
  if (threadIdx.x == 0) {
    double x2 = 0.0;
    for (int k = 0; k < nparts; ++k) x2 += a.npart[k];
    hs = bmake_house(cconj(a.A[IDX2(i, i + 1, a.lda)]), x2);
    if (blockIdx.x == 0) {
      a.taup[i] = hs.tau;
      a.e[i] = hs.beta;
    }
  }
  __syncthreads();
  const int64_t c = i + 1 + (int64_t)blockIdx.x * BRB + threadIdx.x;
  if (c < n) a.Vr[IDX2(c, i, ld)] = (c == i + 1) ? mkc(1.0, 0.0) : cmul(cconj(a.A[IDX2(i, c, a.lda)]), hs.scal);
}

// 2c. row partials of A v over rows > i, columns > i: 64 x 64 tiles, slot =
// column block.
__global__ void __launch_bounds__(BRB) bd_gemv_n(BdArgs a, int dots) {
  __shared__ cplx vs[BT64];
  __shared__ cplx rs[4][BT64];
  __shared__ double red[32];
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n, ldp = n + 1;
  if (dots && blockIdx.y == gridDim.y - 1) {  // Y^H v and V^H v of the panel so far
    const int ii = (int)(i - a.p);
    bd_dots_role(n, i + 1, ii + 1, a.Y, 0, ii, a.Vr, a.p, a.Vr + i * ld, a.s, blockIdx.x, gridDim.x, red);
    return;
  }
  const int64_t r0 = i + 1 + (int64_t)blockIdx.y * BT64, c0 = i + 1 + (int64_t)blockIdx.x * BT64;
  const int tid = threadIdx.x;
  if (tid < BT64) vs[tid] = (c0 + tid < n) ? a.Vr[IDX2(c0 + tid, i, ld)] : mkc(0.0, 0.0);
  __syncthreads();
  const int r = tid & 63, q = tid >> 6;
  const int64_t gr = r0 + r;
  cplx av[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int64_t gc = c0 + q * 16 + u;
    av[u] = (gr < n && gc < n) ? __ldg(a.A + IDX2(gr, gc, a.lda)) : mkc(0.0, 0.0);
  }
  cplx acc = mkc(0.0, 0.0);
#pragma unroll
  for (int u = 0; u < 16; ++u) cfma(acc, av[u], vs[q * 16 + u]);
  rs[q][r] = acc;
  __syncthreads();
  if (tid < BT64) {
    const int64_t rr = r0 + tid;
    if (rr < n)
      a.part[(rr - i - 1) + blockIdx.x * ldp] = cadd(cadd(rs[0][tid], rs[1][tid]), cadd(rs[2][tid], rs[3][tid]));
  }
}

// 2d. x(r) = taup (sum parts - U s_Y - X s_V), r > i -> X(r, ii); 64 rows per
// CTA, 4 threads per row
__global__ void __launch_bounds__(BRB) bd_x_assemble(BdArgs a, int nch) {
  __shared__ cplx sy[NBB], sv[NBB];
  __shared__ cplx red4[4][AR];
  BD_GUARD();
  const int64_t n = a.n, i = a.i, ld = n, ldp = n + 1;
  const int ii = (int)(i - a.p);
  if (threadIdx.x <= ii) sy[threadIdx.x] = a.s[threadIdx.x];
  if (threadIdx.x < ii) sv[threadIdx.x] = a.s[NBB + threadIdx.x];
  __syncthreads();
  const int rl = threadIdx.x & (AR - 1), qq = threadIdx.x / AR;
  const int64_t r = i + 1 + (int64_t)blockIdx.x * AR + rl;
  cplx x = mkc(0.0, 0.0);
  if (r < n) {
    for (int k = qq; k < nch; k += 4) x = cadd(x, a.part[(r - i - 1) + k * ldp]);
    for (int q = qq; q <= ii; q += 4) x = csub(x, cmul(a.U[IDX2(r, a.p + q, ld)], sy[q]));
    for (int q = qq; q < ii; q += 4) x = csub(x, cmul(a.X[IDX2(r, q, ld)], sv[q]));
  }
  red4[qq][rl] = x;
  __syncthreads();
  if (qq == 0 && r < n) {
    x = cadd(cadd(red4[0][rl], red4[1][rl]), cadd(red4[2][rl], red4[3][rl]));
    a.X[IDX2(r, ii, ld)] = cmul(a.taup[i], x);
  }
}

#define BLAUNCH(kern, grid, ...)                 \
  do {                                           \
    prof_launch_begin(s);                        \
    kern<<<(grid), BRB, 0, s>>>(__VA_ARGS__);    \
    prof_launch_end(s, #kern);                   \
    bse_count_launch();                          \
    BSE_LAUNCH_CHECK();                          \
  } while (0)

bse_status gebrd_upper(cudaStream_t s, int64_t n, cplx* A, int64_t lda, const GebrdWork& w,
                       const int64_t* status) {
  if (n <= 0) return BSE_OK;
  const int64_t ld = n;
  BSE_CUDA(cudaMemsetAsync(w.U, 0, sizeof(cplx) * n * n, s));
  BSE_CUDA(cudaMemsetAsync(w.Vr, 0, sizeof(cplx) * n * n, s));
  BdArgs a;
  a.n = n, a.A = A, a.lda = lda, a.U = w.U, a.Vr = w.Vr, a.X = w.X, a.Y = w.Y;
  a.tauq = w.tauq, a.taup = w.taup, a.d = w.d, a.e = w.e;
  a.part = w.part;
  a.npart = (double*)(w.part + bchunks(n) * (n + 1));
  a.s = w.small;
  a.status = status;
  const cplx one = mkc(1.0, 0.0), mone = mkc(-1.0, 0.0);
  for (int64_t p = 0; p < n; p += NBB) {
    const int64_t bs = (n - p) < NBB ? (n - p) : NBB;
    a.p = p;
    for (int64_t i = p; i < p + bs; ++i) {
      a.i = i;
      const int ii = (int)(i - p);
      const unsigned gr = ceil_div_u(n - i, BRB);
      BLAUNCH(bd_col_update, gr, a);
      BLAUNCH(bd_house_left, gr, a, (int)gr);
      if (i == n - 1) break;
      const int64_t m = n - i - 1;  // trailing columns / rows
      // y = tauq (A^H u - Y (U^H u) - V (X^H u))
      dim3 gc(ceil_div_u(m, BT64), ceil_div_u(n - i, BT64) + (ii > 0 ? 1 : 0));
      BLAUNCH(bd_gemv_c, gc, a, ii > 0 ? 1 : 0);
      BLAUNCH(bd_y_assemble, ceil_div_u(m, AR), a, (int)ceil_div_u(n - i, BT64));
      // row update and right reflector
      const unsigned gm = ceil_div_u(m, BRB);
      BLAUNCH(bd_row_update, gm, a);
      BLAUNCH(bd_house_right, gm, a, (int)gm);
      // x = taup (A v - U (Y^H v) - X (V^H v))
      dim3 gn(ceil_div_u(m, BT64), ceil_div_u(m, BT64) + 1);
      BLAUNCH(bd_gemv_n, gn, a, 1);
      BLAUNCH(bd_x_assemble, ceil_div_u(m, AR), a, (int)ceil_div_u(m, BT64));
    }
    const int64_t t0 = p + bs, mt = n - t0;
    if (mt > 0 && p + 2 * bs <= n) {
      // A22 -= U_p Y^H + X V_p^H as ONE product of depth 2 bs: [U_p X] [Y V_p]^H,
      // with X parked in the (still zero) columns p+bs .. p+2bs-1 of U and
      // [Y V_p] assembled in S2; the parked columns are zeroed again before
      // the next panel writes its reflectors there
      cplx* A22 = A + IDX2(t0, t0, lda);
      const size_t rowb = sizeof(cplx) * (size_t)mt;
      BSE_CUDA(cudaMemcpy2DAsync(w.U + IDX2(t0, p + bs, ld), sizeof(cplx) * ld, w.X + IDX2(t0, 0, ld),
                                 sizeof(cplx) * ld, rowb, bs, cudaMemcpyDeviceToDevice, s));
      BSE_CUDA(cudaMemcpy2DAsync(w.S2, sizeof(cplx) * n, w.Y + IDX2(t0, 0, ld), sizeof(cplx) * ld, rowb, bs,
                                 cudaMemcpyDeviceToDevice, s));
      BSE_CUDA(cudaMemcpy2DAsync(w.S2 + IDX2(0, bs, n), sizeof(cplx) * n, w.Vr + IDX2(t0, p, ld), sizeof(cplx) * ld,
                                 rowb, bs, cudaMemcpyDeviceToDevice, s));
      GemmParams<cplx> g = gemm_params<cplx>(mt, mt, 2 * bs, OPN, w.U + IDX2(t0, p, ld), ld, OPC, w.S2, n, mone, one,
                                             A22, lda);
      g.status = status;
      bse_status r = gemm_z(s, g);
      if (r) return r;
      BSE_CUDA(cudaMemset2DAsync(w.U + IDX2(t0, p + bs, ld), sizeof(cplx) * ld, 0, rowb, bs, s));
    } else if (mt > 0) {
      cplx* A22 = A + IDX2(t0, t0, lda);
      GemmParams<cplx> g1 = gemm_params<cplx>(mt, mt, bs, OPN, w.U + IDX2(t0, p, ld), ld, OPC,
                                              w.Y + IDX2(t0, 0, ld), ld, mone, one, A22, lda);
      g1.status = status;
      bse_status r = gemm_z(s, g1);
      if (r) return r;
      GemmParams<cplx> g2 = gemm_params<cplx>(mt, mt, bs, OPN, w.X + IDX2(t0, 0, ld), ld, OPC,
                                              w.Vr + IDX2(t0, p, ld), ld, mone, one, A22, lda);
      g2.status = status;
      if ((r = gemm_z(s, g2))) return r;
    }
  }
  return BSE_OK;
}

bse_status gebrd_backtransform(cudaStream_t s, int side, int64_t n, int64_t k, const GebrdWork& w, cplx* Vout,
                               int64_t ldv, cplx* tmp, const int64_t* status) {
  const int64_t nref = side == 0 ? n : n - 1;  // number of reflectors
  if (nref <= 0) return BSE_OK;
  const int64_t bt = backtransform_block();
  const int64_t npan = (nref + bt - 1) / bt;
  for (int64_t b = npan - 1; b >= 0; --b) {
    const int64_t p = b * bt;
    const int64_t bs = (nref - p) < bt ? (nref - p) : bt;
    bse_status r = side == 0
                       ? apply_block_reflector(s, n, k, w.U, n, p, bs, p, w.tauq, Vout, ldv, tmp, status)
                       : apply_block_reflector(s, n, k, w.Vr, n, p, bs, p + 1, w.taup, Vout, ldv, tmp, status);
    if (r) return r;
  }
  return BSE_OK;
}
