// Batched solver: many independent BSE instances of uneven size n <= 1024,
// the lowest k eigenpairs of each, in ONE persistent launch (Alg. 2 per
// instance).  Each CTA pops the next instance from a queue sorted by size
// (largest first, so the long ones start first) and runs the whole Cholesky
// pipeline for it with CTA-local routines:
//   form M1 = A + B, M2 = A - B; blocked Cholesky of M2 (block 32, the
//   GEMM engine's tile routine for the panel and the trailing update);
//   W = M1 L, M = L^H W (tile routine); unblocked Householder
//   tridiagonalisation of M (lower storage, explicit reflectors kept in M);
//   bisection for the k smallest eigenvalues of T; twisted-factorisation
//   vectors; one Newton-Schulz step; back-transformation one reflector at a
//   time (a warp per column, no barriers); P = L^{-H} V_M by column-wise
//   substitution; X, Y from P and L V_M through the tile routine's fused
//   epilogue (Alg. 2 steps 4-6).
// The SVD method (Alg. 3 per instance, batched_svd_kernel) runs the same way:
//   two blocked Choleskys L1 L1^H = A + B, L2 L2^H = A - B; G = L1^H L2
//   (tile routine); unblocked Householder bidiagonalisation G = Q B P^H (a
//   warp per column for the left reflectors, a row matvec plus a warp per
//   column for the right ones); bisection on the Golub-Kahan form of B for
//   the k smallest singular values; twisted-factorisation vectors split into
//   U_B, V_B; one Newton-Schulz step on each; U = Q U_B, V = P V_B one
//   reflector at a time; X, Y from L1 U and L2 V through the fused epilogue.
// Large instances (n >= BATCH_TEAM_MIN_N) are solved by a team: the CTAs of
// one thread-block cluster (BATCH_TEAM CTAs on as many SMs).  The team splits
// the heavy stages -- the Cholesky panels and trailing updates and the
// congruence / G products (by output tiles), every column of the Householder
// tridiagonalisation or bidiagonalisation (matrix-vector rows, update
// columns; the vector each step needs whole is exchanged through
// distributed shared memory) -- and the k-sized tail by eigenpairs, and
// meets at cluster barriers between dependent steps.  Without teams a whole
// instance stays on one SM; the only global atomics are the queue counters.
#include <float.h>

#include <atomic>
#include <cooperative_groups.h>

#include "gemm_tile.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

constexpr int BT = 256;       // threads per CTA
constexpr int BATCH_TEAM = 4;          // default CTAs (one cluster) per large Alg. 2 instance
constexpr int BATCH_TEAM_MIN_N = 448;  // default: instances this large are solved by a team
constexpr int CNB = 32;       // Cholesky block
constexpr int CLD = CNB + 1;

struct BatchDesc {
  int64_t n, k;
  const cplx* A;
  const cplx* B;
  double* omega;
  cplx* X;
  cplx* Y;
  char* ws;
  int64_t* status;  // code, info
};

struct InstWs {
  cplx *M1, *L, *W, *Linv, *tau, *VM, *P;
  double *d, *e, *e2, *Z, *sc, *E, *lam, *c1, *c2;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__host__ __device__ inline size_t carve_inst(char* base, int64_t n, int64_t k, InstWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = align256(off);
    char* p = base ? base + off : nullptr;
    off += bytes > 0 ? bytes : 1;
    return p;
  };
  const size_t nn = (size_t)n * n, nk = (size_t)n * k;
  InstWs t;
  t.M1 = (cplx*)take(nn * 16);
  t.L = (cplx*)take(nn * 16);
  t.W = (cplx*)take(nn * 16);
  t.Linv = (cplx*)take(CNB * CNB * 16);
  t.tau = (cplx*)take(n * 16);
  t.VM = (cplx*)take(nk * 16);
  t.P = (cplx*)take(nk * 16);
  t.d = (double*)take(n * 8);
  t.e = (double*)take(n * 8);
  t.e2 = (double*)take(n * 8);
  t.Z = (double*)take(nk * 8);
  t.sc = (double*)take(nk * 8);
  t.E = (double*)take((size_t)k * k * 8);
  t.lam = (double*)take(k * 8);
  t.c1 = (double*)take(k * 8);
  t.c2 = (double*)take(k * 8);
  if (w) *w = t;
  return align256(off);
}

size_t batched_inst_bytes(int64_t n, int64_t k) { return carve_inst(nullptr, n, k, nullptr); }
int batched_max_n() { return 1024; }

__device__ __forceinline__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < BT / 32; ++w) t += red[w];
  __syncthreads();
  return t;  // every thread gets the same value
}

__device__ __forceinline__ double cta_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = red[0];
  for (int w = 1; w < BT / 32; ++w) t = fmax(t, red[w]);
  __syncthreads();
  return t;
}

__device__ __forceinline__ double cta_min(double v, double* red) { return -cta_max(-v, red); }

// The CTAs that solve one instance together: a cluster (size > 1) or the
// calling CTA alone (size 1).
struct Team {
  int rank, size;
};

// Barrier of the team.  For a cluster it is barrier.cluster.arrive (release)
// + barrier.cluster.wait (acquire), both at cluster scope, so the global and
// distributed-shared-memory writes of every team member before it are
// visible to every member after it.
__device__ __forceinline__ void team_sync(const Team& tm) {
  if (tm.size > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// The tiles t = rank, rank + size, ... of one product (the order of gemm_cta).
template <typename T, int BK>
__device__ __forceinline__ void gemm_team(const GemmParams<T>& p, const Team& tm) {
  if (p.m <= 0 || p.n <= 0) return;
  int64_t t = 0;
  for (int64_t i0 = 0; i0 < p.m; i0 += GBM)
    for (int64_t j0 = 0; j0 < p.n; j0 += GBN) {
      if (p.lowerC && j0 > i0 + GBM - 1) continue;
      if (t++ % tm.size != tm.rank) continue;
      gemm_tile<T, BK>(p, i0, j0);
    }
}

// ---- Cholesky of the lower triangle of L (n x n, ld n), block CNB ----------
// Every CTA of a team factors the diagonal block in its own shared memory
// (the same arithmetic, so the same bits and the same pivot decision); the
// team's first CTA writes it, and the panel and trailing update are split by
// output tiles.
__device__ bool cta_potrf(int64_t n, cplx* L, cplx* Linv, int64_t* status, cplx* S, cplx* Iv, int* flag,
                          int64_t err_code, Team tm = Team{0, 1}) {
  const int tid = threadIdx.x;
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0), mone = mkc(-1.0, 0.0);
  for (int64_t k0 = 0; k0 < n; k0 += CNB) {
    const int bs = (int)((n - k0) < CNB ? (n - k0) : CNB);
    for (int e = tid; e < CNB * CNB; e += BT) {
      const int i = e % CNB, j = e / CNB;
      S[i + j * CLD] = (i < bs && j < bs && i >= j) ? L[IDX2(k0 + i, k0 + j, n)] : zero;
      Iv[i + j * CLD] = zero;
    }
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int j = 0; j < bs; ++j) {
      if (tid == 0) {
        const double dd = S[j + j * CLD].x;
        if (!(dd > 0.0)) {
          *flag = 1;
          if (tm.rank == 0) {
            status[0] = err_code;
            status[1] = k0 + j + 1;
          }
        } else {
          S[j + j * CLD] = mkc(sqrt(dd), 0.0);
        }
      }
      __syncthreads();
      if (*flag) return false;
      const double rl = 1.0 / S[j + j * CLD].x;
      for (int i = j + 1 + tid; i < bs; i += BT) S[i + j * CLD] = cscale(S[i + j * CLD], rl);
      __syncthreads();
      const int m = bs - j - 1;
      for (int e = tid; e < m * m; e += BT) {
        const int ii = e % m, kc = e / m;
        if (ii < kc) continue;
        const int i = j + 1 + ii, c = j + 1 + kc;
        const cplx a = S[i + j * CLD], b = S[c + j * CLD];
        cplx v = S[i + c * CLD];
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.y * b.x - a.x * b.y;
        S[i + c * CLD] = v;
      }
      __syncthreads();
    }
    if (tid < bs) {
      const int c = tid;
      Iv[c + c * CLD] = mkc(1.0 / S[c + c * CLD].x, 0.0);
      for (int i = c + 1; i < bs; ++i) {
        cplx s = zero;
        for (int kk = c; kk < i; ++kk) cfma(s, S[i + kk * CLD], Iv[kk + c * CLD]);
        Iv[i + c * CLD] = cscale(s, -1.0 / S[i + i * CLD].x);
      }
    }
    __syncthreads();
    if (tm.rank == 0)
      for (int e = tid; e < bs * bs; e += BT) {
        const int i = e % bs, j = e / bs;
        L[IDX2(k0 + i, k0 + j, n)] = (i >= j) ? S[i + j * CLD] : zero;
        Linv[i + j * CNB] = (i >= j) ? Iv[i + j * CLD] : zero;
      }
    __threadfence_block();
    team_sync(tm);
    const int64_t m2 = n - k0 - bs;
    if (m2 <= 0) continue;
    cplx* A21 = L + IDX2(k0 + bs, k0, n);
    cplx* A22 = L + IDX2(k0 + bs, k0 + bs, n);
    GemmParams<cplx> p = gemm_params<cplx>(m2, bs, bs, OPN, A21, n, OPC, Linv, CNB, one, zero, A21, n);
    p.triB = TRI_UP;
    gemm_team<cplx, 8>(p, tm);
    __threadfence_block();
    if (tm.size > 1) team_sync(tm);
    GemmParams<cplx> q = gemm_params<cplx>(m2, m2, bs, OPN, A21, n, OPC, A21, n, mone, one, A22, n);
    q.lowerC = 1;
    gemm_team<cplx, 8>(q, tm);
    __threadfence_block();
    team_sync(tm);
  }
  return true;
}

// ---- unblocked Householder tridiagonalisation of the lower triangle of M ----
// Reflector j is stored explicitly in M(j+1:, j) (unit first entry).
// In a team every CTA forms the reflector and v in its own shared memory (the
// same arithmetic on the same column); w = tau A22 v is split by rows, each
// CTA storing its rows of w into every team member's `ws` (distributed
// shared memory), and the rank-2 update by columns.  The first CTA writes v,
// tau, d and e, after the team has read column j.
__device__ void cta_hetrd(int64_t n, cplx* M, cplx* tau, double* d, double* e, cplx* vs, cplx* ws, double* red,
                          Team tm = Team{0, 1}) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ cplx h_tau, h_scal, h_alpha;
  __shared__ double h_beta;
  for (int64_t j = 0; j + 1 < n; ++j) {
    const int64_t base = j + 1, m = n - base;
    double nrm = 0.0;
    for (int64_t r = 2 + tid; r < m + 1; r += BT) nrm += cabs2(M[IDX2(j + r, j, n)]);  // rows j+2..n-1
    nrm = cta_sum(nrm, red);
    if (tid == 0) {
      const cplx alpha = M[IDX2(base, j, n)];
      if (nrm == 0.0 && alpha.y == 0.0) {
        h_tau = mkc(0.0, 0.0);
        h_beta = alpha.x;
        h_scal = mkc(0.0, 0.0);
      } else {
        const double nr = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + nrm);
        const double beta = (alpha.x >= 0.0) ? -nr : nr;
        h_beta = beta;
        h_tau = mkc((beta - alpha.x) / beta, -alpha.y / beta);
        h_scal = cdiv(mkc(1.0, 0.0), mkc(alpha.x - beta, alpha.y));
      }
      if (tm.rank == 0) {
        d[j] = M[IDX2(j, j, n)].x;
        tau[j] = h_tau;
        e[j] = h_beta;
      }
    }
    __syncthreads();
    for (int64_t r = tid; r < m; r += BT) vs[r] = (r == 0) ? mkc(1.0, 0.0) : cmul(M[IDX2(base + r, j, n)], h_scal);
    __syncthreads();
    // w = tau A22 v for this CTA's rows: lower part (c <= r) by rows, strict
    // upper by columns
    const int64_t per = (m + tm.size - 1) / tm.size, rb0 = tm.rank * per;
    const int64_t rb1 = rb0 + per < m ? rb0 + per : m;
    for (int64_t r = rb0 + tid; r < rb1; r += BT) {
      cplx acc0 = mkc(0.0, 0.0), acc1 = mkc(0.0, 0.0);
      const cplx* Ar = M + IDX2(base + r, base, n);
      int64_t c = 0;
      for (; c + 1 <= r; c += 2) {
        cfma(acc0, Ar[c * n], vs[c]);
        cfma(acc1, Ar[(c + 1) * n], vs[c + 1]);
      }
      if (c <= r) cfma(acc0, Ar[c * n], vs[c]);
      const cplx* Ac = M + IDX2(base, base + r, n);
      for (int64_t rr = r + 1; rr < m; ++rr) cfma_cj(acc1, Ac[rr], vs[rr]);
      const cplx wr = cmul(h_tau, cadd(acc0, acc1));
      if (tm.size > 1) {
        for (int q = 0; q < tm.size; ++q) cg::this_cluster().map_shared_rank(ws, q)[r] = wr;
      } else {
        ws[r] = wr;
      }
    }
    team_sync(tm);
    if (tm.rank == 0)
      for (int64_t r = tid; r < m; r += BT) M[IDX2(base + r, j, n)] = vs[r];
    double dre = 0.0, dim = 0.0;
    for (int64_t r = tid; r < m; r += BT) {
      const cplx t = cmul(cconj(ws[r]), vs[r]);
      dre += t.x, dim += t.y;
    }
    dre = cta_sum(dre, red);
    dim = cta_sum(dim, red);
    if (tid == 0) h_alpha = cscale(cmul(h_tau, mkc(dre, dim)), -0.5);
    __syncthreads();
    for (int64_t r = tid; r < m; r += BT) ws[r] = cadd(ws[r], cmul(h_alpha, vs[r]));
    __syncthreads();
    // A22 -= v w^H + w v^H (lower): warp per column, lanes over rows; the
    // team's CTAs take every size-th column
    for (int64_t c = tm.rank + (int64_t)tm.size * warp; c < m; c += (int64_t)tm.size * (BT / 32)) {
      const cplx wc = cconj(ws[c]), vc = cconj(vs[c]);
      cplx* Acol = M + IDX2(base, base + c, n);
      for (int64_t r = c + lane; r < m; r += 32) {
        cplx a = Acol[r];
        a = csub(a, cadd(cmul(vs[r], wc), cmul(ws[r], vc)));
        if (r == c) a.y = 0.0;
        Acol[r] = a;
      }
    }
    team_sync(tm);
  }
  if (tid == 0 && tm.rank == 0) d[n - 1] = M[IDX2(n - 1, n - 1, n)].x;
  team_sync(tm);
}

__device__ __forceinline__ int bsturm(const double* a, const double* e2, int64_t n, double x, double pivmin) {
  double q = a[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = q < 0.0;
  for (int64_t i = 1; i < n; ++i) {
    q = (a[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

// ---- the whole instance -----------------------------------------------------
// A team solves the instance together up to the tridiagonal matrix (every
// CTA returns from here at the same point); the rest runs on its first CTA.
__device__ void solve_instance(const BatchDesc& D, cplx* vs, cplx* wsv, double* red, cplx* S, cplx* Iv, int* flag,
                               Team tm = Team{0, 1}) {
  const int64_t n = D.n, k = D.k;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  InstWs w;
  carve_inst(D.ws, n, k, &w);
  int64_t* st = D.status;
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  // form M1 (full) and M2 (lower, into L)
  for (int64_t q = tm.rank * BT + tid; q < n * n; q += (int64_t)tm.size * BT) {
    const int64_t i = q % n, j = q / n;
    if (i >= j) {
      const cplx a = D.A[IDX2(i, j, n)], b = D.B[IDX2(i, j, n)];
      w.M1[q] = (i == j) ? mkc(a.x + b.x, 0.0) : cadd(a, b);
      w.L[q] = (i == j) ? mkc(a.x - b.x, 0.0) : csub(a, b);
    } else {
      const cplx a = D.A[IDX2(j, i, n)], b = D.B[IDX2(j, i, n)];
      w.M1[q] = cconj(cadd(a, b));
    }
  }
  __threadfence_block();
  team_sync(tm);
  if (!cta_potrf(n, w.L, w.Linv, st, S, Iv, flag, BSE_ERR_NOT_PD_AMINUSB, tm)) return;
  // W = M1 L ; M = L^H W (lower) into M1
  GemmParams<cplx> p1 = gemm_params<cplx>(n, n, n, OPN, w.M1, n, OPN, w.L, n, one, zero, w.W, n);
  p1.triB = TRI_LO;
  gemm_team<cplx, 8>(p1, tm);
  __threadfence_block();
  team_sync(tm);
  GemmParams<cplx> p2 = gemm_params<cplx>(n, n, n, OPC, w.L, n, OPN, w.W, n, one, zero, w.M1, n);
  p2.triA = TRI_UP;
  p2.lowerC = 1;
  gemm_team<cplx, 8>(p2, tm);
  __threadfence_block();
  team_sync(tm);
  cta_hetrd(n, w.M1, w.tau, w.d, w.e, vs, wsv, red, tm);
  // the rest is split over the team by eigenpairs: pair t belongs to CTA
  // t % size (every member computes the same bounds)
  // tridiagonal: bounds, bisection for the k smallest
  double tn = 0.0, em = 0.0, lo = 1e308, hi = -1e308;
  for (int64_t i = tid; i < n; i += BT) {
    const double ol = i > 0 ? fabs(w.e[i - 1]) : 0.0, orr = i < n - 1 ? fabs(w.e[i]) : 0.0;
    tn = fmax(tn, fabs(w.d[i]) + ol + orr);
    lo = fmin(lo, w.d[i] - ol - orr);
    hi = fmax(hi, w.d[i] + ol + orr);
    if (i < n - 1) {
      if (tm.rank == 0) w.e2[i] = w.e[i] * w.e[i];
      em = fmax(em, w.e[i] * w.e[i]);
    }
  }
  tn = cta_max(tn, red);
  em = cta_max(em, red);
  lo = cta_min(lo, red);
  hi = cta_max(hi, red);
  __threadfence_block();
  team_sync(tm);
  const double pivmin = DBL_MIN * fmax(1.0, em), g = DBL_EPSILON * fmax(tn, DBL_MIN);
  lo -= 2.0 * DBL_EPSILON * tn + 4.0 * pivmin;
  hi += 2.0 * DBL_EPSILON * tn + 4.0 * pivmin;
  for (int64_t t = tm.rank + (int64_t)tm.size * tid; t < k; t += (int64_t)tm.size * BT) {
    double a = lo, b = hi;
    for (int it = 0; it < 256; ++it) {
      const double mid = 0.5 * (a + b), wd = b - a;
      if (wd <= 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)) || wd <= 4.0 * pivmin || mid == a || mid == b) break;
      if (bsturm(w.d, w.e2, n, mid, pivmin) > t) b = mid; else a = mid;
    }
    const double l = 0.5 * (a + b);
    w.lam[t] = l;
    // twisted factorisation vector into Z(:, t)
    double* zc = w.Z + t * n;
    double* sc = w.sc + t * n;
    double x = w.d[0] - l;
    if (fabs(x) < g) x = (x < 0.0) ? -g : g;
    zc[0] = x;
    for (int64_t i = 1; i < n; ++i) {
      x = (w.d[i] - l) - w.e2[i - 1] / x;
      if (fabs(x) < g) x = (x < 0.0) ? -g : g;
      zc[i] = x;
    }
    double y = w.d[n - 1] - l;
    if (fabs(y) < g) y = (y < 0.0) ? -g : g;
    sc[n - 1] = y;
    double best = fabs(zc[n - 1]);
    int64_t r = n - 1;
    for (int64_t i = n - 2; i >= 0; --i) {
      const double ai = w.d[i] - l;
      y = ai - w.e2[i] / y;
      if (fabs(y) < g) y = (y < 0.0) ? -g : g;
      sc[i] = y;
      const double gam = zc[i] + y - ai;
      if (fabs(gam) < best) best = fabs(gam), r = i;
    }
    double nrm2 = 1.0, z = 1.0;
    for (int64_t i = r - 1; i >= 0; --i) {
      z = -(w.e[i] / zc[i]) * z;
      zc[i] = z;
      nrm2 += z * z;
    }
    zc[r] = 1.0;
    z = 1.0;
    for (int64_t i = r; i < n - 1; ++i) {
      z = -(w.e[i] / sc[i + 1]) * z;
      zc[i + 1] = z;
      nrm2 += z * z;
    }
    const double inv = 1.0 / sqrt(nrm2);
    for (int64_t i = 0; i < n; ++i) zc[i] *= inv;
    if (!(l > 0.0)) {
      st[0] = BSE_ERR_NOT_PD_APLUSB;
      st[1] = 0;
    }
    const double om = sqrt(l);
    D.omega[t] = om;
    w.c1[t] = sqrt(om);
    w.c2[t] = 1.0 / sqrt(om);
  }
  __threadfence_block();
  team_sync(tm);
  if (st[0]) return;  // the same word for every member
  // Newton-Schulz: E = Z^T Z - I, Z <- Z - Z E / 2 (k x k small, plain loops)
  for (int64_t q = tm.rank * BT + tid; q < k * k; q += (int64_t)tm.size * BT) {
    const int64_t a = q % k, b = q / k;
    if (a < b) continue;
    const double* za = w.Z + a * n;
    const double* zb = w.Z + b * n;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = fma(za[i], zb[i], s);
    if (a == b) s -= 1.0;
    w.E[a + b * k] = s;
    w.E[b + a * k] = s;
  }
  __threadfence_block();
  team_sync(tm);
  // from here on a member works on its own columns c = rank, rank + size, ...
  const int64_t kc = (k - tm.rank + tm.size - 1) / tm.size;  // this member's column count
  for (int64_t q = tid; q < n * kc; q += BT) {
    const int64_t i = q % n, c = tm.rank + (q / n) * tm.size;
    double s = 0.0;
    for (int64_t b = 0; b < k; ++b) s = fma(w.Z[i + b * n], w.E[b + c * k], s);
    w.sc[i + c * n] = w.Z[i + c * n] - 0.5 * s;
  }
  __threadfence_block();
  __syncthreads();
  for (int64_t q = tid; q < n * kc; q += BT) {
    const int64_t i = q % n, c = tm.rank + (q / n) * tm.size;
    w.VM[i + c * n] = mkc(w.sc[i + c * n], 0.0);
  }
  __threadfence_block();
  __syncthreads();
  // V_M = H_0 ... H_{n-2} Z, one reflector at a time; a warp owns columns
  for (int64_t c = tm.rank + (int64_t)tm.size * warp; c < k; c += (int64_t)tm.size * (BT / 32)) {
    cplx* vc = w.VM + c * n;
    for (int64_t j = n - 2; j >= 0; --j) {
      const cplx* v = w.M1 + IDX2(j + 1, j, n);
      const int64_t m = n - j - 1;
      cplx s = mkc(0.0, 0.0);
      for (int64_t r = lane; r < m; r += 32) cfma_cj(s, v[r], vc[j + 1 + r]);
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      const cplx ts = cmul(w.tau[j], s);
      for (int64_t r = lane; r < m; r += 32) vc[j + 1 + r] = csub(vc[j + 1 + r], cmul(v[r], ts));
      __syncwarp();
    }
  }
  __threadfence_block();
  __syncthreads();
  // P = L^{-H} V_M, column by column (a warp owns a column)
  for (int64_t c = tm.rank + (int64_t)tm.size * warp; c < k; c += (int64_t)tm.size * (BT / 32)) {
    const cplx* vmc = w.VM + c * n;
    cplx* pc = w.P + c * n;
    for (int64_t i = n - 1; i >= 0; --i) {
      const cplx* li = w.L + IDX2(0, i, n);
      cplx s = mkc(0.0, 0.0);
      for (int64_t r = i + 1 + lane; r < n; r += 32) cfma_cj(s, li[r], pc[r]);
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) pc[i] = cscale(csub(vmc[i], s), 1.0 / li[i].x);
      __syncwarp();
    }
  }
  __threadfence_block();
  team_sync(tm);
  // X, Y: v2 = L V_M, X = (c1 P + c2 v2)/2, Y = (c2 v2 - c1 P)/2
  GemmParams<cplx> p3 = gemm_params<cplx>(n, k, n, OPN, w.L, n, OPN, w.VM, n, one, zero, D.X, n);
  p3.triA = TRI_LO;
  p3.epi = EPI_XY;
  p3.P = w.P, p3.ldp = n, p3.c1 = w.c1, p3.c2 = w.c2, p3.Y = D.Y, p3.ldy = n;
  gemm_team<cplx, 8>(p3, tm);
}

// ---- Alg. 3 for one instance --------------------------------------------------
// Workspace: L1, L2, G, Vr (n x n each), tauq, taup (n), d, e, off, e2 (2n),
// Z, sc (2n x k), UB, VB (n x k real), Uc, Vc, T1 (n x k complex), E, c (k).
struct SvdWs {
  cplx *L1, *L2, *G, *Vr, *Linv, *tauq, *taup, *Uc, *Vc, *T1;
  double *d, *e, *off, *e2, *Z, *sc, *UB, *VB, *E, *c1;
};

__host__ __device__ inline size_t carve_svd_inst(char* base, int64_t n, int64_t k, SvdWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = align256(off);
    char* p = base ? base + off : nullptr;
    off += bytes > 0 ? bytes : 1;
    return p;
  };
  const size_t nn = (size_t)n * n, nk = (size_t)n * k;
  SvdWs t;
  t.L1 = (cplx*)take(nn * 16);
  t.L2 = (cplx*)take(nn * 16);
  t.G = (cplx*)take(nn * 16);
  t.Vr = (cplx*)take(nn * 16);
  t.Linv = (cplx*)take(CNB * CNB * 16);
  t.tauq = (cplx*)take(n * 16);
  t.taup = (cplx*)take(n * 16);
  t.Uc = (cplx*)take(nk * 16);
  t.Vc = (cplx*)take(nk * 16);
  t.T1 = (cplx*)take(nk * 16);
  t.d = (double*)take(n * 8);
  t.e = (double*)take(n * 8);
  t.off = (double*)take(2 * n * 8);
  t.e2 = (double*)take(2 * n * 8);
  t.Z = (double*)take(2 * nk * 8);
  t.sc = (double*)take(2 * nk * 8);
  t.UB = (double*)take(nk * 8);
  t.VB = (double*)take(nk * 8);
  t.E = (double*)take((size_t)k * k * 8);
  t.c1 = (double*)take(k * 8);
  if (w) *w = t;
  return align256(off);
}

size_t batched_svd_inst_bytes(int64_t n, int64_t k) { return carve_svd_inst(nullptr, n, k, nullptr); }

// Householder reflector of x = (alpha, rest) with ||rest||^2 = xn2: H^H x = beta e_1
__device__ __forceinline__ void house_params(cplx alpha, double xn2, cplx* tau, cplx* scal, double* beta) {
  if (xn2 == 0.0 && alpha.y == 0.0) {
    *tau = mkc(0.0, 0.0);
    *beta = alpha.x;
    *scal = mkc(0.0, 0.0);
  } else {
    const double nr = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
    const double b = (alpha.x >= 0.0) ? -nr : nr;
    *beta = b;
    *tau = mkc((b - alpha.x) / b, -alpha.y / b);
    *scal = cdiv(mkc(1.0, 0.0), mkc(alpha.x - b, alpha.y));
  }
}

// unblocked bidiagonalisation of G (n x n, ld n): left reflector u_i kept in
// G(i:, i) (unit first entry), right reflector v_i in Vr(i+1:, i)
// In a team every CTA forms u and v (the left and right reflectors) in its
// own shared memory from the same column / row; the updates are split by
// columns, t = tau G v by rows (each CTA storing its rows of t into every
// member's `ts`); the first CTA writes u, v, the taus, d and e after the
// team has read what they overwrite.
__device__ void cta_gebrd(int64_t n, cplx* G, cplx* Vr, cplx* tauq, cplx* taup, double* d, double* e, cplx* ts,
                          double* red, cplx* us, cplx* vrs, Team tm = Team{0, 1}) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ cplx h_tau, h_scal;
  __shared__ double h_beta;
  const int64_t cstride = (int64_t)tm.size * (BT / 32);
  for (int64_t i = 0; i < n; ++i) {
    // left reflector on G(i:, i)
    double nrm = 0.0;
    for (int64_t r = i + 1 + tid; r < n; r += BT) nrm += cabs2(G[IDX2(r, i, n)]);
    nrm = cta_sum(nrm, red);
    if (tid == 0) {
      cplx t, sc;
      double b;
      house_params(G[IDX2(i, i, n)], nrm, &t, &sc, &b);
      h_tau = t, h_scal = sc, h_beta = b;
      if (tm.rank == 0) {
        tauq[i] = t;
        d[i] = b;
      }
    }
    __syncthreads();
    for (int64_t r = i + tid; r < n; r += BT) us[r - i] = (r == i) ? mkc(1.0, 0.0) : cmul(G[IDX2(r, i, n)], h_scal);
    __syncthreads();
    // G(i:, c) -= conj(tau) u (u^H G(i:, c)), c > i: warp per column
    const cplx ctau = cconj(h_tau);
    for (int64_t c = i + 1 + tm.rank + (int64_t)tm.size * warp; c < n; c += cstride) {
      cplx sdot = mkc(0.0, 0.0);
      for (int64_t r = i + lane; r < n; r += 32) cfma_cj(sdot, us[r - i], G[IDX2(r, c, n)]);
      for (int o = 16; o > 0; o >>= 1) {
        sdot.x += __shfl_xor_sync(0xffffffffu, sdot.x, o);
        sdot.y += __shfl_xor_sync(0xffffffffu, sdot.y, o);
      }
      const cplx f = cmul(ctau, sdot);
      for (int64_t r = i + lane; r < n; r += 32) G[IDX2(r, c, n)] = csub(G[IDX2(r, c, n)], cmul(us[r - i], f));
    }
    team_sync(tm);
    if (tm.rank == 0)
      for (int64_t r = i + tid; r < n; r += BT) G[IDX2(r, i, n)] = us[r - i];
    if (i + 1 >= n) break;
    // right reflector from x = conj(G(i, i+1:))
    nrm = 0.0;
    for (int64_t c = i + 2 + tid; c < n; c += BT) nrm += cabs2(G[IDX2(i, c, n)]);
    nrm = cta_sum(nrm, red);
    if (tid == 0) {
      cplx t, sc;
      double b;
      house_params(cconj(G[IDX2(i, i + 1, n)]), nrm, &t, &sc, &b);
      h_tau = t, h_scal = sc, h_beta = b;
      if (tm.rank == 0) {
        taup[i] = t;
        e[i] = b;
      }
    }
    __syncthreads();
    for (int64_t c = i + 1 + tid; c < n; c += BT) {
      const cplx v = (c == i + 1) ? mkc(1.0, 0.0) : cmul(cconj(G[IDX2(i, c, n)]), h_scal);
      vrs[c - i - 1] = v;
      if (tm.rank == 0) Vr[IDX2(c, i, n)] = v;
    }
    __syncthreads();
    // G(i+1:, i+1:) <- G - tau (G v) v^H: t = G v by rows (this CTA's rows),
    // then warp per column
    const int64_t m = n - i - 1, per = (m + tm.size - 1) / tm.size, rb0 = tm.rank * per;
    const int64_t rb1 = rb0 + per < m ? rb0 + per : m;
    for (int64_t rr = rb0 + tid; rr < rb1; rr += BT) {
      const int64_t r = i + 1 + rr;
      cplx acc = mkc(0.0, 0.0);
      for (int64_t c = i + 1; c < n; ++c) cfma(acc, G[IDX2(r, c, n)], vrs[c - i - 1]);
      const cplx tr = cmul(h_tau, acc);
      if (tm.size > 1) {
        for (int q = 0; q < tm.size; ++q) cg::this_cluster().map_shared_rank(ts, q)[rr] = tr;
      } else {
        ts[rr] = tr;
      }
    }
    team_sync(tm);
    for (int64_t c = i + 1 + tm.rank + (int64_t)tm.size * warp; c < n; c += cstride) {
      const cplx vc = cconj(vrs[c - i - 1]);
      for (int64_t r = i + 1 + lane; r < n; r += 32) G[IDX2(r, c, n)] = csub(G[IDX2(r, c, n)], cmul(ts[r - i - 1], vc));
    }
    team_sync(tm);
  }
}

// A team splits Alg. 3 as it splits Alg. 2: the Choleskys, G = L1^H L2 and
// the bidiagonalisation by tiles, columns and rows, the k-sized tail by
// singular triplets (triplet t on CTA t % size).  us, vrs: two n-entry
// shared buffers of the bidiagonalisation (S and Iv are free by then).
__device__ void solve_instance_svd(const BatchDesc& D, cplx* vs, double* red, cplx* S, cplx* Iv, int* flag,
                                   cplx* us, Team tm = Team{0, 1}) {
  const int64_t n = D.n, k = D.k;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  SvdWs w;
  carve_svd_inst(D.ws, n, k, &w);
  int64_t* st = D.status;
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  for (int64_t q = tm.rank * BT + tid; q < n * n; q += (int64_t)tm.size * BT) {
    const int64_t i = q % n, j = q / n;
    if (i >= j) {
      const cplx a = D.A[IDX2(i, j, n)], b = D.B[IDX2(i, j, n)];
      w.L1[q] = (i == j) ? mkc(a.x + b.x, 0.0) : cadd(a, b);
      w.L2[q] = (i == j) ? mkc(a.x - b.x, 0.0) : csub(a, b);
    }
  }
  __threadfence_block();
  team_sync(tm);
  if (!cta_potrf(n, w.L1, w.Linv, st, S, Iv, flag, BSE_ERR_NOT_PD_APLUSB, tm)) return;
  if (!cta_potrf(n, w.L2, w.Linv, st, S, Iv, flag, BSE_ERR_NOT_PD_AMINUSB, tm)) return;
  // G = L1^H L2
  GemmParams<cplx> pg = gemm_params<cplx>(n, n, n, OPC, w.L1, n, OPN, w.L2, n, one, zero, w.G, n);
  pg.triA = TRI_UP;
  pg.triB = TRI_LO;
  gemm_team<cplx, 8>(pg, tm);
  __threadfence_block();
  team_sync(tm);
  cta_gebrd(n, w.G, w.Vr, w.tauq, w.taup, w.d, w.e, vs, red, us, S, tm);
  // Golub-Kahan tridiagonal (zero diagonal), size N = 2n
  const int64_t N = 2 * n;
  double tn = 0.0, em = 0.0;
  for (int64_t i = tid; i < N - 1; i += BT) {
    const double o = (i & 1) ? w.e[i >> 1] : w.d[i >> 1];
    if (tm.rank == 0) {
      w.off[i] = o;
      w.e2[i] = o * o;
    }
    tn = fmax(tn, 2.0 * fabs(o));
    em = fmax(em, o * o);
  }
  tn = cta_max(tn, red);
  em = cta_max(em, red);
  __threadfence_block();
  team_sync(tm);
  const double pivmin = DBL_MIN * fmax(1.0, em), g = DBL_EPSILON * fmax(tn, DBL_MIN);
  const double lo0 = -tn - 4.0 * pivmin, hi0 = tn + 4.0 * pivmin;
  for (int64_t t = tm.rank + (int64_t)tm.size * tid; t < k; t += (int64_t)tm.size * BT) {
    const int tt = (int)(n + t);  // the (t+1)-th smallest positive eigenvalue of TGK
    double a = lo0, b = hi0;
    for (int it = 0; it < 256; ++it) {
      const double mid = 0.5 * (a + b), wd = b - a;
      if (wd <= 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)) || wd <= 4.0 * pivmin || mid == a || mid == b) break;
      double q = -mid;
      if (fabs(q) < pivmin) q = -pivmin;
      int cnt = q < 0.0;
      for (int64_t i = 1; i < N; ++i) {
        q = -mid - w.e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
      }
      if (cnt > tt) b = mid; else a = mid;
    }
    const double l = 0.5 * (a + b);
    double* zc = w.Z + t * N;
    double* sc = w.sc + t * N;
    double x = -l;
    if (fabs(x) < g) x = (x < 0.0) ? -g : g;
    zc[0] = x;
    for (int64_t i = 1; i < N; ++i) {
      x = -l - w.e2[i - 1] / x;
      if (fabs(x) < g) x = (x < 0.0) ? -g : g;
      zc[i] = x;
    }
    double y = -l;
    if (fabs(y) < g) y = (y < 0.0) ? -g : g;
    sc[N - 1] = y;
    double best = fabs(zc[N - 1]);
    int64_t r = N - 1;
    for (int64_t i = N - 2; i >= 0; --i) {
      y = -l - w.e2[i] / y;
      if (fabs(y) < g) y = (y < 0.0) ? -g : g;
      sc[i] = y;
      const double gam = zc[i] + y + l;
      if (fabs(gam) < best) best = fabs(gam), r = i;
    }
    double nrm2 = 1.0, z = 1.0;
    for (int64_t i = r - 1; i >= 0; --i) {
      z = -(w.off[i] / zc[i]) * z;
      zc[i] = z;
      nrm2 += z * z;
    }
    zc[r] = 1.0;
    z = 1.0;
    for (int64_t i = r; i < N - 1; ++i) {
      z = -(w.off[i] / sc[i + 1]) * z;
      zc[i + 1] = z;
      nrm2 += z * z;
    }
    const double inv = sqrt(2.0 / nrm2);  // u, v halves get unit norm
    for (int64_t i = 0; i < n; ++i) {
      w.VB[i + t * n] = zc[2 * i] * inv;
      w.UB[i + t * n] = zc[2 * i + 1] * inv;
    }
    if (!(l > 0.0)) {
      st[0] = BSE_ERR_NOT_PD_APLUSB;
      st[1] = 0;
    }
    D.omega[t] = l;
    w.c1[t] = 1.0 / sqrt(l);
  }
  __threadfence_block();
  team_sync(tm);
  if (st[0]) return;  // the same word for every member
  // Newton-Schulz on U_B and V_B (k x k Gram, plain loops); from the update
  // on a member works on its own columns c = rank, rank + size, ...
  const int64_t kc = (k - tm.rank + tm.size - 1) / tm.size;
  for (int pass = 0; pass < 2; ++pass) {
    double* Zm = pass == 0 ? w.UB : w.VB;
    for (int64_t q = tm.rank * BT + tid; q < k * k; q += (int64_t)tm.size * BT) {
      const int64_t a = q % k, b = q / k;
      if (a < b) continue;
      double s2 = 0.0;
      for (int64_t i = 0; i < n; ++i) s2 = fma(Zm[i + a * n], Zm[i + b * n], s2);
      if (a == b) s2 -= 1.0;
      w.E[a + b * k] = s2;
      w.E[b + a * k] = s2;
    }
    __threadfence_block();
    team_sync(tm);
    for (int64_t q = tid; q < n * kc; q += BT) {
      const int64_t i = q % n, c = tm.rank + (q / n) * tm.size;
      double s2 = 0.0;
      for (int64_t b = 0; b < k; ++b) s2 = fma(Zm[i + b * n], w.E[b + c * k], s2);
      w.sc[i + c * n] = Zm[i + c * n] - 0.5 * s2;
    }
    __threadfence_block();
    __syncthreads();
    cplx* out = pass == 0 ? w.Uc : w.Vc;
    for (int64_t q = tid; q < n * kc; q += BT) {
      const int64_t i = q % n, c = tm.rank + (q / n) * tm.size;
      out[i + c * n] = mkc(w.sc[i + c * n], 0.0);
    }
    __threadfence_block();
    team_sync(tm);  // E is rewritten by the next pass
  }
  // back-transformations: U = H_L(0) ... H_L(n-1) U_B, V = H_R(0) ... H_R(n-2) V_B
  for (int64_t c = tm.rank + (int64_t)tm.size * warp; c < k; c += (int64_t)tm.size * (BT / 32)) {
    cplx* uc = w.Uc + c * n;
    for (int64_t j = n - 1; j >= 0; --j) {
      const cplx* u = w.G + IDX2(j, j, n);
      const int64_t m = n - j;
      cplx sdot = mkc(0.0, 0.0);
      for (int64_t r = lane; r < m; r += 32) cfma_cj(sdot, u[r], uc[j + r]);
      for (int o = 16; o > 0; o >>= 1) {
        sdot.x += __shfl_xor_sync(0xffffffffu, sdot.x, o);
        sdot.y += __shfl_xor_sync(0xffffffffu, sdot.y, o);
      }
      const cplx f = cmul(w.tauq[j], sdot);
      for (int64_t r = lane; r < m; r += 32) uc[j + r] = csub(uc[j + r], cmul(u[r], f));
      __syncwarp();
    }
    cplx* vc = w.Vc + c * n;
    for (int64_t j = n - 2; j >= 0; --j) {
      const cplx* v = w.Vr + IDX2(j + 1, j, n);
      const int64_t m = n - j - 1;
      cplx sdot = mkc(0.0, 0.0);
      for (int64_t r = lane; r < m; r += 32) cfma_cj(sdot, v[r], vc[j + 1 + r]);
      for (int o = 16; o > 0; o >>= 1) {
        sdot.x += __shfl_xor_sync(0xffffffffu, sdot.x, o);
        sdot.y += __shfl_xor_sync(0xffffffffu, sdot.y, o);
      }
      const cplx f = cmul(w.taup[j], sdot);
      for (int64_t r = lane; r < m; r += 32) vc[j + 1 + r] = csub(vc[j + 1 + r], cmul(v[r], f));
      __syncwarp();
    }
  }
  __threadfence_block();
  team_sync(tm);
  // T1 = L1 U; X, Y from T1 and L2 V, c1 = c2 = omega^{-1/2}
  GemmParams<cplx> p1 = gemm_params<cplx>(n, k, n, OPN, w.L1, n, OPN, w.Uc, n, one, zero, w.T1, n);
  p1.triA = TRI_LO;
  gemm_team<cplx, 8>(p1, tm);
  __threadfence_block();
  team_sync(tm);
  GemmParams<cplx> p2 = gemm_params<cplx>(n, k, n, OPN, w.L2, n, OPN, w.Vc, n, one, zero, D.X, n);
  p2.triA = TRI_LO;
  p2.epi = EPI_XY;
  p2.P = w.T1, p2.ldp = n, p2.c1 = w.c1, p2.c2 = w.c1, p2.Y = D.Y, p2.ldy = n;
  gemm_team<cplx, 8>(p2, tm);
}

__global__ void __launch_bounds__(BT, 1) batched_svd_kernel(const BatchDesc* __restrict__ desc, int64_t count,
                                                            int* counter) {
  extern __shared__ cplx dyn[];
  cplx* vs = dyn;                    // 1024
  cplx* S = dyn + 2048;              // CNB x CLD
  cplx* Iv = S + CNB * CLD;          // CNB x CLD
  __shared__ double red[BT / 32];
  __shared__ int next, flag;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = next;
    __syncthreads();
    if (idx >= count) break;
    solve_instance_svd(desc[idx], vs, red, S, Iv, &flag, dyn + 1024);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(BT, 1) batched_chol_kernel(const BatchDesc* __restrict__ desc, int64_t count,
                                                             int* counter) {
  extern __shared__ cplx dyn[];
  cplx* vs = dyn;                    // 1024
  cplx* wsv = dyn + 1024;            // 1024
  cplx* S = dyn + 2048;              // CNB x CLD
  cplx* Iv = S + CNB * CLD;          // CNB x CLD
  __shared__ double red[BT / 32];
  __shared__ int next, flag;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = next;
    __syncthreads();
    if (idx >= count) break;
    solve_instance(desc[idx], vs, wsv, red, S, Iv, &flag);
    __syncthreads();
  }
}

// With teams: the clusters take the first `nbig` instances of the
// size-ordered queue one at a time, a team per instance; when none is left,
// every CTA takes the remaining (small) instances alone from a second
// counter.  METHOD: BSE_METHOD_CHOL (Alg. 2) or BSE_METHOD_SVD (Alg. 3).
template <int METHOD>
__global__ void __launch_bounds__(BT, 1) batched_team_kernel(const BatchDesc* __restrict__ desc, int64_t count,
                                                             int64_t nbig, int* counters) {
  extern __shared__ cplx dyn[];
  cplx* vs = dyn;                    // 1024
  cplx* wsv = dyn + 1024;            // 1024
  cplx* S = dyn + 2048;              // CNB x CLD
  cplx* Iv = S + CNB * CLD;          // CNB x CLD
  __shared__ double red[BT / 32];
  __shared__ int next, flag;
  cg::cluster_group cl = cg::this_cluster();
  const Team tm{(int)cl.block_rank(), (int)cl.num_blocks()};
  for (;;) {
    if (tm.rank == 0 && threadIdx.x == 0) {
      const int i = atomicAdd(counters, 1);
      for (int q = 0; q < tm.size; ++q) *cl.map_shared_rank(&next, q) = i;
    }
    cl.sync();
    const int idx = next;
    cl.sync();
    if (idx >= nbig) break;
    if (METHOD == BSE_METHOD_SVD)
      solve_instance_svd(desc[idx], vs, red, S, Iv, &flag, wsv, tm);
    else
      solve_instance(desc[idx], vs, wsv, red, S, Iv, &flag, tm);
    __syncthreads();
  }
  for (;;) {
    if (threadIdx.x == 0) next = (int)nbig + atomicAdd(counters + 1, 1);
    __syncthreads();
    const int idx = next;
    __syncthreads();
    if (idx >= count) break;
    if (METHOD == BSE_METHOD_SVD)
      solve_instance_svd(desc[idx], vs, red, S, Iv, &flag, wsv);
    else
      solve_instance(desc[idx], vs, wsv, red, S, Iv, &flag);
    __syncthreads();
  }
}

size_t batched_smem_bytes() { return sizeof(cplx) * (2048 + 2 * CNB * CLD); }

int batched_team_default() { return BATCH_TEAM; }
int batched_team_min_n_default() { return BATCH_TEAM_MIN_N; }

// Largest grid of whole teams of `team` CTAs that can be resident at once
// (0: none), looked up once per device, method and team size.
static int team_grid_query(const void* kern, size_t smem, int team) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = team, attr[0].val.clusterDim.y = 1, attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(team, 1, 1);
  cfg.blockDim = dim3(BT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters * team;
}

static int team_grid(int method, size_t smem, int team) {
  constexpr int kMaxDev = 64;
  // grid + 1 per method and team size 1, 2, 4, 8 (0: not yet looked up)
  static std::atomic<int> grid_of[kMaxDev][2][4];
  const int slot = team == 8 ? 3 : team == 4 ? 2 : team == 2 ? 1 : 0, ms = method == BSE_METHOD_SVD ? 1 : 0;
  const void* kern = ms ? (const void*)batched_team_kernel<BSE_METHOD_SVD> : (const void*)batched_team_kernel<BSE_METHOD_CHOL>;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return team_grid_query(kern, smem, team);
  }
  int g = grid_of[dev][ms][slot].load(std::memory_order_relaxed);
  if (!g) {
    g = team_grid_query(kern, smem, team) + 1;
    grid_of[dev][ms][slot].store(g, std::memory_order_relaxed);
  }
  return g - 1;
}

bse_status batched_chol_launch(cudaStream_t s, const void* desc, int64_t count, int* counter, int grid, int method,
                               int64_t nbig, int team) {
  const size_t smem = batched_smem_bytes();
  bse_status r = set_smem_attr((const void*)batched_chol_kernel, (int)smem);
  if (!r) r = set_smem_attr((const void*)batched_svd_kernel, (int)smem);
  if (!r) r = set_smem_attr((const void*)batched_team_kernel<BSE_METHOD_CHOL>, (int)smem);
  if (!r) r = set_smem_attr((const void*)batched_team_kernel<BSE_METHOD_SVD>, (int)smem);
  if (r) return r;
  BSE_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
  const int tgrid = (nbig > 0 && team > 1) ? team_grid(method, smem, team) : 0;
  if (tgrid > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = team, attr[0].val.clusterDim.y = 1, attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)tgrid, 1, 1);
    cfg.blockDim = dim3(BT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (method == BSE_METHOD_SVD)
      BSE_CUDA(cudaLaunchKernelEx(&cfg, batched_team_kernel<BSE_METHOD_SVD>, (const BatchDesc*)desc, count, nbig,
                                  counter));
    else
      BSE_CUDA(cudaLaunchKernelEx(&cfg, batched_team_kernel<BSE_METHOD_CHOL>, (const BatchDesc*)desc, count, nbig,
                                  counter));
  } else if (method == BSE_METHOD_SVD) {
    batched_svd_kernel<<<grid, BT, smem, s>>>((const BatchDesc*)desc, count, counter);
  } else {
    batched_chol_kernel<<<grid, BT, smem, s>>>((const BatchDesc*)desc, count, counter);
  }
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

size_t batched_desc_bytes() { return sizeof(BatchDesc); }

void batched_fill_desc(void* slot, int64_t n, int64_t k, const void* A, const void* B, double* omega, void* X, void* Y,
                       char* ws, int64_t* status) {
  BatchDesc d;
  d.n = n, d.k = k, d.A = (const cplx*)A, d.B = (const cplx*)B, d.omega = omega, d.X = (cplx*)X, d.Y = (cplx*)Y;
  d.ws = ws, d.status = status;
  *(BatchDesc*)slot = d;
}

// ---- one instance, no allocation ----------------------------------------------
// The Cholesky pipeline of ONE instance (the same device routines as
// batched_chol_kernel) with its parameters passed by value and its workspace
// and two status words in scratch memory the caller hands in: no queue
// counter and no descriptor table, so the host needs no device allocation
// for it.  The status words must start at zero; the kernel clears them
// itself before use.
__global__ void __launch_bounds__(BT, 1) single_chol_kernel(BatchDesc d) {
  extern __shared__ cplx dyn[];
  cplx* vs = dyn;                    // 1024
  cplx* wsv = dyn + 1024;            // 1024
  cplx* S = dyn + 2048;              // CNB x CLD
  cplx* Iv = S + CNB * CLD;          // CNB x CLD
  __shared__ double red[BT / 32];
  __shared__ int flag;
  if (threadIdx.x == 0) {
    d.status[0] = 0;
    d.status[1] = 0;
  }
  __threadfence_block();
  __syncthreads();
  solve_instance(d, vs, wsv, red, S, Iv, &flag);
}

cudaError_t single_chol_prepare() {
  return cudaFuncSetAttribute(single_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batched_smem_bytes());
}

cudaError_t single_chol_launch(cudaStream_t s, int64_t n, int64_t k, const void* A, const void* B, double* omega,
                               void* X, void* Y, char* ws, int64_t* status) {
  BatchDesc d;
  d.n = n, d.k = k, d.A = (const cplx*)A, d.B = (const cplx*)B, d.omega = omega, d.X = (cplx*)X, d.Y = (cplx*)Y;
  d.ws = ws, d.status = status;
  single_chol_kernel<<<1, BT, batched_smem_bytes(), s>>>(d);
  bse_count_launch();
  return cudaGetLastError();
}
