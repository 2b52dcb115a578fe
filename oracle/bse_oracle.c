/*
 * bse_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * form-I Bethe-Salpeter eigenproblem H1 = [A B; -B -A] (A, B Hermitian,
 * A+B and A-B positive definite), Benner & Penke, arXiv 2008.08825.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or constant with the
 * CUDA library.
 *
 * Storage: every matrix is complex128, column-major, element (i,j) at
 * p[i + j*ld].  Only the lower triangle of the Hermitian inputs is read.
 *
 * What each function follows:
 *   oracle_cholesky       Alg. 2 step 1 / Alg. 3 steps 1-2 (L L^H = M),
 *                         the textbook right-looking column algorithm.
 *   oracle_congruence     Alg. 2 step 2, M = L^H (A+B) L, explicit loops.
 *   oracle_product        Alg. 3 step 3, G = L1^H L2, explicit loops.
 *   oracle_jacobi_eigh    two-sided cyclic complex Jacobi (Jacobi 1846,
 *                         relative stopping rule of Demmel & Veselic 1992)
 *                         for the Hermitian eigendecomposition of Alg. 2.
 *   oracle_jacobi_svd     one-sided cyclic Jacobi (Hestenes 1958) for the
 *                         SVD of Alg. 3.
 *   oracle_solve_chol     Alg. 2 end to end (steps 1-6).
 *   oracle_solve_svd      Alg. 3 end to end (steps 1-6).
 *   oracle_grad           first-order perturbation of omega (Thm. 3 item 3
 *                         with the Sigma-normalisation of Thm. 4 / Eq. (13)):
 *                         d omega_i = x^H dA x + y^H dA y + x^H dB y + y^H dB x.
 *
 * Parallelism: OpenMP over the disjoint rotation pairs of one round of a
 * round-robin (circle-method) ordering, and over independent columns in the
 * triangular loops.  Every pair / column is computed by one thread with a
 * fixed operation order, so the results are bit-identical for any thread
 * count.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

#define AT(p, i, j, ld) ((p)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)])

enum {
  ORACLE_OK = 0,
  ORACLE_ERR_ARG = 1,
  ORACLE_ERR_NOT_PD_AMINUSB = 2,
  ORACLE_ERR_NOT_PD_APLUSB = 3,
  ORACLE_ERR_NO_CONVERGENCE = 4,
  ORACLE_ERR_NOMEM = 8
};

#define ORACLE_MAX_SWEEPS 60

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Cholesky factorisation L L^H = M of a Hermitian matrix (lower triangle of
 * M is read).  Right-looking column algorithm: for column j, the pivot is
 * the updated diagonal entry; the column below is divided by its square
 * root; then the trailing lower triangle receives the rank-1 update
 * -l_j l_j^H.  Returns 0, or the 1-based index of the first column whose
 * pivot is not > 0 (or is NaN), like LAPACK's info.  L is lower triangular
 * with a real positive diagonal; its strict upper triangle is set to 0.
 */
int64_t oracle_cholesky(int64_t n, const zc* M, int64_t ldm, zc* L, int64_t ldl) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i)
      AT(L, i, j, ldl) = (i >= j) ? AT(M, i, j, ldm) : 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double d = creal(AT(L, j, j, ldl));
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    AT(L, j, j, ldl) = ljj;
    for (int64_t i = j + 1; i < n; ++i) AT(L, i, j, ldl) /= ljj;
    /* trailing update, column k of the remaining lower triangle */
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; ++k) {
      zc lkj = conj(AT(L, k, j, ldl));
      for (int64_t i = k; i < n; ++i) AT(L, i, k, ldl) -= AT(L, i, j, ldl) * lkj;
    }
  }
  return 0;
}

/* M = L^H * M1 * L, with M1 Hermitian (lower triangle read) and L lower
 * triangular.  T = M1 L first (M1 expanded to full Hermitian), then
 * M = L^H T.  Written out as plain triple loops; the full (Hermitian up to
 * rounding) product is returned, lower triangle taken as authoritative.   */
int oracle_congruence(int64_t n, const zc* M1, int64_t ld1, const zc* L, int64_t ldl, zc* M,
                      int64_t ldm) {
  zc* H = (zc*)malloc(sizeof(zc) * n * n);
  zc* T = (zc*)malloc(sizeof(zc) * n * n);
  if (!H || !T) {
    free(H);
    free(T);
    return ORACLE_ERR_NOMEM;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i)
      AT(H, i, j, n) = (i >= j) ? AT(M1, i, j, ld1) : conj(AT(M1, j, i, ld1));
  /* T(:,j) = sum_{k>=j} H(:,k) L(k,j) */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) AT(T, i, j, n) = 0.0;
    for (int64_t k = j; k < n; ++k) {
      zc lkj = AT(L, k, j, ldl);
      for (int64_t i = 0; i < n; ++i) AT(T, i, j, n) += AT(H, i, k, n) * lkj;
    }
  }
  /* M(i,j) = sum_{k>=i} conj(L(k,i)) T(k,j) */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      zc s = 0.0;
      for (int64_t k = i; k < n; ++k) s += conj(AT(L, k, i, ldl)) * AT(T, k, j, n);
      AT(M, i, j, ldm) = s;
    }
  }
  /* Hermitian by construction: make it exactly so from the lower triangle */
  for (int64_t j = 0; j < n; ++j) {
    AT(M, j, j, ldm) = creal(AT(M, j, j, ldm));
    for (int64_t i = j + 1; i < n; ++i) AT(M, j, i, ldm) = conj(AT(M, i, j, ldm));
  }
  free(H);
  free(T);
  return ORACLE_OK;
}

/* G = L1^H * L2 with L1, L2 lower triangular: G(i,j) = sum_{k>=max(i,j)}
 * conj(L1(k,i)) L2(k,j).                                                  */
void oracle_product(int64_t n, const zc* L1, int64_t ld1, const zc* L2, int64_t ld2, zc* G,
                    int64_t ldg) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      zc s = 0.0;
      int64_t k0 = i > j ? i : j;
      for (int64_t k = k0; k < n; ++k) s += conj(AT(L1, k, i, ld1)) * AT(L2, k, j, ld2);
      AT(G, i, j, ldg) = s;
    }
  }
}

/* Round-robin (circle method) schedule on m = even number of slots:
 * slot 0 is fixed, slots 1..m-1 rotate.  In round r, position `pos` holds
 * player 0 (pos 0) or 1 + (pos - 1 + r) mod (m - 1).  Pair k of the round is
 * (position k, position m-1-k).  Every unordered pair meets exactly once in
 * the m-1 rounds of a sweep.                                              */
static int64_t rr_player(int64_t m, int64_t r, int64_t pos) {
  if (pos == 0) return 0;
  return 1 + (pos - 1 + r) % (m - 1);
}

/* Complex Jacobi rotation for the 2x2 Hermitian (or Gram) matrix
 * [[a, g], [conj(g), b]] with g = |g| e^{i phi}: with D = diag(1, e^{-i phi})
 * the matrix becomes real, and the real rotation R = [[c, s], [-s, c]] with
 * t = s/c the smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (b - a)/(2|g|),
 * diagonalises it.  J = D R = [[c, s], [-s e^{-i phi}, c e^{-i phi}]].     */
typedef struct {
  double c, s, t, absg;
  zc eph; /* e^{-i phi} */
} rot_t;

static rot_t make_rot(double a, double b, zc g) {
  rot_t r;
  r.absg = cabs(g);
  r.eph = conj(g) / r.absg;
  double zeta = (b - a) / (2.0 * r.absg);
  double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  r.t = t;
  r.c = 1.0 / sqrt(1.0 + t * t);
  r.s = r.c * t;
  return r;
}

/* [u, v] <- [u, v] J  (columns of length len, stride 1) */
static void rot_cols(int64_t len, zc* u, zc* v, rot_t r) {
  zc se = r.s * r.eph, ce = r.c * r.eph;
  for (int64_t i = 0; i < len; ++i) {
    zc up = u[i], vp = v[i];
    u[i] = r.c * up - se * vp;
    v[i] = r.s * up + ce * vp;
  }
}

/* ------------------------------------------------------------------------
 * One-sided (Hestenes) cyclic Jacobi SVD  G = U diag(sigma) V^H.
 * W = G is rotated from the right until its columns are mutually orthogonal:
 * a pair (p, q) is rotated when |w_p^H w_q| > tol * ||w_p|| ||w_q||,
 * tol = sqrt(n) * 2^-53 (the rounding floor of an inner product of length n).
 * The sweep loop stops after a sweep without rotation.  Then
 * sigma_j = ||w_j||, u_j = w_j / sigma_j, and V holds the accumulated
 * rotations.  Output unordered (caller sorts).
 */
int oracle_jacobi_svd(int64_t n, const zc* G, int64_t ldg, double* sigma, zc* U, int64_t ldu,
                      zc* V, int64_t ldv, int* sweeps_out) {
  zc* W = (zc*)malloc(sizeof(zc) * n * n);
  zc* Vw = (zc*)malloc(sizeof(zc) * n * n);
  if (!W || !Vw) {
    free(W);
    free(Vw);
    return ORACLE_ERR_NOMEM;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      AT(W, i, j, n) = AT(G, i, j, ldg);
      AT(Vw, i, j, n) = (i == j) ? 1.0 : 0.0;
    }
  const double tol = sqrt((double)n) * (DBL_EPSILON / 2.0);
  const int64_t m = (n % 2 == 0) ? n : n + 1;
  int sweep, converged = 0;
  for (sweep = 1; sweep <= ORACLE_MAX_SWEEPS && n > 1; ++sweep) {
    int64_t rotated = 0;
    for (int64_t r = 0; r < m - 1; ++r) {
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : rotated)
      for (int64_t k = 0; k < m / 2; ++k) {
        int64_t p = rr_player(m, r, k), q = rr_player(m, r, m - 1 - k);
        if (p >= n || q >= n) continue;
        if (p > q) {
          int64_t tmp = p;
          p = q;
          q = tmp;
        }
        zc* wp = &AT(W, 0, p, n);
        zc* wq = &AT(W, 0, q, n);
        double alpha = 0.0, beta = 0.0;
        zc gamma = 0.0;
        for (int64_t i = 0; i < n; ++i) {
          alpha += creal(wp[i]) * creal(wp[i]) + cimag(wp[i]) * cimag(wp[i]);
          beta += creal(wq[i]) * creal(wq[i]) + cimag(wq[i]) * cimag(wq[i]);
          gamma += conj(wp[i]) * wq[i];
        }
        if (cabs(gamma) > tol * sqrt(alpha) * sqrt(beta)) {
          rot_t rt = make_rot(alpha, beta, gamma);
          rot_cols(n, wp, wq, rt);
          rot_cols(n, &AT(Vw, 0, p, n), &AT(Vw, 0, q, n), rt);
          rotated += 1;
        }
      }
    }
    if (rotated == 0) {
      converged = 1;
      break;
    }
  }
  if (n <= 1) converged = 1, sweep = 0;
  for (int64_t j = 0; j < n; ++j) {
    double s2 = 0.0;
    for (int64_t i = 0; i < n; ++i)
      s2 += creal(AT(W, i, j, n)) * creal(AT(W, i, j, n)) + cimag(AT(W, i, j, n)) * cimag(AT(W, i, j, n));
    double s = sqrt(s2);
    sigma[j] = s;
    for (int64_t i = 0; i < n; ++i) {
      AT(U, i, j, ldu) = AT(W, i, j, n) / s;
      AT(V, i, j, ldv) = AT(Vw, i, j, n);
    }
  }
  if (sweeps_out) *sweeps_out = sweep;
  free(W);
  free(Vw);
  return converged ? ORACLE_OK : ORACLE_ERR_NO_CONVERGENCE;
}

/* ------------------------------------------------------------------------
 * Two-sided cyclic Jacobi for a Hermitian positive definite M (lower
 * triangle read):  M = V diag(lam) V^H.  A pair (p, q) is rotated when
 * |m_pq| > tol * sqrt(m_pp m_qq), tol = n * 2^-53 (relative criterion for
 * positive definite matrices).  The rotations of one round act on disjoint
 * index pairs, so they are computed from the same matrix and applied to all
 * columns (M J), then to all rows (J^H M); the annihilated entries are then
 * set to exactly 0.
 */
int oracle_jacobi_eigh(int64_t n, const zc* M, int64_t ldm, double* lam, zc* V, int64_t ldv,
                       int* sweeps_out) {
  zc* W = (zc*)malloc(sizeof(zc) * n * n);
  zc* Vw = (zc*)malloc(sizeof(zc) * n * n);
  int64_t m = (n % 2 == 0) ? n : n + 1;
  rot_t* rots = (rot_t*)malloc(sizeof(rot_t) * (m / 2 + 1));
  int64_t* pp = (int64_t*)malloc(sizeof(int64_t) * (m / 2 + 1));
  int64_t* qq = (int64_t*)malloc(sizeof(int64_t) * (m / 2 + 1));
  unsigned char* act = (unsigned char*)malloc(m / 2 + 1);
  if (!W || !Vw || !rots || !pp || !qq || !act) {
    free(W), free(Vw), free(rots), free(pp), free(qq), free(act);
    return ORACLE_ERR_NOMEM;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      AT(W, i, j, n) = (i > j) ? AT(M, i, j, ldm) : (i == j ? creal(AT(M, i, i, ldm)) : conj(AT(M, j, i, ldm)));
      AT(Vw, i, j, n) = (i == j) ? 1.0 : 0.0;
    }
  const double tol = (double)n * (DBL_EPSILON / 2.0);
  int sweep, converged = 0;
  for (sweep = 1; sweep <= ORACLE_MAX_SWEEPS && n > 1; ++sweep) {
    int64_t rotated = 0;
    for (int64_t r = 0; r < m - 1; ++r) {
      int64_t nact = 0;
      for (int64_t k = 0; k < m / 2; ++k) {
        int64_t p = rr_player(m, r, k), q = rr_player(m, r, m - 1 - k);
        act[k] = 0;
        if (p >= n || q >= n) continue;
        if (p > q) {
          int64_t tmp = p;
          p = q;
          q = tmp;
        }
        pp[k] = p;
        qq[k] = q;
        double a = creal(AT(W, p, p, n)), b = creal(AT(W, q, q, n));
        zc g = AT(W, p, q, n);
        if (cabs(g) > tol * sqrt(a * b)) {
          rots[k] = make_rot(a, b, g);
          act[k] = 1;
          ++nact;
        }
      }
      if (nact == 0) continue;
      rotated += nact;
      /* M <- M J  and  V <- V J  (columns) */
#pragma omp parallel for schedule(dynamic, 4)
      for (int64_t k = 0; k < m / 2; ++k) {
        if (!act[k]) continue;
        rot_cols(n, &AT(W, 0, pp[k], n), &AT(W, 0, qq[k], n), rots[k]);
        rot_cols(n, &AT(Vw, 0, pp[k], n), &AT(Vw, 0, qq[k], n), rots[k]);
      }
      /* M <- J^H M  (rows): row_p' = c row_p - s e^{+i phi} row_q,
                             row_q' = s row_p + c e^{+i phi} row_q           */
#pragma omp parallel for schedule(dynamic, 4)
      for (int64_t k = 0; k < m / 2; ++k) {
        if (!act[k]) continue;
        rot_t rt = rots[k];
        int64_t p = pp[k], q = qq[k];
        zc e = conj(rt.eph);
        for (int64_t j = 0; j < n; ++j) {
          zc xp = AT(W, p, j, n), xq = AT(W, q, j, n);
          AT(W, p, j, n) = rt.c * xp - rt.s * e * xq;
          AT(W, q, j, n) = rt.s * xp + rt.c * e * xq;
        }
      }
      /* the rotation annihilates (p, q) by construction: store the exact 0 */
      for (int64_t k = 0; k < m / 2; ++k) {
        if (!act[k]) continue;
        AT(W, pp[k], qq[k], n) = 0.0;
        AT(W, qq[k], pp[k], n) = 0.0;
      }
    }
    /* re-symmetrise the diagonal (imaginary parts are rounding noise) */
    for (int64_t j = 0; j < n; ++j) AT(W, j, j, n) = creal(AT(W, j, j, n));
    if (rotated == 0) {
      converged = 1;
      break;
    }
  }
  if (n <= 1) converged = 1, sweep = 0;
  for (int64_t j = 0; j < n; ++j) {
    lam[j] = creal(AT(W, j, j, n));
    for (int64_t i = 0; i < n; ++i) AT(V, i, j, ldv) = AT(Vw, i, j, n);
  }
  if (sweeps_out) *sweeps_out = sweep;
  free(W), free(Vw), free(rots), free(pp), free(qq), free(act);
  return converged ? ORACLE_OK : ORACLE_ERR_NO_CONVERGENCE;
}

/* Ascending order of omega; ties keep the lower index first (stable). */
static double* g_sort_key;
static int cmp_idx(const void* a, const void* b) {
  int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  if (g_sort_key[i] < g_sort_key[j]) return -1;
  if (g_sort_key[i] > g_sort_key[j]) return 1;
  return (i < j) ? -1 : (i > j);
}
static void argsort_ascending(int64_t n, double* key, int64_t* idx) {
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  g_sort_key = key;
  qsort(idx, (size_t)n, sizeof(int64_t), cmp_idx);
}

/* Final setup shared by Alg. 2 and Alg. 3 (their last step):
 * X = (V1 + V2)/2, Y = (V2 - V1)/2, columns written in ascending omega.   */
static void final_setup(int64_t n, const double* om, const zc* V1, const zc* V2, double* omega,
                        zc* X, int64_t ldx, zc* Y, int64_t ldy) {
  int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  double* key = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j) key[j] = om[j];
  argsort_ascending(n, key, idx);
  for (int64_t jj = 0; jj < n; ++jj) {
    int64_t j = idx[jj];
    omega[jj] = om[j];
    if (X && Y)
      for (int64_t i = 0; i < n; ++i) {
        zc v1 = AT(V1, i, j, n), v2 = AT(V2, i, j, n);
        AT(X, i, jj, ldx) = 0.5 * (v1 + v2);
        AT(Y, i, jj, ldy) = 0.5 * (v2 - v1);
      }
  }
  free(idx);
  free(key);
}

/* M1 = A + B (lower triangle) when sgn = +1, M2 = A - B when sgn = -1.    */
static void form_m(int64_t n, const zc* A, int64_t lda, const zc* B, int64_t ldb, double sgn,
                   zc* M) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i)
      AT(M, i, j, n) = (i >= j) ? AT(A, i, j, lda) + sgn * AT(B, i, j, ldb) : 0.0;
}

/* ------------------------------------------------------------------------
 * Alg. 2 (CHOL): L L^H = A - B; M = L^H (A + B) L; M V_M = V_M D;
 * Lambda = D^{1/2}; V1 = L^{-H} V_M Lambda^{1/2}; V2 = L V_M Lambda^{-1/2};
 * X = (V1 + V2)/2, Y = (V2 - V1)/2.  Outputs ascending omega; X, Y may be
 * NULL for eigenvalues only.  info: failing column for NOT_PD, else sweeps.
 */
int oracle_solve_chol(int64_t n, const zc* A, int64_t lda, const zc* B, int64_t ldb, double* omega,
                      zc* X, int64_t ldx, zc* Y, int64_t ldy, int64_t* info) {
  if (n < 0) return ORACLE_ERR_ARG;
  if (n == 0) return ORACLE_OK;
  size_t nn = (size_t)n * (size_t)n;
  zc *M1 = malloc(sizeof(zc) * nn), *M2 = malloc(sizeof(zc) * nn), *L = malloc(sizeof(zc) * nn);
  zc *M = malloc(sizeof(zc) * nn), *VM = malloc(sizeof(zc) * nn);
  zc *V1 = malloc(sizeof(zc) * nn), *V2 = malloc(sizeof(zc) * nn);
  double *d = malloc(sizeof(double) * n), *om = malloc(sizeof(double) * n);
  int rc = ORACLE_OK;
  if (!M1 || !M2 || !L || !M || !VM || !V1 || !V2 || !d || !om) {
    rc = ORACLE_ERR_NOMEM;
    goto done;
  }
  form_m(n, A, lda, B, ldb, +1.0, M1);
  form_m(n, A, lda, B, ldb, -1.0, M2);
  int64_t col = oracle_cholesky(n, M2, n, L, n); /* step 1 */
  if (col) {
    if (info) *info = col;
    rc = ORACLE_ERR_NOT_PD_AMINUSB;
    goto done;
  }
  rc = oracle_congruence(n, M1, n, L, n, M, n); /* step 2: M = L^H (A+B) L */
  if (rc) goto done;
  int sweeps = 0;
  rc = oracle_jacobi_eigh(n, M, n, d, VM, n, &sweeps); /* M V_M = V_M D */
  if (info) *info = sweeps;
  if (rc) goto done;
  for (int64_t j = 0; j < n; ++j) {
    if (!(d[j] > 0.0)) { /* M is PD in exact arithmetic; guard rounding */
      rc = ORACLE_ERR_NOT_PD_APLUSB;
      if (info) *info = j + 1;
      goto done;
    }
    om[j] = sqrt(d[j]); /* step 3: Lambda = D^{1/2} */
  }
  /* step 4: V1 = L^{-H} V_M Lambda^{1/2}: back substitution with the upper
     triangular L^H, column by column: (L^H)(i,k) = conj(L(k,i)).          */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double sc = sqrt(om[j]);
    for (int64_t i = n - 1; i >= 0; --i) {
      zc s = AT(VM, i, j, n);
      for (int64_t k = i + 1; k < n; ++k) s -= conj(AT(L, k, i, n)) * AT(V1, k, j, n);
      AT(V1, i, j, n) = s / creal(AT(L, i, i, n));
    }
    for (int64_t i = 0; i < n; ++i) AT(V1, i, j, n) *= sc;
  }
  /* step 5: V2 = L V_M Lambda^{-1/2} */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double sc = 1.0 / sqrt(om[j]);
    for (int64_t i = 0; i < n; ++i) {
      zc s = 0.0;
      for (int64_t k = 0; k <= i; ++k) s += AT(L, i, k, n) * AT(VM, k, j, n);
      AT(V2, i, j, n) = s * sc;
    }
  }
  final_setup(n, om, V1, V2, omega, X, ldx, Y, ldy); /* step 6 */
done:
  free(M1), free(M2), free(L), free(M), free(VM), free(V1), free(V2), free(d), free(om);
  return rc;
}

/* ------------------------------------------------------------------------
 * Alg. 3 (CHOL+SVD): L1 L1^H = A + B; L2 L2^H = A - B;
 * U Lambda V^H = L1^H L2 (one-sided Jacobi); V1 = L1 U Lambda^{-1/2};
 * V2 = L2 V Lambda^{-1/2}; X = (V1 + V2)/2, Y = (V2 - V1)/2.  omega is read
 * directly off the singular values.
 */
int oracle_solve_svd(int64_t n, const zc* A, int64_t lda, const zc* B, int64_t ldb, double* omega,
                     zc* X, int64_t ldx, zc* Y, int64_t ldy, int64_t* info) {
  if (n < 0) return ORACLE_ERR_ARG;
  if (n == 0) return ORACLE_OK;
  size_t nn = (size_t)n * (size_t)n;
  zc *M1 = malloc(sizeof(zc) * nn), *M2 = malloc(sizeof(zc) * nn);
  zc *L1 = malloc(sizeof(zc) * nn), *L2 = malloc(sizeof(zc) * nn), *G = malloc(sizeof(zc) * nn);
  zc *U = malloc(sizeof(zc) * nn), *V = malloc(sizeof(zc) * nn);
  zc *V1 = malloc(sizeof(zc) * nn), *V2 = malloc(sizeof(zc) * nn);
  double* sg = malloc(sizeof(double) * n);
  int rc = ORACLE_OK;
  if (!M1 || !M2 || !L1 || !L2 || !G || !U || !V || !V1 || !V2 || !sg) {
    rc = ORACLE_ERR_NOMEM;
    goto done;
  }
  form_m(n, A, lda, B, ldb, +1.0, M1);
  form_m(n, A, lda, B, ldb, -1.0, M2);
  int64_t col = oracle_cholesky(n, M1, n, L1, n); /* step 1 */
  if (col) {
    if (info) *info = col;
    rc = ORACLE_ERR_NOT_PD_APLUSB;
    goto done;
  }
  col = oracle_cholesky(n, M2, n, L2, n); /* step 2 */
  if (col) {
    if (info) *info = col;
    rc = ORACLE_ERR_NOT_PD_AMINUSB;
    goto done;
  }
  oracle_product(n, L1, n, L2, n, G, n); /* step 3: G = L1^H L2 */
  int sweeps = 0;
  rc = oracle_jacobi_svd(n, G, n, sg, U, n, V, n, &sweeps);
  if (info) *info = sweeps;
  if (rc) goto done;
  /* steps 4-5: V1 = L1 U Lambda^{-1/2}, V2 = L2 V Lambda^{-1/2} */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double sc = 1.0 / sqrt(sg[j]);
    for (int64_t i = 0; i < n; ++i) {
      zc s1 = 0.0, s2 = 0.0;
      for (int64_t k = 0; k <= i; ++k) {
        s1 += AT(L1, i, k, n) * AT(U, k, j, n);
        s2 += AT(L2, i, k, n) * AT(V, k, j, n);
      }
      AT(V1, i, j, n) = s1 * sc;
      AT(V2, i, j, n) = s2 * sc;
    }
  }
  final_setup(n, sg, V1, V2, omega, X, ldx, Y, ldy); /* step 6 */
done:
  free(M1), free(M2), free(L1), free(L2), free(G), free(U), free(V), free(V1), free(V2), free(sg);
  return rc;
}

/* ------------------------------------------------------------------------
 * Gradient of L = sum_i w_i omega_i with respect to Hermitian A and B.
 * Thm. 3 item 3: the left eigenvector of H for omega_i is v_i^H Sigma, and
 * with v_i^H Sigma v_i = 1 (Eq. (13)) first-order perturbation gives
 * d omega_i = v_i^H Sigma dH v_i = v_i^H [dA dB; dB dA] v_i
 *           = <x x^H + y y^H, dA> + <x y^H + y x^H, dB>   (Frobenius, real).
 * dA = sum_i w_i (x_i x_i^H + y_i y_i^H), dB = sum_i w_i (x_i y_i^H + y_i x_i^H),
 * full n x n Hermitian outputs.  X, Y hold the k selected columns.
 */
void oracle_grad(int64_t n, int64_t k, const zc* X, int64_t ldx, const zc* Y, int64_t ldy,
                 const double* w, zc* dA, int64_t ldda, zc* dB, int64_t lddb) {
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < n; ++b) {
    for (int64_t a = 0; a < n; ++a) {
      zc ga = 0.0, gb = 0.0;
      for (int64_t i = 0; i < k; ++i) {
        zc xa = AT(X, a, i, ldx), xb = AT(X, b, i, ldx);
        zc ya = AT(Y, a, i, ldy), yb = AT(Y, b, i, ldy);
        ga += w[i] * (xa * conj(xb) + ya * conj(yb));
        gb += w[i] * (xa * conj(yb) + ya * conj(xb));
      }
      AT(dA, a, b, ldda) = ga;
      AT(dB, a, b, lddb) = gb;
    }
  }
}
