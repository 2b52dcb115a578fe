// Eigenpairs of a real symmetric tridiagonal matrix T (diagonal a, off-
// diagonal off), the "D" and "V_M" of Alg. 2 after the Householder
// reduction, and -- in Golub-Kahan form (zero diagonal, off = d1, e1, d2, e2,
// ..., size 2n) -- the singular triplets of the bidiagonal of Alg. 3.
//
//  * splitting: off(k) with |off(k)| <= eps * ||T|| is set to 0 and T is
//    treated block by block (Golub-Kahan form: only at the e positions, so
//    every block keeps even size and its +-sigma pairing);
//  * eigenvalues: Sturm-count bisection, one thread per eigenvalue, to
//    relative width 2 eps (for the Golub-Kahan form this is bisection on the
//    singular values, which keeps their high relative accuracy);
//  * eigenvectors: one thread per eigenvalue solves with the twisted
//    factorisation T - lambda I = N_r D_r N_r^T (top-down and bottom-up
//    pivots, twist index r = argmin |gamma_r|): z_r = 1 and the two
//    recurrences outward -- one step of inverse iteration from the best unit
//    vector;
//  * orthogonalisation: one Newton-Schulz step Z <- Z (3I - Z^T Z)/2 (the
//    Gram matrix in FP64, the small correction product in FP32) brings the
//    O(eps ||T|| / gap) loss of orthogonality of close eigenvalues down to
//    O(eps) without changing the residuals beyond O(eps ||T||).
#include <float.h>

#include "kernels.cuh"
#include "prof.cuh"

// prm: 0 pivmin, 1 tnorm, 2 twist guard, 3 lower bound, 4 upper bound
// iprm: 0 number of blocks
__global__ void tri_prep_kernel(int64_t N, const double* __restrict__ a_in, const double* __restrict__ off_in, int mode,
                                double* __restrict__ a, double* __restrict__ off, double* __restrict__ e2,
                                int* __restrict__ bstart, double* __restrict__ prm, int* __restrict__ iprm) {
  __shared__ double red_t[32], red_e[32], red_lo[32], red_hi[32];
  __shared__ double tnorm_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  double tn = 0.0, em = 0.0, lo = 1e308, hi = -1e308;
  for (int64_t k = tid; k < N; k += nt) {
    const double ak = a_in ? a_in[k] : 0.0;
    const double ol = (k > 0) ? fabs(off_in[k - 1]) : 0.0;
    const double orr = (k < N - 1) ? fabs(off_in[k]) : 0.0;
    tn = fmax(tn, fabs(ak) + ol + orr);
    lo = fmin(lo, ak - ol - orr);
    hi = fmax(hi, ak + ol + orr);
    if (k < N - 1) em = fmax(em, off_in[k] * off_in[k]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((tid & 31) == 0) red_t[tid >> 5] = tn, red_e[tid >> 5] = em, red_lo[tid >> 5] = lo, red_hi[tid >> 5] = hi;
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < nt / 32; ++w)
      tn = fmax(tn, red_t[w]), em = fmax(em, red_e[w]), lo = fmin(lo, red_lo[w]), hi = fmax(hi, red_hi[w]);
    const double pivmin = DBL_MIN * fmax(1.0, em);
    prm[0] = pivmin;
    prm[1] = tn;
    prm[2] = DBL_EPSILON * fmax(tn, DBL_MIN);
    const double pad = 2.0 * DBL_EPSILON * tn + 4.0 * pivmin;
    prm[3] = lo - pad;
    prm[4] = hi + pad;
    tnorm_s = tn;
  }
  __syncthreads();
  const double tol = DBL_EPSILON * tnorm_s;
  for (int64_t k = tid; k < N; k += nt) {
    a[k] = a_in ? a_in[k] : 0.0;
    if (k < N - 1) {
      double o = off_in[k];
      const bool may_split = (mode == 0) || (k & 1);
      if (may_split && fabs(o) <= tol) o = 0.0;
      off[k] = o;
      e2[k] = o * o;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int nb = 0;
    bstart[0] = 0;
    for (int64_t k = 0; k < N - 1; ++k)
      if (off[k] == 0.0) bstart[++nb] = (int)(k + 1);
    bstart[++nb] = (int)N;
    iprm[0] = nb;
  }
}

__device__ __forceinline__ int sturm_count(const double* __restrict__ a, const double* __restrict__ e2, int b0, int b1,
                                           double x, double pivmin) {
  double q = a[b0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = q < 0.0;
  for (int k = b0 + 1; k < b1; ++k) {
    q = (a[k] - x) - e2[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

// slot s -> (block, local target index): mode 0 slots follow bstart,
// mode 1 slots follow bstart / 2 and take the upper half of each block.
__device__ __forceinline__ int find_block(const int* bstart, int nb, int64_t s, int mode) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t st = mode == 0 ? bstart[mid] : bstart[mid] / 2;
    if (st <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Sturm counts of an unreduced T at TRI_GRID - 1 equally spaced interior
// points of the spectrum's enclosing interval: every eigenvalue's bisection
// then starts from the grid cell that contains it (log2(TRI_GRID) halvings
// saved), with the same invariant count(lo) <= t < count(hi).
constexpr int TRI_GRID = 8192;

__global__ void tri_grid_kernel(int64_t N, const double* __restrict__ a, const double* __restrict__ e2,
                                const int* __restrict__ iprm, const double* __restrict__ prm, int* __restrict__ cnt,
                                const int64_t* status) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= TRI_GRID - 1) return;
  if (*(volatile const int64_t*)status) return;
  if (iprm[0] != 1) return;  // split matrices bisect from the full interval
  const double lo = prm[3], hi = prm[4];
  const double x = lo + (hi - lo) * ((double)(g + 1) / (double)TRI_GRID);
  cnt[g] = sturm_count(a, e2, 0, (int)N, x, prm[0]);
}

// Multisection: TRI_MS consecutive lanes of a warp share one eigenvalue and
// evaluate Sturm counts at TRI_MS interior points of its interval in each
// round, which shrinks it by TRI_MS + 1 (log2(5) bits per round instead of
// one).  The FP64 pipe is the bound of a Sturm step (a division per entry);
// one lane per eigenvalue leaves it mostly idle, four keep it busy.
constexpr int TRI_MS = 4;
__global__ void tri_bisect_kernel(int64_t total, const double* __restrict__ a, const double* __restrict__ e2,
                                  const int* __restrict__ bstart, const int* __restrict__ iprm,
                                  const double* __restrict__ prm, int mode, double* __restrict__ lam,
                                  int* __restrict__ blk, const int* __restrict__ cnt, const int64_t* status) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t s = gt / TRI_MS;
  const int sub = (int)(gt % TRI_MS);
  if (s >= total) return;  // the whole group of TRI_MS lanes
  if (*(volatile const int64_t*)status) return;
  const unsigned gmask = ((1u << TRI_MS) - 1u) << ((threadIdx.x & 31) & ~(TRI_MS - 1));
  const int nb = iprm[0];
  const int b = find_block(bstart, nb, s, mode);
  const int b0 = bstart[b], b1 = bstart[b + 1];
  const int m = b1 - b0;
  const int t = mode == 0 ? (int)(s - b0) : m / 2 + (int)(s - b0 / 2);
  const double pivmin = prm[0];
  double lo = prm[3], hi = prm[4];
  if (nb == 1) {
    // first grid point with count > t: eigenvalue t lies in (x_{g}, x_{g+1}]
    int l = 0, h = TRI_GRID - 1;  // search over cnt[0 .. TRI_GRID-2]; h = "none"
    while (l < h) {
      const int mid = (l + h) >> 1;
      if (cnt[mid] > t) h = mid; else l = mid + 1;
    }
    const double w = (hi - lo) / (double)TRI_GRID;
    const double glo = l > 0 ? lo + w * (double)l : lo;
    const double ghi = l < TRI_GRID - 1 ? lo + w * (double)(l + 1) : hi;
    lo = glo;
    hi = ghi;
  }
  for (int it = 0; it < 128; ++it) {
    const double w = hi - lo;
    const double x0 = lo + w * (1.0 / (TRI_MS + 1)), xl = lo + w * ((double)TRI_MS / (TRI_MS + 1));
    if (w <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) || w <= 4.0 * pivmin || x0 <= lo || xl >= hi) break;
    const double x = lo + w * ((double)(sub + 1) / (TRI_MS + 1));
    const unsigned above = __ballot_sync(gmask, sturm_count(a, e2, b0, b1, x, pivmin) > t) >>
                           ((threadIdx.x & 31) & ~(TRI_MS - 1));
    // the eigenvalue lies between the last point with count <= t and the
    // first with count > t (the counts grow with x)
    const int f = above ? __ffs(above) - 1 : TRI_MS;
    const double nlo = f > 0 ? lo + w * ((double)f / (TRI_MS + 1)) : lo;
    const double nhi = f < TRI_MS ? lo + w * ((double)(f + 1) / (TRI_MS + 1)) : hi;
    lo = nlo;
    hi = nhi;
  }
  if (sub == 0) {
    lam[s] = 0.5 * (lo + hi);
    blk[s] = b;
  }
}

__global__ void tri_rank_kernel(int64_t total, const double* __restrict__ lam, const int* __restrict__ iprm,
                                int* __restrict__ rank) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= total) return;
  if (iprm[0] == 1) {
    rank[s] = (int)s;
    return;
  }
  const double v = lam[s];
  int r = 0;
  for (int64_t t = 0; t < total; ++t) {
    const double u = lam[t];
    r += (u < v) || (u == v && t < s);
  }
  rank[s] = r;
}

// eigenvalues in ascending order for the selected range, and the vectors
__global__ void tri_vec_kernel(int64_t total, int64_t il, int64_t iu, const double* __restrict__ a,
                               const double* __restrict__ off, const double* __restrict__ e2,
                               const int* __restrict__ bstart, const double* __restrict__ prm,
                               const double* __restrict__ lam, const int* __restrict__ blk,
                               const int* __restrict__ rank, double* __restrict__ lam_out, double* __restrict__ Z,
                               int64_t ldz, double* __restrict__ scratch, int64_t ldsc, const int64_t* status) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= total) return;
  if (*(volatile const int64_t*)status) return;
  const int64_t rk = rank[s];
  if (rk < il || rk > iu) return;
  const int64_t col = rk - il;
  const double l = lam[s];
  lam_out[col] = l;
  if (!Z) return;
  const int b = blk[s];
  const int b0 = bstart[b], b1 = bstart[b + 1];
  const int m = b1 - b0;
  const double g = prm[2];
  double* zc = Z + col * ldz + b0;
  double* sc = scratch + col * ldsc + b0;
  // pass 1: top-down pivots dp(k) (stored in zc)
  double x = a[b0] - l;
  if (fabs(x) < g) x = (x < 0.0) ? -g : g;
  zc[0] = x;
  for (int k = 1; k < m; ++k) {
    x = (a[b0 + k] - l) - e2[b0 + k - 1] / x;
    if (fabs(x) < g) x = (x < 0.0) ? -g : g;
    zc[k] = x;
  }
  // pass 2: bottom-up pivots dm(k) (stored in sc) and the twist index
  double y = a[b1 - 1] - l;
  if (fabs(y) < g) y = (y < 0.0) ? -g : g;
  sc[m - 1] = y;
  double best = fabs(zc[m - 1]);
  int r = m - 1;
  for (int k = m - 2; k >= 0; --k) {
    const double ak = a[b0 + k] - l;
    y = ak - e2[b0 + k] / y;
    if (fabs(y) < g) y = (y < 0.0) ? -g : g;
    sc[k] = y;
    const double gam = zc[k] + y - ak;
    if (fabs(gam) < best) best = fabs(gam), r = k;
  }
  // pass 3: the vector
  double nrm2 = 1.0;
  double z = 1.0;
  for (int k = r - 1; k >= 0; --k) {
    z = -(off[b0 + k] / zc[k]) * z;
    zc[k] = z;
    nrm2 += z * z;
  }
  zc[r] = 1.0;
  z = 1.0;
  for (int k = r; k < m - 1; ++k) {
    z = -(off[b0 + k] / sc[k + 1]) * z;
    zc[k + 1] = z;
    nrm2 += z * z;
  }
  const double inv = 1.0 / sqrt(nrm2);
  for (int k = 0; k < m; ++k) zc[k] *= inv;
}

// E (k x k, lower half computed) -> full symmetric, minus I, as float
__global__ void ns_prep_kernel(int64_t k, const double* __restrict__ E, float* __restrict__ Ef) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= k || j >= k) return;
  const double v = (i >= j) ? E[i + j * k] : E[j + i * k];
  Ef[i + j * k] = (float)(v - (i == j ? 1.0 : 0.0));
}

__global__ void to_float_kernel(int64_t N, int64_t k, const double* __restrict__ Z, int64_t ldz, float* __restrict__ Zf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < N && j < k) Zf[i + j * N] = (float)Z[i + j * ldz];
}

__global__ void ns_update_kernel(int64_t N, int64_t k, double* __restrict__ Z, int64_t ldz, const float* __restrict__ D) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < N && j < k) Z[i + j * ldz] -= 0.5 * (double)D[i + j * N];
}

// One Newton-Schulz step Z <- Z - Z E / 2 with E = Z^T Z - I.  E needs FP64
// (its entries are O(eps ||T|| / gap) and come from cancellation), only its
// lower half is computed; the product Z E is O(|E|) and needs only ~7 digits,
// so it runs in FP32 (FFMA), its rounding error O(1e-7 |E|) being far below
// FP64 rounding of Z.
bse_status orthonormalize_columns(cudaStream_t s, int64_t N, int64_t k, double* Z, int64_t ldz, const TriWork& w,
                                  const int64_t* status) {
  if (k <= 0 || N <= 0) return BSE_OK;
  GemmParams<double> pe = gemm_params<double>(k, k, N, OPT, Z, ldz, OPN, Z, ldz, 1.0, 0.0, w.E, k);
  pe.lowerC = 1;
  pe.status = status;
  bse_status r = gemm_d(s, pe);
  if (r) return r;
  float* Zf = (float*)w.Z2;
  float* D = Zf + N * k;
  dim3 gk(ceil_div_u(k, 256), (unsigned)k), gn(ceil_div_u(N, 256), (unsigned)k);
  ns_prep_kernel<<<gk, 256, 0, s>>>(k, w.E, w.Ef);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  to_float_kernel<<<gn, 256, 0, s>>>(N, k, Z, ldz, Zf);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  GemmParams<float> pz = gemm_params<float>(N, k, k, OPN, Zf, N, OPN, w.Ef, k, 1.0f, 0.0f, D, N);
  pz.status = status;
  if ((r = gemm_f(s, pz))) return r;
  ns_update_kernel<<<gn, 256, 0, s>>>(N, k, Z, ldz, D);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

bse_status tridiag_eig(cudaStream_t s, int64_t N, const double* a, const double* off, int mode, int64_t il,
                       int64_t iu, double* lam_out, double* Z, int64_t ldz, const TriWork& w, int64_t* status) {
  if (N <= 0) return BSE_OK;
  const int64_t total = mode == 0 ? N : N / 2;
  const int64_t k = iu - il + 1;
  prof_launch_begin(s);
  tri_prep_kernel<<<1, 1024, 0, s>>>(N, a, off, mode, w.a, w.off, w.e2, w.bstart, w.prm, w.iprm);
  prof_launch_end(s, "tri_prep_kernel");
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  prof_launch_begin(s);
  tri_grid_kernel<<<ceil_div_u(TRI_GRID, 128), 128, 0, s>>>(N, w.a, w.e2, w.iprm, w.prm, w.grid, status);
  prof_launch_end(s, "tri_grid_kernel");
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  prof_launch_begin(s);
  tri_bisect_kernel<<<ceil_div_u(total * TRI_MS, 64), 64, 0, s>>>(total, w.a, w.e2, w.bstart, w.iprm, w.prm, mode, w.lam,
                                                         w.blk, w.grid, status);
  prof_launch_end(s, "tri_bisect_kernel");
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  tri_rank_kernel<<<ceil_div_u(total, 256), 256, 0, s>>>(total, w.lam, w.iprm, w.rank);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  if (Z) BSE_CUDA(cudaMemset2DAsync(Z, sizeof(double) * ldz, 0, sizeof(double) * N, k, s));
  prof_launch_begin(s);
  tri_vec_kernel<<<ceil_div_u(total, 64), 64, 0, s>>>(total, il, iu, w.a, w.off, w.e2, w.bstart, w.prm, w.lam,
                                                      w.blk, w.rank, lam_out, Z, ldz, w.scratch, N, status);
  prof_launch_end(s, "tri_vec_kernel");
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

int tri_grid_points() { return TRI_GRID; }
