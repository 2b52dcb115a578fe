// Internal host-side launchers of the solver stages (not part of the C ABI).
#pragma once
#include "gemm.cuh"

// ---- potrf.cu ----
int chol_block_size();
size_t chol_linv_elems(int64_t n);
bse_status potrf_lower(cudaStream_t s, int64_t n, cplx* A, int64_t lda, cplx* Linv, int64_t* status,
                       int64_t err_code);
bse_status trsm_lower_conjtrans(cudaStream_t s, int64_t n, int64_t k, const cplx* L, int64_t ldl,
                                const cplx* Linv, cplx* R, int64_t ldr, const int64_t* status);

// ---- elementwise.cu ----
// M1 = A + B written as a full Hermitian matrix (ld ldm) when full != 0,
// else only the lower triangle; sgn = +1 for A + B, -1 for A - B.
bse_status form_sum(cudaStream_t s, int64_t n, const cplx* A, int64_t lda, const cplx* B, int64_t ldb,
                    double sgn, cplx* M, int64_t ldm, int full);
// Mirror the lower triangle into the upper one (conjugate), real diagonal.
bse_status hermitian_fill_upper(cudaStream_t s, int64_t n, cplx* M, int64_t ldm);
// Z (real, n x k, ld ldz) -> V (complex, ld ldv)
bse_status real_to_complex(cudaStream_t s, int64_t n, int64_t k, const double* Z, int64_t ldz, cplx* V,
                           int64_t ldv);
// E(i,i) -= 1 for i < k
bse_status sub_identity(cudaStream_t s, int64_t k, double* E, int64_t lde);
// omega and the scale vectors of the final setup from the eigenvalues of
// the reduced problem.  mode 0 (CHOL): lam are eigenvalues of M, omega =
// sqrt(lam), c1 = sqrt(omega), c2 = 1/sqrt(omega).  mode 1 (SVD): lam are
// singular values, omega = lam, c1 = c2 = 1/sqrt(omega).
bse_status finish_omega(cudaStream_t s, int64_t k, const double* lam, int mode, double* omega_out,
                        double* c1, double* c2, const int64_t* status);
// Mixed form: Rayleigh-quotient refinement of omega against the original
// A, B (through full Hermitian M1 = A + B, M2 = A - B) and relative residuals.
// work: 4 n k complex.  est: k doubles, est_max: 1 double (device).
// replace = 0 keeps omega and only computes the residuals.
bse_status refine_omega(cudaStream_t s, int64_t n, int64_t k, const cplx* M1, const cplx* M2, const cplx* X,
                        int64_t ldx, const cplx* Y, int64_t ldy, cplx* work, double* omega, double* est,
                        double* est_max, const int64_t* status, int replace);
// zero a complex matrix block
bse_status zero_c(cudaStream_t s, int64_t m, int64_t n, cplx* A, int64_t lda);
bse_status sqrt_factors(cudaStream_t s, int64_t n, const double* d, double* qp, double* qm, int64_t* status);
bse_status scale_columns(cudaStream_t s, int64_t n, int64_t k, const cplx* Q, int64_t ldq, const double* q, cplx* W,
                         int64_t ldw);
// gradient (Thm. 3 item 3): dA = X W X^H + Y W Y^H, dB = X W Y^H + Y W X^H
bse_status grad_outer(cudaStream_t s, int64_t n, int64_t k, const cplx* X, int64_t ldx, const cplx* Y,
                      int64_t ldy, const double* w, cplx* dA, int64_t ldda, cplx* dB, int64_t lddb);

// ---- hetrd.cu ----  Householder reduction of a Hermitian matrix to real
// symmetric tridiagonal form (lower storage) and its back-transformation.
struct HetrdWork {
  cplx* V;        // n x n, column j = reflector j (explicit 1, zeros above)
  cplx* W;        // n x nbt, current panel's W
  cplx* tau;      // n
  double* d;      // n  (diagonal of T)
  double* e;      // n  (e[j] = T(j+1, j), j < n-1)
  cplx* part;     // partial-sum scratch, hetrd_part_elems(n)
  cplx* small;    // small scratch (>= 4 * nbt * nbt + 64)
  cplx* S2;       // n x 2 nbt: one operand of the merged trailing update
};
int hetrd_panel();
// reflectors per block in the back-transformations (T factor of this width)
int backtransform_block();
size_t backtransform_tmp_elems(int64_t k);  // workspace of apply_block_reflector
size_t hetrd_part_elems(int64_t n);
bse_status hetrd_lower(cudaStream_t s, int64_t n, cplx* A, int64_t lda, const HetrdWork& w,
                       const int64_t* status);
// Vout = Q Vout where Q = H_0 ... H_{n-2} from hetrd_lower; Vout is n x k.
bse_status hetrd_backtransform(cudaStream_t s, int64_t n, int64_t k, const HetrdWork& w, cplx* Vout,
                               int64_t ldv, cplx* tmp, const int64_t* status);

// ---- tridiag.cu ----  eigenpairs of a real symmetric tridiagonal matrix.
struct TriWork {
  double* a;       // N diagonal (copied, may be split-modified)
  double* off;     // N off-diagonal (off[k] = T(k+1, k))
  double* e2;      // N squares of off
  double* lam;     // N eigenvalues in block order
  int* blk;        // N block of each slot
  int* rank;       // N global ascending rank of each slot
  int* bstart;     // N + 1 block starts
  double* prm;     // 8 doubles: pivmin, tnorm, ...
  int* iprm;       // 8 ints: number of blocks, ...
  double* scratch; // N * kmax doubles (twisted factorisation)
  double* E;       // kmax * kmax (orthogonalisation Gram matrix)
  float* Ef;       // kmax * kmax
  double* Z2;      // N * kmax doubles (also holds two N * kmax float arrays)
  int* grid;       // tri_grid_points() Sturm counts
};
int tri_grid_points();
// mode 0: all N eigenvalues of T.  mode 1 (Golub-Kahan form, zero diagonal,
// even N): the N/2 positive eigenvalues (the upper half of each block).
// Selected ascending indices [il, iu] (0-based, inclusive) of the computed set.
// Writes lam_out[0..k) ascending and Z (N x k, ld ldz) orthonormal columns.
bse_status tridiag_eig(cudaStream_t s, int64_t N, const double* a, const double* off, int mode,
                       int64_t il, int64_t iu, double* lam_out, double* Z, int64_t ldz,
                       const TriWork& w, int64_t* status);
bse_status orthonormalize_columns(cudaStream_t s, int64_t N, int64_t k, double* Z, int64_t ldz,
                                  const TriWork& w, const int64_t* status);

// ---- gebrd.cu ----  Householder bidiagonalisation G = Q_L B Q_R^H (B real upper bidiagonal).
struct GebrdWork {
  cplx* U;        // n x n left reflectors (explicit)
  cplx* Vr;       // n x n right reflectors (explicit)
  cplx* X;        // n x nbt
  cplx* Y;        // n x nbt
  cplx* tauq;     // n
  cplx* taup;     // n
  double* d;      // n
  double* e;      // n
  cplx* part;     // partial-sum scratch
  cplx* small;    // small scratch
  cplx* S2;       // n x 2 nbt: one operand of the merged trailing update
};
size_t gebrd_part_elems(int64_t n);
bse_status gebrd_upper(cudaStream_t s, int64_t n, cplx* A, int64_t lda, const GebrdWork& w,
                       const int64_t* status);
// side 0: Vout = Q_L Vout;  side 1: Vout = Q_R Vout
bse_status gebrd_backtransform(cudaStream_t s, int side, int64_t n, int64_t k, const GebrdWork& w,
                               cplx* Vout, int64_t ldv, cplx* tmp, const int64_t* status);

// generic: Vout[r0:, :] = (I - Vp Tp Vp^H) Vout[r0:, :] for a panel of
// explicit reflectors (columns c0..c0+bs of Vbuf, nonzero from row r0 on)
bse_status apply_block_reflector(cudaStream_t s, int64_t n, int64_t k, const cplx* Vbuf, int64_t ldvb,
                                 int64_t c0, int64_t bs, int64_t r0, const cplx* tau, cplx* Vout,
                                 int64_t ldv, cplx* tmp, const int64_t* status);

// ---- batched.cu ----  persistent one-CTA-per-instance Cholesky-method solver
size_t batched_inst_bytes(int64_t n, int64_t k);
int batched_max_n();
size_t batched_desc_bytes();
void batched_fill_desc(void* slot, int64_t n, int64_t k, const void* A, const void* B, double* omega, void* X,
                       void* Y, char* ws, int64_t* status);
size_t batched_svd_inst_bytes(int64_t n, int64_t k);
cudaError_t single_chol_prepare();
cudaError_t single_chol_launch(cudaStream_t s, int64_t n, int64_t k, const void* A, const void* B, double* omega,
                               void* X, void* Y, char* ws, int64_t* status);
// counter: two ints (queue counters); nbig: the first nbig instances of the
// size-ordered table are solved by teams of `team` CTAs (team 1 or nbig 0:
// every instance on one CTA)
bse_status batched_chol_launch(cudaStream_t s, const void* desc, int64_t count, int* counter, int grid,
                               int method, int64_t nbig, int team);
int batched_team_default();
int batched_team_min_n_default();

// ---- launch shapes chosen per handle (autotuned), current for one solve ----
struct LaunchTuning {
  int hemv_items;  // tridiagonalisation matvec: at most this many row tiles per work item (1..16; 0: 8)
  int splitk_max;  // back-transformations: at most this many split-K layers of V^H Z (1..8; 0: 8)
};
void tuning_set_current(const LaunchTuning& t);
LaunchTuning tuning_current();

// ---- ozgemm.cu ----  FP64-accurate complex GEMM on the BF16 tensor cores
enum { OZ_ENGINE_TCGEN05 = 0, OZ_ENGINE_MMA_SYNC = 1 };
struct OzWork {
  void* ptr;      // slice / scale workspace (NULL: tensor-core products off)
  size_t bytes;
  int64_t min_mnk;  // products with m*n*k below this stay on the DFMA engine
  int engine;       // OZ_ENGINE_TCGEN05 (TMEM accumulators, TMA) or OZ_ENGINE_MMA_SYNC
  int64_t wait_cycles;  // tcgen05 engine: limit of its pipeline waits in clock cycles (0: default, ~1 s)
};
void oz_set_current(const OzWork& w);
OzWork oz_current();
size_t oz_work_bytes(int64_t maxdim, int slices);
// fp64_flops: the product's useful FP64-equivalent flops (for the profiler)
bse_status gemm_z_oz_raw(cudaStream_t s, const GemmParams<cplx>& p, double fp64_flops);
bse_status gemm_d_oz_raw(cudaStream_t s, const GemmParams<double>& p, double fp64_flops);
