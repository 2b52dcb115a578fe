/*
 * bse.h -- C ABI of the GB300 (sm_103a) solvers for the form-I Bethe-Salpeter
 * eigenproblem of Benner & Penke, "Efficient and Accurate Algorithms for
 * Solving the Bethe-Salpeter Eigenvalue Problem for Crystalline Systems"
 * (arXiv 2008.08825).
 *
 * Problem (Eq. (3), Section 1): H1 = [A B; -B -A] with A = A^H, B = B^H, and
 * A + B, A - B positive definite (Lemma Qtransform item 2).  Then H1 has real
 * eigenvalues +-omega_i, omega_i > 0 (Thm. 5, Lemma ComputeNegEvecs).  The
 * solvers return the n positive eigenvalues omega (ascending) and the
 * eigenvector block V = [X; Y] in C^{2n x n} with H1 V = V diag(omega) and
 * V^H Sigma V = X^H X - Y^H Y = I (Thm. ProdEig, Eq. (13); Section 4).  The
 * eigenvector of -omega_i is [Y_i; X_i] (Lemma ComputeNegEvecs) and is not
 * materialised.
 *
 * Conventions for every entry point below:
 *   - Complex matrices are complex128 stored as interleaved (re, im) doubles,
 *     column-major: element (i, j) of a matrix with leading dimension ld is at
 *     p[2*(i + j*ld)] (real) and p[2*(i + j*ld) + 1] (imaginary).  ld >= max(1, n).
 *   - Unless a name ends in _host (or is bse_ooc_run's host tiles), every data
 *     pointer is a DEVICE pointer, allocated and owned by the caller.  Inputs
 *     are never modified.
 *   - Only the lower triangle (diagonal included) of the Hermitian inputs A, B
 *     is read; the imaginary parts of their diagonals are ignored.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; the call then synchronises that stream, reads the
 *     device-side status word and returns it.  Outputs are written only when
 *     the status is BSE_OK.
 *   - A handle is not thread-safe: use one handle per host thread.
 *   - On any status other than BSE_OK, bse_last_error() gives a message.
 */
#ifndef BSE_GB300_H
#define BSE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BSE_OK = 0,
  BSE_ERR_ARG = 1,              /* invalid argument (size, leading dimension, NULL pointer) */
  BSE_ERR_NOT_PD_AMINUSB = 2,   /* A - B not positive definite; info = failing column (1-based) */
  BSE_ERR_NOT_PD_APLUSB = 3,    /* A + B not positive definite; info = failing column (1-based) */
  BSE_ERR_NO_CONVERGENCE = 4,   /* an iteration (bisection, refinement) hit its cap */
  BSE_ERR_REFINE = 5,           /* mixed-precision refinement did not converge */
  BSE_ERR_TIMEOUT = 6,          /* a bounded device-side wait expired */
  BSE_ERR_CUDA = 7,             /* a CUDA runtime call failed (see bse_last_error) */
  BSE_ERR_NOMEM = 8,            /* workspace allocation failed */
  BSE_ERR_NOT_IMPLEMENTED = 9,  /* option not supported by this build */
  BSE_ERR_TOO_LARGE = 10        /* bse_solve_chol_noalloc: n above BSE_NOALLOC_MAX_N */
} bse_status;

typedef enum { BSE_PREC_FP64 = 0, BSE_PREC_MIXED = 1 } bse_precision;
/* BSE_METHOD_TDA only names the workspace of bse_solve_tda in bse_workspace_size */
typedef enum { BSE_METHOD_CHOL = 0, BSE_METHOD_SVD = 1, BSE_METHOD_SQRT = 2, BSE_METHOD_TDA = 3 } bse_method;

typedef struct bse_info {
  int64_t info;          /* failing column (1-based) for NOT_PD, else 0 */
  double err_est;        /* mixed form with vectors: max_i ||Hcal1 v_i - omega_i Sigma v_i|| /
                            (omega_i ||v_i||) after refinement, else 0 */
  int32_t refine_iters;  /* mixed form with vectors: 1 (one Rayleigh-quotient sweep), else 0 */
  int32_t reserved;
} bse_info;

typedef struct bse_context* bse_handle;

/* Create / destroy a solver context bound to the current CUDA device.  The
 * context owns a device workspace that grows on demand (cudaMalloc) unless
 * the caller supplies one with bse_set_workspace. */
bse_status bse_create(bse_handle* h);
bse_status bse_destroy(bse_handle h);

/* Message describing the last failure on this host thread ("" if none). */
const char* bse_last_error(void);

/* Bytes of device workspace a solve of size n needs (method: bse_method;
 * prec: bse_precision), for all n eigenpairs. */
bse_status bse_workspace_size(int64_t n, int method, int prec, size_t* bytes);

/* Use caller-owned device memory [ptr, ptr + bytes) as workspace (256-byte
 * aligned).  The memory must stay valid while the handle uses it; pass
 * ptr = NULL to return to internally allocated workspace. */
bse_status bse_set_workspace(bse_handle h, void* ptr, size_t bytes);

/* Handle options. */
typedef enum {
  /* Mixed form: complex products with m*n*k below this value stay on the FP64
   * FMA engine, larger ones use the split-operand tensor-core engine
   * (default 1 << 24).  1 sends every product through the tensor cores. */
  BSE_OPT_TC_MIN_MNK = 1,
  /* Batched solves: CTAs per SM in the persistent kernel's grid, 1 or 2
   * (default 1).  One CTA per SM gives each instance the SM's whole FP64
   * pipe and registers (shorter critical path for the largest instances);
   * two hide more latency where registers allow two resident CTAs.  Chosen
   * per workload by the autotuner (autotune.py). */
  BSE_OPT_BATCH_CTAS_PER_SM = 2,
  /* Mixed form: the tensor-core engine of the split-operand products.
   * 0 (default): tcgen05.mma with TMEM accumulators, operands staged by TMA
   * bulk-tensor copies; 1: warp-level mma.sync (the earlier engine, kept for
   * comparison).  Both give the same FP32 level sums exactly (the combined
   * set of levels >= 7 up to its rounding). */
  BSE_OPT_TC_ENGINE = 3,
  /* Mixed form, tcgen05 engine: limit, in SM clock cycles, of each wait of
   * its pipeline (copy landed, stage free, accumulators ready).  0 (default)
   * means 2e9 cycles, about 1 s.  When a wait runs out the product stops
   * issuing, lets the copies and MMAs it started finish (those waits keep
   * the default limit, so nothing is left in flight), frees its TMEM and
   * records BSE_ERR_TIMEOUT; the solve then returns BSE_ERR_TIMEOUT and
   * writes no output.  A tiny value forces that path (a test uses it); the
   * handle stays usable. */
  BSE_OPT_TC_WAIT_CYCLES = 4,
  /* Batched solves: instances with n >= BSE_OPT_BATCH_TEAM_MIN_N (default
   * 448) are solved by a team of BSE_OPT_BATCH_TEAM CTAs (1, 2, 4 or 8;
   * default 4), one thread-block cluster on as many SMs, so the largest
   * instances do not set the batch's critical path; 1 puts every instance
   * on one CTA.  Neither changes a result bit (the team splits work, not
   * sums).  Chosen per workload by the autotuner (autotune.py). */
  BSE_OPT_BATCH_TEAM = 5,
  BSE_OPT_BATCH_TEAM_MIN_N = 6,
  /* Launch shapes (0 = the library default; autotune.py picks them per
   * device and size): the Householder tridiagonalisation's matrix-vector
   * kernel takes at most BSE_OPT_HEMV_ITEM_TILES row tiles per work item
   * (1..16, default 8); the back-transformations split the k range of their
   * thin V^H Z products into at most BSE_OPT_SPLITK_MAX layers (1..8,
   * default 8).  Both change only the order of FP64 sums. */
  BSE_OPT_HEMV_ITEM_TILES = 7,
  BSE_OPT_SPLITK_MAX = 8
} bse_option;
bse_status bse_set_option(bse_handle h, int option, int64_t value);

/*
 * Cholesky method, Alg. 2 (Section 3.2):
 *   L L^H = A - B;  M = L^H (A + B) L;  M V_M = V_M D;  Lambda = D^{1/2};
 *   V1 = L^{-H} V_M Lambda^{1/2};  V2 = L V_M Lambda^{-1/2};
 *   X = (V1 + V2)/2,  Y = (V2 - V1)/2.
 * n        problem size (H1 is 2n x 2n), n >= 0.
 * A, B     device, n x n Hermitian, lower triangle read, leading dims lda, ldb.
 * il, iu   1-based inclusive index range into the ascending omega; il = 1,
 *          iu = n returns all pairs.  k = iu - il + 1 columns are returned.
 * prec     BSE_PREC_FP64: all arithmetic on the FP64 pipe.
 *          BSE_PREC_MIXED: the large complex products (Cholesky updates,
 *          congruence, reduction updates, back-transformations, triangular
 *          solve and products) run on the BF16 tensor cores with exact
 *          operand splitting (8 slices of 7 bits per FP64 value, exact FP32
 *          partial sums per level, FP64 recombination: the Ozaki scheme), so
 *          they carry FP64-level normwise error; pivots, matrix-vector
 *          products of the reductions, the tridiagonal solve and all
 *          element-wise work stay FP64.  With vectors, the Cholesky and
 *          square-root methods then refine omega against the original A, B:
 *          omega_i becomes the Rayleigh quotient v_i^H Hcal1 v_i /
 *          v_i^H Sigma v_i of the pencil (Hcal1, Sigma) of Eq. (1) (second
 *          order in the vector error; it removes the omega^2 error of
 *          Eq. (SquaredErr)).  The SVD method keeps its singular values,
 *          which are relatively accurate where the quotient is accurate only
 *          normwise.  info->err_est reports the largest relative residual.
 * omega    device, k doubles, ascending.
 * X, Y     device, n x k complex, leading dims ldx, ldy; both NULL for
 *          eigenvalues only.
 * info     host pointer (may be NULL), filled on return.
 * Errors: BSE_ERR_ARG, BSE_ERR_NOT_PD_AMINUSB (info = column), BSE_ERR_CUDA,
 *         BSE_ERR_NOMEM, BSE_ERR_NO_CONVERGENCE.
 */
bse_status bse_solve_chol(bse_handle h, int64_t n, const double* A, int64_t lda, const double* B,
                          int64_t ldb, int64_t il, int64_t iu, int prec, double* omega, double* X,
                          int64_t ldx, double* Y, int64_t ldy, bse_info* info, void* stream);

/*
 * SVD method, Alg. 3 (Section 3.3):
 *   L1 L1^H = A + B;  L2 L2^H = A - B;  U Lambda V^H = L1^H L2 (SVD);
 *   V1 = L1 U Lambda^{-1/2};  V2 = L2 V Lambda^{-1/2};
 *   X = (V1 + V2)/2,  Y = (V2 - V1)/2.
 * omega are the singular values of L1^H L2 (not square roots of computed
 * squares; Section 3.3 after Alg. 3).  Arguments as for bse_solve_chol;
 * additional error BSE_ERR_NOT_PD_APLUSB (info = column).
 */
bse_status bse_solve_svd(bse_handle h, int64_t n, const double* A, int64_t lda, const double* B,
                         int64_t ldb, int64_t il, int64_t iu, int prec, double* omega, double* X,
                         int64_t ldx, double* Y, int64_t ldy, bse_info* info, void* stream);

/*
 * Square-root method, Alg. 1 (Section 3.1), the established approach the
 * paper compares against (Table 2: 28 2/3 n^3 flops against 13 1/3 for
 * Alg. 2):
 *   S = (A - B)^{1/2} = Q D^{1/2} Q^H from the eigendecomposition
 *   A - B = Q D Q^H;  M = S (A + B) S;  M V_M = V_M D_M;  Lambda = D_M^{1/2};
 *   V1 = S^{-1} V_M Lambda^{1/2};  V2 = S V_M Lambda^{-1/2};
 *   X = (V1 + V2)/2,  Y = (V2 - V1)/2.
 * Arguments, precisions and errors as for bse_solve_chol, except that
 * BSE_ERR_NOT_PD_AMINUSB reports in info the 1-based index (ascending) of a
 * non-positive eigenvalue of A - B, and a non-positive eigenvalue of M gives
 * BSE_ERR_NOT_PD_APLUSB (info 0).  The profiler's stage 1 covers the square
 * root (eigensolve of A - B, S and S^{-1}).
 */
bse_status bse_solve_sqrt(bse_handle h, int64_t n, const double* A, int64_t lda, const double* B,
                          int64_t ldb, int64_t il, int64_t iu, int prec, double* omega, double* X,
                          int64_t ldx, double* Y, int64_t ldy, bse_info* info, void* stream);

/*
 * Tamm-Dancoff approximation, B = 0 (Section 4, the TDA remark on the LiF
 * example): H1 = [A 0; 0 -A], so omega are the eigenvalues of A (ascending)
 * and the eigenvector of omega_i is [x_i; 0] with x_i^H x_i = 1; Y is not
 * materialised.  One Householder reduction of A, the tridiagonal solve and
 * one back-transformation (the eigensolve of Alg. 2 step 2 applied to A).
 * A        device, n x n Hermitian, lower triangle read; must be positive
 *          definite (else BSE_ERR_NOT_PD_APLUSB, info 0).
 * il, iu   1-based inclusive range into the ascending omega.
 * omega    device, k = iu - il + 1 doubles.
 * X        device, n x k complex, leading dimension ldx; NULL for
 *          eigenvalues only.
 * FP64 arithmetic throughout.
 */
bse_status bse_solve_tda(bse_handle h, int64_t n, const double* A, int64_t lda, int64_t il, int64_t iu,
                         double* omega, double* X, int64_t ldx, bse_info* info, void* stream);

/*
 * Gradient of L = sum_i w_i omega_i with respect to Hermitian A and B.
 * Thm. 3 item 3 (left eigenvector of H1 is v^H Sigma) with the
 * Sigma-normalisation of Eq. (13) give d omega_i = v_i^H [dA dB; dB dA] v_i,
 * hence (Frobenius inner product on Hermitian matrices)
 *   dA = sum_i w_i (x_i x_i^H + y_i y_i^H),  dB = sum_i w_i (x_i y_i^H + y_i x_i^H).
 * Valid for simple omega_i only (not differentiable at multiplicity > 1).
 * X, Y     device, n x k, the k selected columns of a solve's output.
 * w        device, k doubles (dL/d omega_i).
 * dA, dB   device, n x n complex, full Hermitian matrices written.
 */
bse_status bse_grad(bse_handle h, int64_t n, int64_t k, const double* X, int64_t ldx, const double* Y,
                    int64_t ldy, const double* w, double* dA, int64_t ldda, double* dB, int64_t lddb,
                    void* stream);

/*
 * End-to-end variant: identical to bse_solve_chol (method = BSE_METHOD_CHOL),
 * bse_solve_svd (BSE_METHOD_SVD) or bse_solve_sqrt (BSE_METHOD_SQRT), but
 * every data pointer (A, B, omega, X,
 * Y) is a HOST pointer.  The library copies A and B to device workspace
 * (pinned host memory gives full PCIe/C2C bandwidth), solves, and copies
 * omega, X, Y back before returning.
 */
bse_status bse_solve_host(bse_handle h, int method, int64_t n, const double* A, int64_t lda,
                          const double* B, int64_t ldb, int64_t il, int64_t iu, int prec,
                          double* omega, double* X, int64_t ldx, double* Y, int64_t ldy,
                          bse_info* info, void* stream);

/*
 * Batched solves (Alg. 2 or Alg. 3 for each instance): `count` independent
 * problems of sizes n[i] (1 <= n[i] <= 1024), the k lowest eigenpairs of each
 * (k_i = min(k, n[i])), in ONE persistent kernel launch: each CTA takes the
 * next instance from a queue ordered by decreasing n and solves it alone.
 * n        host array, count sizes.
 * A, B     host arrays of count DEVICE pointers; instance i is n[i] x n[i]
 *          Hermitian with leading dimension n[i] (lower triangle read).
 * omega    host array of count device pointers to k_i doubles (ascending).
 * X, Y     host arrays of count device pointers to n[i] x k_i complex
 *          matrices, leading dimension n[i].
 * status   host array of count int64 (may be NULL): 0 or the instance's
 *          bse_status code.  The return value is BSE_OK when every instance
 *          succeeded, else the first failing instance's code.
 * method   BSE_METHOD_CHOL or BSE_METHOD_SVD;
 * prec     BSE_PREC_FP64.
 */
bse_status bse_solve_batched(bse_handle h, int64_t count, const int64_t* n, const double* const* A,
                             const double* const* B, int64_t k, int method, int prec, double* const* omega,
                             double* const* X, double* const* Y, int64_t* status, void* stream);

/*
 * Enqueue-only form of bse_solve_batched, for CUDA-graph capture: copies
 * the instance table from library-owned pinned host memory, resets the
 * queue, launches the persistent kernel and returns without synchronising.
 * dstatus  DEVICE array of 2*count int64 written by the kernel (code, info
 *          per instance); read it after synchronising the stream.
 * The pointer arrays must describe the same sizes on every replay of a
 * captured graph (the table is rebuilt at capture time).
 */
bse_status bse_solve_batched_async(bse_handle h, int64_t count, const int64_t* n, const double* const* A,
                                   const double* const* B, int64_t k, int method, int prec,
                                   double* const* omega, double* const* X, double* const* Y,
                                   int64_t* dstatus, void* stream);

/* Number of CUDA kernel launches the library has issued so far in this
 * process (all handles, all entry points). */
int64_t bse_launch_count(bse_handle h);

/*
 * Profiling (tracing aid, not part of the paper): while enabled, the solves
 * of this handle record CUDA events around each pipeline stage and around
 * every launch of the FP64 GEMM engine, on the solve's stream.  Times are
 * device times between those events; GEMM flops count only the useful
 * (structurally nonzero) multiply-adds, 8 real flops per complex MAC.
 * bse_profile_enable resets the counters; bse_profile_read returns them
 * (the solves already synchronise their stream, so no extra sync happens).
 */
#define BSE_NSTAGES 10
/* stage index: 0 form A+-B, 1 Cholesky (square root for Alg. 1),
 * 2 congruence / product L1^H L2,
 * 3 Householder reduction, 4 tridiagonal eigensolve, 5 orthogonalisation,
 * 6 back-transformation, 7 post-processing + final setup, 8 gradient,
 * 9 refinement (mixed form) */
typedef struct bse_profile_data {
  double stage_ms[BSE_NSTAGES];
  int64_t stage_calls[BSE_NSTAGES];
  double gemm_ms;         /* sum of per-launch device times of the GEMM engine */
  double gemm_flops;      /* useful flops of those launches */
  int64_t gemm_launches;
  int64_t launches;       /* all kernel launches while enabled */
  /* mixed form: the tensor-core product kernels alone (operand splitting
   * excluded), with the FP64-equivalent useful flops of their products;
   * one BF16 slice-pair product set is 36 times those flops */
  double tc_ms;
  double tc_flops;
  int64_t tc_launches;
} bse_profile_data;
/* enable: 0 off, 1 stages and GEMMs, 2 additionally every launch of the
 * reduction and tridiagonal kernels (adds two events per launch). */
bse_status bse_profile_enable(bse_handle h, int enable);
bse_status bse_profile_read(bse_handle h, bse_profile_data* out);
/* Level-2 per-kernel summary, one "name launches total_ms" line per kernel,
 * written NUL-terminated into buf (truncated to len); returns the full length. */
int64_t bse_profile_kernels(bse_handle h, char* buf, size_t len);

/*
 * Out-of-core tile executor for the BLAS3 stages of Alg. 2 (form A +- B,
 * step 1's Cholesky factorisation L L^H = A - B and step 2's congruence
 * M = L^H (A + B) L) when the matrices live in HOST memory: the problem
 * sizes of Section 4's runtime discussion (n ~ 1e5, 160 GB per complex
 * matrix) exceed the GPU's memory with A, B, L and M together.
 *
 * A run executes a PLAN: a list of operations on nb x nb complex128 tiles
 * (column-major, leading dimension nb) made by a planner that knows the task
 * order (the package's ooc.plan: Belady eviction under a tile budget):
 *   LOAD t     host tile t -> a free device slot (copy stream)
 *   ALLOC t    a free device slot, zero-filled, becomes tile t (no transfer)
 *   COMPUTE i  task i on the caller's stream (its tiles must be resident)
 *   STORE t    device tile t -> host tile t (copy stream)
 *   FREE t     tile t gives its slot back
 * Copies run on a copy stream and tasks on three compute streams (the
 * caller's and two the call creates), ordered only by events on the tiles
 * they share (a task waits for its tiles' last writers and, for the tile it
 * writes, for the reads since; a LOAD waits for the previous tile of its
 * slot): copies overlap tasks and independent tasks overlap each other.
 * The results do not depend on that overlap (same bits on every run).
 *
 * Tasks (out is read and written unless the plan ALLOCs it first):
 *   FORM_SUM   out = in0 + in1             (tiles of A and B -> A + B)
 *   FORM_DIFF  out = in0 - in1             (-> A - B)
 *   POTRF      out = chol(out), lower; the strict upper part is set to 0;
 *              the tile's inverse conjugate transpose is kept for TRSM
 *   TRSM       out = out L^{-H}, L the tile in0 (the latest POTRF's tile)
 *   HERK       out -= in0 in0^H            (lower part of out only)
 *   GEMM_SUB   out -= in0 in1^H
 *   GEMM_ACC   out += op(in0) in1, op by flags:
 *              BSE_OOC_IN0_CONJT   op(in0) = in0^H
 *              BSE_OOC_IN0_HERM    in0 is a Hermitian diagonal tile stored in
 *                                  its lower part: op(in0) = tril + tril(-1)^H
 *              BSE_OOC_IN0_LOWER   in0 is lower triangular (structure mask)
 *              BSE_OOC_IN1_LOWER   in1 is lower triangular (structure mask)
 *
 * nb          tile size, 1 <= nb <= 4096.
 * host_tiles  ntiles HOST pointers, each to nb*nb complex128 (2 nb^2 doubles);
 *             page-locked memory lets copies overlap with tasks.  Tiles that
 *             are only ALLOCed and never stored may be NULL.
 * ops, nops   the plan, executed in order.
 * tasks       ntasks task descriptors referenced by COMPUTE.
 * budget      device tile slots (>= the tiles any one task touches); the
 *             library allocates budget + 1 slots and scratch for the run in
 *             the handle's workspace.
 * info        host, may be NULL: info->info = failing 1-based GLOBAL column
 *             of a POTRF task that met a non-positive pivot (the plan's
 *             tile row of that task times nb plus the column in the tile;
 *             the row is taken from the task's BSE_OOC_ROW(flags) field).
 * stream      the caller's stream (one of the compute streams; it waits for
 *             the others at the end); the call returns after every STORE
 *             has completed.
 * Errors: BSE_ERR_ARG (a plan that is inconsistent: a tile used while not
 * resident, loaded twice, more than `budget` resident, an index out of
 * range; nothing is enqueued then), BSE_ERR_NOT_PD_AMINUSB, BSE_ERR_CUDA,
 * BSE_ERR_NOMEM.  FP64 arithmetic (the GEMM engine) in every task.
 */
typedef enum { BSE_OOC_LOAD = 0, BSE_OOC_ALLOC = 1, BSE_OOC_COMPUTE = 2, BSE_OOC_STORE = 3, BSE_OOC_FREE = 4 } bse_ooc_opkind;
typedef enum {
  BSE_OOC_FORM_SUM = 0,
  BSE_OOC_FORM_DIFF = 1,
  BSE_OOC_POTRF = 2,
  BSE_OOC_TRSM = 3,
  BSE_OOC_HERK = 4,
  BSE_OOC_GEMM_SUB = 5,
  BSE_OOC_GEMM_ACC = 6
} bse_ooc_taskkind;
#define BSE_OOC_IN0_CONJT 1
#define BSE_OOC_IN0_HERM 2
#define BSE_OOC_IN0_LOWER 4
#define BSE_OOC_IN1_LOWER 8
/* POTRF: tile row k of the task stored in flags bits 8..31 */
#define BSE_OOC_ROW(flags) ((int64_t)(((uint32_t)(flags)) >> 8))
typedef struct bse_ooc_op {
  int32_t kind;  /* bse_ooc_opkind */
  int32_t arg;   /* tile index (LOAD, ALLOC, STORE, FREE) or task index (COMPUTE) */
} bse_ooc_op;
typedef struct bse_ooc_task {
  int32_t kind;  /* bse_ooc_taskkind */
  int32_t out;   /* tile written */
  int32_t in0;   /* tiles read, -1 when unused */
  int32_t in1;
  int32_t flags;
} bse_ooc_task;
bse_status bse_ooc_run(bse_handle h, int64_t nb, int64_t ntiles, void* const* host_tiles, int64_t nops,
                       const bse_ooc_op* ops, int64_t ntasks, const bse_ooc_task* tasks, int64_t budget,
                       bse_info* info, void* stream);

/*
 * Allocation-free Cholesky solve of ONE small problem.  The paper has no
 * counterpart: this entry point serves callers that cannot allocate device
 * memory (device memory wholly held by another allocator's pool; latency-
 * critical loops where cudaMalloc/cudaFree would lock or synchronise the
 * device; services that must not meet out-of-memory after start-up).  It
 * computes what bse_solve_chol computes with il = 1, iu = k (Alg. 2, the
 * lowest k pairs), with one thread block on one SM, and allocates nothing:
 * no device or pinned memory, no handle, no host heap.  Its workspace is a
 * fixed __device__ array of BSE_NOALLOC_SCRATCH_BYTES that exists once the
 * CUDA module holding it is loaded on the device.  Under CUDA's default lazy
 * module loading that load happens inside the first call on each device,
 * and it is the one point where device memory is taken (the scratch plus the
 * modules' code): make the first call at start-up, before another allocator
 * claims the memory.  A call with n == 0 does this set-up and solves nothing.
 * n        1 <= n <= BSE_NOALLOC_MAX_N; larger n returns BSE_ERR_TOO_LARGE
 *          without launching anything; n == 0 (set-up only) or k == 0
 *          returns BSE_OK.
 * k        0 <= k <= n.
 * A, B     device, n x n Hermitian, leading dimension n (packed), lower
 *          triangle read.
 * omega    device, k doubles (ascending).
 * X, Y     device, n x k, leading dimension n.
 * info     host, may be NULL: info->info = failing 1-based column for the
 *          not-positive-definite codes, else 0.
 * stream   work is enqueued on it, then the stream is synchronised.
 * Set-up: the first call with a device current loads the modules, looks up
 * the scratch address for that device and sets the kernel's attributes;
 * make that first call before any stream capture on it.
 * Calls that overlap on one device share the scratch and race: serialise
 * them.  This entry point reports through its return code only; it does not
 * update bse_last_error().
 */
#define BSE_NOALLOC_MAX_N 256
#define BSE_NOALLOC_SCRATCH_BYTES (8 * 1024 * 1024)
bse_status bse_solve_chol_noalloc(int64_t n, int64_t k, const double* A, const double* B, double* omega, double* X,
                                  double* Y, bse_info* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BSE_GB300_H */
