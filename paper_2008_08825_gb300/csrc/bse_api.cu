// C ABI (include/bse.h): handle, workspace planning and the two solver
// pipelines of the paper.
//
// Alg. 2 (CHOL), all on the device, one stream:
//   form M1 = A + B (full Hermitian) and M2 = A - B (lower)        [Thm. ProdEig]
//   L L^H = M2                        blocked Cholesky             [step 1]
//   W = M1 L, M = L^H W (lower)       two triangular GEMMs         [step 2]
//   T = Q^H M Q                       Householder tridiagonal      [step 2]
//   T Z = Z D (selected)              bisection + twisted vectors  [step 2]
//   V_M = Q Z                         blocked back-transformation  [step 2]
//   omega = sqrt(D)                                                [step 3]
//   P = L^{-H} V_M                    blocked triangular solve     [step 4]
//   X, Y = ((c1 P + c2 L V_M)/2, (c2 L V_M - c1 P)/2),
//   c1 = sqrt(omega), c2 = 1/sqrt(omega)   triangular GEMM + fused epilogue [steps 4-6]
// Alg. 3 (SVD):
//   L1 L1^H = A + B, L2 L2^H = A - B  blocked Cholesky x2          [steps 1-2]
//   G = L1^H L2                       triangular x triangular GEMM [step 3]
//   G = Q_L B Q_R^H                   Householder bidiagonal       [step 3]
//   Golub-Kahan tridiagonal of B: bisection + twisted vectors      [step 3]
//   U = Q_L U_B, V = Q_R V_B          blocked back-transformations [step 3]
//   X, Y from L1 U and L2 V with c1 = c2 = 1/sqrt(omega)           [steps 4-6]
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "prof.cuh"

// ---- ooc.cu ----
size_t ooc_ws_bytes(int64_t nb, int64_t budget);
const char* ooc_validate(int64_t nb, int64_t ntiles, void* const* host_tiles, int64_t nops, const bse_ooc_op* ops,
                         int64_t ntasks, const bse_ooc_task* tasks, int64_t budget, std::string& why);
bse_status ooc_execute(cudaStream_t s, void* ws, int64_t nb, int64_t ntiles, void* const* host_tiles, int64_t nops,
                       const bse_ooc_op* ops, const bse_ooc_task* tasks, int64_t budget, int64_t** status_out);

static thread_local std::string g_err;
void bse_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }
long long bse_total_launches();

struct bse_context {
  int device = 0;
  void* ws = nullptr;      // internal workspace
  size_t ws_bytes = 0;
  void* user_ws = nullptr;  // caller-supplied workspace
  size_t user_bytes = 0;
  void* io = nullptr;       // staging for bse_solve_host
  size_t io_bytes = 0;
  int64_t* host_status = nullptr;  // pinned, 2 entries
  Profiler* prof = nullptr;
  int prof_on = 0;
  void* bws = nullptr;       // batched workspace
  size_t bws_bytes = 0;
  char* bdesc_host = nullptr;  // pinned instance table
  size_t bdesc_bytes = 0;
  int sms = 0;
  int64_t oz_min = (int64_t)1 << 24;
  int oz_engine = OZ_ENGINE_TCGEN05;
  int64_t oz_wait = 0;  // 0: the engine's default wait limit
  int batch_cps = 1;
  int batch_team = 0;          // 0: the library default
  int tune_hemv = 0;           // launch shapes (0: the library defaults)
  int tune_splitk = 0;
  int64_t batch_team_min = 0;  // 0: the library default
};

// Makes the handle's profiler current for this thread for one entry point;
// on exit synchronises the stream (the entry points do anyway) and folds the
// recorded events into the counters.
struct ProfGuard {
  bse_context* h;
  cudaStream_t s;
  ProfGuard(bse_context* hh, cudaStream_t ss) : h(hh), s(ss) { prof_set_current(h->prof_on ? h->prof : nullptr); }
  ~ProfGuard() {
    if (prof_current()) {
      cudaStreamSynchronize(s);
      prof_flush(h->prof);
    }
    prof_set_current(nullptr);
  }
};

// Makes the handle's launch shapes current for one entry point.
struct TuneGuard {
  explicit TuneGuard(const bse_context* h) { tuning_set_current(LaunchTuning{h->tune_hemv, h->tune_splitk}); }
  ~TuneGuard() { tuning_set_current(LaunchTuning{0, 0}); }
};

// Makes the tensor-core product workspace current for one solve (mixed form).
struct OzGuard {
  explicit OzGuard(const OzWork& w) { oz_set_current(w); }
  ~OzGuard() { oz_set_current(OzWork{nullptr, 0, 0, OZ_ENGINE_TCGEN05, 0}); }
};

// ---------------------------------------------------------------------------
// Workspace plan: a bump allocator over one region, 256-byte aligned pieces.
struct Plan {
  char* base;
  size_t off = 0;
  explicit Plan(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += sizeof(T) * (count > 0 ? count : 1);
    return p;
  }
};

struct TriPlan {
  TriWork w;
  void carve(Plan& pl, int64_t N, int64_t k) {
    w.a = pl.take<double>(N);
    w.off = pl.take<double>(N);
    w.e2 = pl.take<double>(N);
    w.lam = pl.take<double>(N);
    w.blk = pl.take<int>(N);
    w.rank = pl.take<int>(N);
    w.bstart = pl.take<int>(N + 2);
    w.prm = pl.take<double>(8);
    w.iprm = pl.take<int>(8);
    w.scratch = pl.take<double>((size_t)N * k);
    w.E = pl.take<double>((size_t)k * k);
    w.Ef = pl.take<float>((size_t)k * k);
    w.Z2 = pl.take<double>((size_t)N * k);
    w.grid = pl.take<int>(tri_grid_points());
  }
};

struct RefineBufs {
  cplx *F1, *F2, *work;  // full M1, full M2, 4 n k
  double *est, *est_max;
};

static void carve_refine(Plan& pl, RefineBufs& r, int64_t n, int64_t k, int prec) {
  const bool on = prec == BSE_PREC_MIXED;
  r.F1 = on ? pl.take<cplx>((size_t)n * n) : nullptr;
  r.F2 = on ? pl.take<cplx>((size_t)n * n) : nullptr;
  r.work = on ? pl.take<cplx>((size_t)4 * n * k) : nullptr;
  r.est = on ? pl.take<double>(k) : nullptr;
  r.est_max = on ? pl.take<double>(1) : nullptr;
}

struct CholBuffers {
  void* oz;
  RefineBufs rf;
  int64_t* status;
  cplx *M1, *L, *Linv, *W, *P;
  HetrdWork h;
  TriPlan t;
  double *Z, *lam, *c1, *c2;
  cplx* tmp;
};

static void carve_chol(Plan& pl, CholBuffers& b, int64_t n, int64_t k, int prec) {
  const int nbt = hetrd_panel();
  b.oz = prec == BSE_PREC_MIXED ? pl.take<char>(oz_work_bytes(n, 8)) : nullptr;
  carve_refine(pl, b.rf, n, k, prec);
  b.status = pl.take<int64_t>(4);
  b.M1 = pl.take<cplx>((size_t)n * n);
  b.L = pl.take<cplx>((size_t)n * n);
  b.Linv = pl.take<cplx>(chol_linv_elems(n));
  b.W = pl.take<cplx>((size_t)n * n);
  b.P = pl.take<cplx>((size_t)n * k);
  b.h.V = pl.take<cplx>((size_t)n * n);
  b.h.W = pl.take<cplx>((size_t)n * nbt);
  b.h.tau = pl.take<cplx>(n);
  b.h.d = pl.take<double>(n);
  b.h.e = pl.take<double>(n);
  b.h.part = pl.take<cplx>(hetrd_part_elems(n));
  b.h.small = pl.take<cplx>(4 * nbt * nbt + 64);
  b.h.S2 = pl.take<cplx>((size_t)n * 2 * nbt);
  b.t.carve(pl, n, k);
  b.Z = pl.take<double>((size_t)n * k);
  b.lam = pl.take<double>(k);
  b.c1 = pl.take<double>(k);
  b.c2 = pl.take<double>(k);
  b.tmp = pl.take<cplx>(backtransform_tmp_elems(k));
}

struct SvdBuffers {
  void* oz;
  RefineBufs rf;
  int64_t* status;
  cplx *L1, *L2, *Linv, *G, *Uc, *Vc, *T1;
  GebrdWork g;
  TriPlan t;
  double *Z, *UB, *VB, *lam, *c1, *c2, *off;
  cplx* tmp;
};

static void carve_svd(Plan& pl, SvdBuffers& b, int64_t n, int64_t k, int prec) {
  const int nbt = 32;
  b.oz = prec == BSE_PREC_MIXED ? pl.take<char>(oz_work_bytes(n, 8)) : nullptr;
  carve_refine(pl, b.rf, n, k, prec);
  b.status = pl.take<int64_t>(4);
  b.L1 = pl.take<cplx>((size_t)n * n);
  b.L2 = pl.take<cplx>((size_t)n * n);
  b.Linv = pl.take<cplx>(chol_linv_elems(n));
  b.G = pl.take<cplx>((size_t)n * n);
  b.Uc = pl.take<cplx>((size_t)n * k);
  b.Vc = pl.take<cplx>((size_t)n * k);
  b.T1 = pl.take<cplx>((size_t)n * k);
  b.g.U = pl.take<cplx>((size_t)n * n);
  b.g.Vr = pl.take<cplx>((size_t)n * n);
  b.g.X = pl.take<cplx>((size_t)n * nbt);
  b.g.Y = pl.take<cplx>((size_t)n * nbt);
  b.g.tauq = pl.take<cplx>(n);
  b.g.taup = pl.take<cplx>(n);
  b.g.d = pl.take<double>(n);
  b.g.e = pl.take<double>(n);
  b.g.part = pl.take<cplx>(gebrd_part_elems(n));
  b.g.small = pl.take<cplx>(4 * nbt + 64);
  b.g.S2 = pl.take<cplx>((size_t)n * 2 * nbt);
  b.t.carve(pl, 2 * n, k);
  b.Z = pl.take<double>((size_t)2 * n * k);
  b.UB = pl.take<double>((size_t)n * k);
  b.VB = pl.take<double>((size_t)n * k);
  b.off = pl.take<double>(2 * n);
  b.lam = pl.take<double>(k);
  b.c1 = pl.take<double>(k);
  b.c2 = pl.take<double>(k);
  b.tmp = pl.take<cplx>(backtransform_tmp_elems(k));
}

// Alg. 1: M1 = A + B (full), A - B reduced in M, its eigenvectors Q, the square
// root S and its inverse Si, a product buffer T; the reduction and tridiagonal
// work serve both eigensolves (all n vectors for the square root).
struct SqrtBuffers {
  void* oz;
  RefineBufs rf;
  int64_t* status;
  cplx *M1, *M, *Q, *S, *Si, *T;
  HetrdWork h;
  TriPlan t;
  double *Z, *d2, *qp, *qm, *lam, *c1, *c2;
  cplx* tmp;
};

static void carve_sqrt(Plan& pl, SqrtBuffers& b, int64_t n, int64_t k, int prec) {
  const int nbt = hetrd_panel();
  b.oz = prec == BSE_PREC_MIXED ? pl.take<char>(oz_work_bytes(n, 8)) : nullptr;
  carve_refine(pl, b.rf, n, k, prec);
  b.status = pl.take<int64_t>(4);
  b.M1 = pl.take<cplx>((size_t)n * n);
  b.M = pl.take<cplx>((size_t)n * n);
  b.Q = pl.take<cplx>((size_t)n * n);
  b.S = pl.take<cplx>((size_t)n * n);
  b.Si = pl.take<cplx>((size_t)n * n);
  b.T = pl.take<cplx>((size_t)n * n);
  b.h.V = pl.take<cplx>((size_t)n * n);
  b.h.W = pl.take<cplx>((size_t)n * nbt);
  b.h.tau = pl.take<cplx>(n);
  b.h.d = pl.take<double>(n);
  b.h.e = pl.take<double>(n);
  b.h.part = pl.take<cplx>(hetrd_part_elems(n));
  b.h.small = pl.take<cplx>(4 * nbt * nbt + 64);
  b.h.S2 = pl.take<cplx>((size_t)n * 2 * nbt);
  b.t.carve(pl, n, n);
  b.Z = pl.take<double>((size_t)n * n);
  b.d2 = pl.take<double>(n);
  b.qp = pl.take<double>(n);
  b.qm = pl.take<double>(n);
  b.lam = pl.take<double>(k);
  b.c1 = pl.take<double>(k);
  b.c2 = pl.take<double>(k);
  b.tmp = pl.take<cplx>(backtransform_tmp_elems(n));
}

// Tamm-Dancoff (B = 0): the Hermitian eigenproblem of A alone
struct TdaBuffers {
  int64_t* status;
  cplx* M;
  HetrdWork h;
  TriPlan t;
  double *Z, *lam, *c1, *c2;
  cplx* tmp;
};

static void carve_tda(Plan& pl, TdaBuffers& b, int64_t n, int64_t k) {
  const int nbt = hetrd_panel();
  b.status = pl.take<int64_t>(4);
  b.M = pl.take<cplx>((size_t)n * n);
  b.h.V = pl.take<cplx>((size_t)n * n);
  b.h.W = pl.take<cplx>((size_t)n * nbt);
  b.h.tau = pl.take<cplx>(n);
  b.h.d = pl.take<double>(n);
  b.h.e = pl.take<double>(n);
  b.h.part = pl.take<cplx>(hetrd_part_elems(n));
  b.h.small = pl.take<cplx>(4 * nbt * nbt + 64);
  b.h.S2 = pl.take<cplx>((size_t)n * 2 * nbt);
  b.t.carve(pl, n, k);
  b.Z = pl.take<double>((size_t)n * k);
  b.lam = pl.take<double>(k);
  b.c1 = pl.take<double>(k);
  b.c2 = pl.take<double>(k);
  b.tmp = pl.take<cplx>(backtransform_tmp_elems(k));
}

static size_t plan_bytes(int64_t n, int64_t k, int method, int prec) {
  Plan pl(nullptr);
  if (method == BSE_METHOD_CHOL) {
    CholBuffers b;
    carve_chol(pl, b, n, k, prec);
  } else if (method == BSE_METHOD_SVD) {
    SvdBuffers b;
    carve_svd(pl, b, n, k, prec);
  } else if (method == BSE_METHOD_SQRT) {
    SqrtBuffers b;
    carve_sqrt(pl, b, n, k, prec);
  } else {
    TdaBuffers b;
    carve_tda(pl, b, n, k);
  }
  return pl.off + 256;
}

static bse_status ensure_ws(bse_context* h, size_t bytes, void** out) {
  if (h->user_ws) {
    if (h->user_bytes < bytes) {
      bse_internal_set_error("caller-supplied workspace too small");
      return BSE_ERR_NOMEM;
    }
    *out = h->user_ws;
    return BSE_OK;
  }
  if (h->ws_bytes < bytes) {
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      bse_internal_set_error("cudaMalloc of workspace failed");
      return BSE_ERR_NOMEM;
    }
    h->ws_bytes = bytes;
  }
  *out = h->ws;
  return BSE_OK;
}

// ---------------------------------------------------------------------------
// Kernels for the Golub-Kahan set-up and the singular-vector split.
__global__ void gk_offdiag_kernel(int64_t n, const double* d, const double* e, double* off) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) off[2 * i] = d[i];
  if (i < n - 1) off[2 * i + 1] = e[i];
}
// z = [v1, u1, v2, u2, ...]/sqrt(2):  U_B(i, c) = sqrt2 z(2i+1, c), V_B(i, c) = sqrt2 z(2i, c)
__global__ void gk_split_kernel(int64_t n, int64_t k, const double* Z, int64_t ldz, double* UB, double* VB) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i >= n || c >= k) return;
  const double r2 = 1.4142135623730951;
  VB[i + c * n] = r2 * Z[2 * i + c * ldz];
  UB[i + c * n] = r2 * Z[2 * i + 1 + c * ldz];
}

#define TRY(x)                \
  do {                        \
    bse_status r_ = (x);      \
    if (r_ != BSE_OK) return r_; \
  } while (0)

static bse_status check_common(bse_handle h, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                               int64_t il, int64_t iu, int prec, double* omega, double* X, int64_t ldx, double* Y,
                               int64_t ldy) {
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  if (n < 0) return bse_internal_set_error("n < 0"), BSE_ERR_ARG;
  if (n == 0) return BSE_OK;
  if (!A || !B || !omega) return bse_internal_set_error("NULL A, B or omega"), BSE_ERR_ARG;
  if (lda < n || ldb < n) return bse_internal_set_error("lda or ldb < n"), BSE_ERR_ARG;
  if (il < 1 || iu > n || il > iu) return bse_internal_set_error("need 1 <= il <= iu <= n"), BSE_ERR_ARG;
  if ((X == nullptr) != (Y == nullptr)) return bse_internal_set_error("X and Y must both be given or both NULL"), BSE_ERR_ARG;
  if (X && (ldx < n || ldy < n)) return bse_internal_set_error("ldx or ldy < n"), BSE_ERR_ARG;
  if (prec != BSE_PREC_FP64 && prec != BSE_PREC_MIXED) return bse_internal_set_error("unknown precision"), BSE_ERR_ARG;
  return BSE_OK;
}

static bse_status finish(bse_context* h, cudaStream_t s, const int64_t* dstatus, bse_info* info,
                         const double* est_max = nullptr) {
  BSE_CUDA(cudaMemcpyAsync(h->host_status, dstatus, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (est_max) BSE_CUDA(cudaMemcpyAsync(h->host_status + 2, est_max, sizeof(double), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  const int64_t code = h->host_status[0];
  if (info) {
    info->info = h->host_status[1];
    double e = 0.0;
    if (est_max) memcpy(&e, h->host_status + 2, sizeof(double));
    info->err_est = e;
    info->refine_iters = est_max ? 1 : 0;
  }
  if (code != 0) {
    char buf[128];
    snprintf(buf, sizeof buf, "device status %lld (info %lld)", (long long)code, (long long)h->host_status[1]);
    bse_internal_set_error(buf);
  }
  return (bse_status)code;
}

static bse_status solve_chol_dev(bse_context* h, int64_t n, const cplx* A, int64_t lda, const cplx* B, int64_t ldb,
                                 int64_t il, int64_t iu, int prec, double* omega, cplx* X, int64_t ldx, cplx* Y,
                                 int64_t ldy, bse_info* info, cudaStream_t s) {
  const int64_t k = iu - il + 1;
  void* ws;
  TRY(ensure_ws(h, plan_bytes(n, k, BSE_METHOD_CHOL, prec), &ws));
  Plan pl(ws);
  CholBuffers b;
  carve_chol(pl, b, n, k, prec);
  OzGuard ozg(OzWork{b.oz, b.oz ? oz_work_bytes(n, 8) : 0, h->oz_min, h->oz_engine, h->oz_wait});
  int64_t* st = b.status;
  BSE_CUDA(cudaMemsetAsync(st, 0, 4 * sizeof(int64_t), s));
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  TuneGuard tgd(h);
  ProfGuard pgd(h, s);
  // M1 = A + B (full), M2 = A - B (lower, in L)
  {
    StageScope sc(0, s);
    TRY(form_sum(s, n, A, lda, B, ldb, +1.0, b.M1, n, 1));
    TRY(form_sum(s, n, A, lda, B, ldb, -1.0, b.L, n, 0));
    if (b.rf.F1 && X) {
      TRY(form_sum(s, n, A, lda, B, ldb, +1.0, b.rf.F1, n, 1));
      TRY(form_sum(s, n, A, lda, B, ldb, -1.0, b.rf.F2, n, 1));
    }
  }
  {
    StageScope sc(1, s);
    TRY(potrf_lower(s, n, b.L, n, b.Linv, st, BSE_ERR_NOT_PD_AMINUSB));
  }
  // W = M1 L ; M = L^H W (lower) into M1's buffer
  StageScope sc2(2, s);
  GemmParams<cplx> p1 = gemm_params<cplx>(n, n, n, OPN, b.M1, n, OPN, b.L, n, one, zero, b.W, n);
  p1.triB = TRI_LO;
  p1.status = st;
  TRY(gemm_z(s, p1));
  GemmParams<cplx> p2 = gemm_params<cplx>(n, n, n, OPC, b.L, n, OPN, b.W, n, one, zero, b.M1, n);
  p2.triA = TRI_UP;
  p2.lowerC = 1;
  p2.status = st;
  TRY(gemm_z(s, p2));
  prof_stage_end(2, s);
  // Hermitian eigendecomposition of M
  {
    StageScope sc(3, s);
    TRY(hetrd_lower(s, n, b.M1, n, b.h, st));
  }
  {
    StageScope sc(4, s);
    TRY(tridiag_eig(s, n, b.h.d, b.h.e, 0, il - 1, iu - 1, b.lam, X ? b.Z : nullptr, n, b.t.w, st));
    TRY(finish_omega(s, k, b.lam, 0, omega, b.c1, b.c2, st));
  }
  if (!X) return finish(h, s, st, info);
  {
    StageScope sc(5, s);
    TRY(orthonormalize_columns(s, n, k, b.Z, n, b.t.w, st));
  }
  cplx* VM = b.W;  // reuse: V_M = Q Z (n x k)
  {
    StageScope sc(6, s);
    TRY(real_to_complex(s, n, k, b.Z, n, VM, n));
    TRY(hetrd_backtransform(s, n, k, b.h, VM, n, b.tmp, st));
  }
  // P = L^{-H} V_M
  StageScope sc7(7, s);
  BSE_CUDA(cudaMemcpy2DAsync(b.P, sizeof(cplx) * n, VM, sizeof(cplx) * n, sizeof(cplx) * n, k,
                             cudaMemcpyDeviceToDevice, s));
  TRY(trsm_lower_conjtrans(s, n, k, b.L, n, b.Linv, b.P, n, st));
  // X, Y from P (= V1 unscaled) and L V_M (= V2 unscaled)
  GemmParams<cplx> p3 = gemm_params<cplx>(n, k, n, OPN, b.L, n, OPN, VM, n, one, zero, X, ldx);
  p3.triA = TRI_LO;
  p3.status = st;
  p3.epi = EPI_XY;
  p3.P = b.P, p3.ldp = n, p3.c1 = b.c1, p3.c2 = b.c2, p3.Y = Y, p3.ldy = ldy;
  TRY(gemm_z(s, p3));
  if (b.rf.F1) {
    StageScope scr(9, s);
    TRY(refine_omega(s, n, k, b.rf.F1, b.rf.F2, X, ldx, Y, ldy, b.rf.work, omega, b.rf.est, b.rf.est_max, st, 1));
    return finish(h, s, st, info, b.rf.est_max);
  }
  return finish(h, s, st, info);
}

static bse_status solve_svd_dev(bse_context* h, int64_t n, const cplx* A, int64_t lda, const cplx* B, int64_t ldb,
                                int64_t il, int64_t iu, int prec, double* omega, cplx* X, int64_t ldx, cplx* Y,
                                int64_t ldy, bse_info* info, cudaStream_t s) {
  const int64_t k = iu - il + 1;
  void* ws;
  TRY(ensure_ws(h, plan_bytes(n, k, BSE_METHOD_SVD, prec), &ws));
  Plan pl(ws);
  SvdBuffers b;
  carve_svd(pl, b, n, k, prec);
  OzGuard ozg(OzWork{b.oz, b.oz ? oz_work_bytes(n, 8) : 0, h->oz_min, h->oz_engine, h->oz_wait});
  int64_t* st = b.status;
  BSE_CUDA(cudaMemsetAsync(st, 0, 4 * sizeof(int64_t), s));
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  TuneGuard tgd(h);
  ProfGuard pgd(h, s);
  {
    StageScope sc(0, s);
    TRY(form_sum(s, n, A, lda, B, ldb, +1.0, b.L1, n, 0));
    TRY(form_sum(s, n, A, lda, B, ldb, -1.0, b.L2, n, 0));
    if (b.rf.F1 && X) {
      TRY(form_sum(s, n, A, lda, B, ldb, +1.0, b.rf.F1, n, 1));
      TRY(form_sum(s, n, A, lda, B, ldb, -1.0, b.rf.F2, n, 1));
    }
  }
  {
    StageScope sc(1, s);
    TRY(potrf_lower(s, n, b.L1, n, b.Linv, st, BSE_ERR_NOT_PD_APLUSB));
    TRY(potrf_lower(s, n, b.L2, n, b.Linv, st, BSE_ERR_NOT_PD_AMINUSB));
  }
  // G = L1^H L2
  prof_stage_begin(2, s);
  GemmParams<cplx> pg = gemm_params<cplx>(n, n, n, OPC, b.L1, n, OPN, b.L2, n, one, zero, b.G, n);
  pg.triA = TRI_UP;
  pg.triB = TRI_LO;
  pg.status = st;
  TRY(gemm_z(s, pg));
  prof_stage_end(2, s);
  {
    StageScope sc(3, s);
    TRY(gebrd_upper(s, n, b.G, n, b.g, st));
  }
  // Golub-Kahan tridiagonal (size 2n, zero diagonal)
  prof_stage_begin(4, s);
  gk_offdiag_kernel<<<ceil_div_u(n, 256), 256, 0, s>>>(n, b.g.d, b.g.e, b.off);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  TRY(tridiag_eig(s, 2 * n, nullptr, b.off, 1, il - 1, iu - 1, b.lam, X ? b.Z : nullptr, 2 * n, b.t.w, st));
  TRY(finish_omega(s, k, b.lam, 1, omega, b.c1, b.c2, st));
  prof_stage_end(4, s);
  if (!X) return finish(h, s, st, info);
  {
    StageScope sc(5, s);
    dim3 gsp(ceil_div_u(n, 256), (unsigned)k);
    gk_split_kernel<<<gsp, 256, 0, s>>>(n, k, b.Z, 2 * n, b.UB, b.VB);
    bse_count_launch();
    BSE_LAUNCH_CHECK();
    TRY(orthonormalize_columns(s, n, k, b.UB, n, b.t.w, st));
    TRY(orthonormalize_columns(s, n, k, b.VB, n, b.t.w, st));
  }
  {
    StageScope sc(6, s);
    TRY(real_to_complex(s, n, k, b.UB, n, b.Uc, n));
    TRY(real_to_complex(s, n, k, b.VB, n, b.Vc, n));
    TRY(gebrd_backtransform(s, 0, n, k, b.g, b.Uc, n, b.tmp, st));
    TRY(gebrd_backtransform(s, 1, n, k, b.g, b.Vc, n, b.tmp, st));
  }
  StageScope sc7(7, s);
  // T1 = L1 U ; X, Y from T1 and L2 V with c1 = c2 = 1/sqrt(omega)
  GemmParams<cplx> p1 = gemm_params<cplx>(n, k, n, OPN, b.L1, n, OPN, b.Uc, n, one, zero, b.T1, n);
  p1.triA = TRI_LO;
  p1.status = st;
  TRY(gemm_z(s, p1));
  GemmParams<cplx> p2 = gemm_params<cplx>(n, k, n, OPN, b.L2, n, OPN, b.Vc, n, one, zero, X, ldx);
  p2.triA = TRI_LO;
  p2.status = st;
  p2.epi = EPI_XY;
  p2.P = b.T1, p2.ldp = n, p2.c1 = b.c1, p2.c2 = b.c2, p2.Y = Y, p2.ldy = ldy;
  TRY(gemm_z(s, p2));
  if (b.rf.F1) {
    StageScope scr(9, s);
    // Alg. 3's singular values keep their relative accuracy (the Golub-Kahan
    // bisection); the Rayleigh quotient of the pencil is accurate only
    // normwise, so for the SVD method omega stays and only the residuals go out
    TRY(refine_omega(s, n, k, b.rf.F1, b.rf.F2, X, ldx, Y, ldy, b.rf.work, omega, b.rf.est, b.rf.est_max, st, 0));
    return finish(h, s, st, info, b.rf.est_max);
  }
  return finish(h, s, st, info);
}


// ---------------------------------------------------------------------------
// Batched solves.
// Alg. 1 (square-root method): S = (A - B)^{1/2} from the eigendecomposition
// A - B = Q diag(d) Q^H; M = S (A + B) S; M V_M = V_M D; Lambda = D^{1/2};
// V1 = S^{-1} V_M Lambda^{1/2}, V2 = S V_M Lambda^{-1/2}; X, Y as in Alg. 2.
static bse_status solve_sqrt_dev(bse_context* h, int64_t n, const cplx* A, int64_t lda, const cplx* B, int64_t ldb,
                                 int64_t il, int64_t iu, int prec, double* omega, cplx* X, int64_t ldx, cplx* Y,
                                 int64_t ldy, bse_info* info, cudaStream_t s) {
  const int64_t k = iu - il + 1;
  void* ws;
  TRY(ensure_ws(h, plan_bytes(n, k, BSE_METHOD_SQRT, prec), &ws));
  Plan pl(ws);
  SqrtBuffers b;
  carve_sqrt(pl, b, n, k, prec);
  OzGuard ozg(OzWork{b.oz, b.oz ? oz_work_bytes(n, 8) : 0, h->oz_min, h->oz_engine, h->oz_wait});
  int64_t* st = b.status;
  BSE_CUDA(cudaMemsetAsync(st, 0, 4 * sizeof(int64_t), s));
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  TuneGuard tgd(h);
  ProfGuard pgd(h, s);
  {
    StageScope sc(0, s);
    TRY(form_sum(s, n, A, lda, B, ldb, +1.0, b.M1, n, 1));
    TRY(form_sum(s, n, A, lda, B, ldb, -1.0, b.M, n, 0));
    if (b.rf.F1 && X) {
      TRY(form_sum(s, n, A, lda, B, ldb, +1.0, b.rf.F1, n, 1));
      TRY(form_sum(s, n, A, lda, B, ldb, -1.0, b.rf.F2, n, 1));
    }
  }
  {
    // the square root of A - B (Alg. 1 step 1): a full Hermitian eigensolve
    StageScope sc(1, s);
    TRY(hetrd_lower(s, n, b.M, n, b.h, st));
    TRY(tridiag_eig(s, n, b.h.d, b.h.e, 0, 0, n - 1, b.d2, b.Z, n, b.t.w, st));
    TRY(orthonormalize_columns(s, n, n, b.Z, n, b.t.w, st));
    TRY(real_to_complex(s, n, n, b.Z, n, b.Q, n));
    TRY(hetrd_backtransform(s, n, n, b.h, b.Q, n, b.tmp, st));
    TRY(sqrt_factors(s, n, b.d2, b.qp, b.qm, st));
    TRY(scale_columns(s, n, n, b.Q, n, b.qp, b.T, n));
    GemmParams<cplx> ps = gemm_params<cplx>(n, n, n, OPN, b.T, n, OPC, b.T, n, one, zero, b.S, n);
    ps.lowerC = 1;
    ps.status = st;
    TRY(gemm_z(s, ps));
    TRY(hermitian_fill_upper(s, n, b.S, n));
    TRY(scale_columns(s, n, n, b.Q, n, b.qm, b.T, n));
    GemmParams<cplx> pi = gemm_params<cplx>(n, n, n, OPN, b.T, n, OPC, b.T, n, one, zero, b.Si, n);
    pi.lowerC = 1;
    pi.status = st;
    TRY(gemm_z(s, pi));
    TRY(hermitian_fill_upper(s, n, b.Si, n));
  }
  {
    // M = S (A + B) S (lower), into M
    StageScope sc(2, s);
    GemmParams<cplx> p1 = gemm_params<cplx>(n, n, n, OPN, b.M1, n, OPN, b.S, n, one, zero, b.T, n);
    p1.status = st;
    TRY(gemm_z(s, p1));
    GemmParams<cplx> p2 = gemm_params<cplx>(n, n, n, OPN, b.S, n, OPN, b.T, n, one, zero, b.M, n);
    p2.lowerC = 1;
    p2.status = st;
    TRY(gemm_z(s, p2));
  }
  {
    StageScope sc(3, s);
    TRY(hetrd_lower(s, n, b.M, n, b.h, st));
  }
  {
    StageScope sc(4, s);
    TRY(tridiag_eig(s, n, b.h.d, b.h.e, 0, il - 1, iu - 1, b.lam, X ? b.Z : nullptr, n, b.t.w, st));
    TRY(finish_omega(s, k, b.lam, 0, omega, b.c1, b.c2, st));
  }
  if (!X) return finish(h, s, st, info);
  {
    StageScope sc(5, s);
    TRY(orthonormalize_columns(s, n, k, b.Z, n, b.t.w, st));
  }
  cplx* VM = b.Q;  // reuse: V_M (n x k)
  {
    StageScope sc(6, s);
    TRY(real_to_complex(s, n, k, b.Z, n, VM, n));
    TRY(hetrd_backtransform(s, n, k, b.h, VM, n, b.tmp, st));
  }
  StageScope sc7(7, s);
  // P = S^{-1} V_M (V1 unscaled) into T; X, Y from P and S V_M (V2 unscaled)
  GemmParams<cplx> p3 = gemm_params<cplx>(n, k, n, OPN, b.Si, n, OPN, VM, n, one, zero, b.T, n);
  p3.status = st;
  TRY(gemm_z(s, p3));
  GemmParams<cplx> p4 = gemm_params<cplx>(n, k, n, OPN, b.S, n, OPN, VM, n, one, zero, X, ldx);
  p4.status = st;
  p4.epi = EPI_XY;
  p4.P = b.T, p4.ldp = n, p4.c1 = b.c1, p4.c2 = b.c2, p4.Y = Y, p4.ldy = ldy;
  TRY(gemm_z(s, p4));
  if (b.rf.F1) {
    StageScope scr(9, s);
    TRY(refine_omega(s, n, k, b.rf.F1, b.rf.F2, X, ldx, Y, ldy, b.rf.work, omega, b.rf.est, b.rf.est_max, st, 1));
    return finish(h, s, st, info, b.rf.est_max);
  }
  return finish(h, s, st, info);
}

// Tamm-Dancoff approximation (B = 0): omega = eig(A) (ascending, positive),
// X = the unit eigenvectors of A, Y = 0 (not materialised).
static bse_status solve_tda_dev(bse_context* h, int64_t n, const cplx* A, int64_t lda, int64_t il, int64_t iu,
                                double* omega, cplx* X, int64_t ldx, bse_info* info, cudaStream_t s) {
  const int64_t k = iu - il + 1;
  void* ws;
  TRY(ensure_ws(h, plan_bytes(n, k, BSE_METHOD_TDA, BSE_PREC_FP64), &ws));
  Plan pl(ws);
  TdaBuffers b;
  carve_tda(pl, b, n, k);
  int64_t* st = b.status;
  BSE_CUDA(cudaMemsetAsync(st, 0, 4 * sizeof(int64_t), s));
  TuneGuard tgd(h);
  ProfGuard pgd(h, s);
  {
    StageScope sc(0, s);
    TRY(form_sum(s, n, A, lda, A, lda, 0.0, b.M, n, 0));
  }
  {
    StageScope sc(3, s);
    TRY(hetrd_lower(s, n, b.M, n, b.h, st));
  }
  {
    StageScope sc(4, s);
    TRY(tridiag_eig(s, n, b.h.d, b.h.e, 0, il - 1, iu - 1, b.lam, X ? b.Z : nullptr, n, b.t.w, st));
    TRY(finish_omega(s, k, b.lam, 1, omega, b.c1, b.c2, st));
  }
  if (!X) return finish(h, s, st, info);
  {
    StageScope sc(5, s);
    TRY(orthonormalize_columns(s, n, k, b.Z, n, b.t.w, st));
  }
  {
    StageScope sc(6, s);
    TRY(real_to_complex(s, n, k, b.Z, n, X, ldx));
    TRY(hetrd_backtransform(s, n, k, b.h, X, ldx, b.tmp, st));
  }
  return finish(h, s, st, info);
}

static bse_status batched_enqueue(bse_context* h, int64_t count, const int64_t* n, const double* const* A,
                                  const double* const* B, int64_t k, int method, int prec, double* const* omega,
                                  double* const* X, double* const* Y, int64_t** dstatus_out, int64_t* dstatus_user,
                                  cudaStream_t s) {
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  if (count < 0 || k < 1) return bse_internal_set_error("count < 0 or k < 1"), BSE_ERR_ARG;
  if (method != BSE_METHOD_CHOL && method != BSE_METHOD_SVD) return bse_internal_set_error("unknown method"), BSE_ERR_ARG;
  if (prec != BSE_PREC_FP64) return bse_internal_set_error("batched solves are FP64 only"), BSE_ERR_NOT_IMPLEMENTED;
  if (count == 0) return BSE_OK;
  if (!n || !A || !B || !omega || !X || !Y) return bse_internal_set_error("NULL array"), BSE_ERR_ARG;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > batched_max_n()) return bse_internal_set_error("batched n out of [1, 1024]"), BSE_ERR_ARG;
    if (!A[i] || !B[i] || !omega[i] || !X[i] || !Y[i]) return bse_internal_set_error("NULL instance pointer"), BSE_ERR_ARG;
  }
  // largest first (longest-processing-time order for the persistent queue)
  std::vector<int64_t> order(count);
  for (int64_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return n[a] > n[b]; });
  size_t ws_total = 0;
  std::vector<size_t> offs(count);
  for (int64_t q = 0; q < count; ++q) {
    const int64_t i = order[q];
    offs[q] = ws_total;
    const int64_t ki = k < n[i] ? k : n[i];
    ws_total += method == BSE_METHOD_SVD ? batched_svd_inst_bytes(n[i], ki) : batched_inst_bytes(n[i], ki);
  }
  const size_t desc_bytes = (batched_desc_bytes() * count + 255) & ~(size_t)255;
  const size_t stat_bytes = ((size_t)16 * count + 255) & ~(size_t)255;
  const size_t need = ws_total + desc_bytes + stat_bytes + 256;
  if (h->bws_bytes < need) {
    if (h->bws) cudaFree(h->bws);
    h->bws = nullptr;
    h->bws_bytes = 0;
    if (cudaMalloc(&h->bws, need) != cudaSuccess) {
      cudaGetLastError();
      return bse_internal_set_error("cudaMalloc of batched workspace failed"), BSE_ERR_NOMEM;
    }
    h->bws_bytes = need;
  }
  if (h->bdesc_bytes < desc_bytes) {
    if (h->bdesc_host) cudaFreeHost(h->bdesc_host);
    h->bdesc_host = nullptr;
    h->bdesc_bytes = 0;
    if (cudaMallocHost(&h->bdesc_host, desc_bytes) != cudaSuccess) {
      cudaGetLastError();
      return bse_internal_set_error("cudaMallocHost of the instance table failed"), BSE_ERR_NOMEM;
    }
    h->bdesc_bytes = desc_bytes;
  }
  char* base = (char*)h->bws;
  char* ddesc = base + ws_total;
  int64_t* dstat = dstatus_user ? dstatus_user : (int64_t*)(ddesc + desc_bytes);
  int* counter = (int*)(ddesc + desc_bytes + stat_bytes);
  for (int64_t q = 0; q < count; ++q) {
    const int64_t i = order[q];
    batched_fill_desc(h->bdesc_host + q * batched_desc_bytes(), n[i], k < n[i] ? k : n[i], A[i], B[i], omega[i],
                      X[i], Y[i], base + offs[q], dstat + 2 * i);
  }
  BSE_CUDA(cudaMemcpyAsync(ddesc, h->bdesc_host, batched_desc_bytes() * count, cudaMemcpyHostToDevice, s));
  BSE_CUDA(cudaMemsetAsync(dstat, 0, 16 * count, s));
  const int grid = (int)std::min<int64_t>(count, (int64_t)h->sms * h->batch_cps);
  const int team = h->batch_team ? h->batch_team : batched_team_default();
  const int64_t team_min = h->batch_team_min ? h->batch_team_min : batched_team_min_n_default();
  int64_t nbig = 0;  // the table is sorted by decreasing n
  while (nbig < count && n[order[nbig]] >= team_min) ++nbig;
  TRY(batched_chol_launch(s, ddesc, count, counter, grid, method, nbig, team));
  if (dstatus_out) *dstatus_out = dstat;
  return BSE_OK;
}

extern "C" bse_status bse_solve_batched_async(bse_handle h, int64_t count, const int64_t* n, const double* const* A,
                                              const double* const* B, int64_t k, int method, int prec,
                                              double* const* omega, double* const* X, double* const* Y,
                                              int64_t* dstatus, void* stream) {
  if (!dstatus && count > 0) return bse_internal_set_error("NULL dstatus"), BSE_ERR_ARG;
  return batched_enqueue(h, count, n, A, B, k, method, prec, omega, X, Y, nullptr, dstatus, (cudaStream_t)stream);
}

extern "C" bse_status bse_solve_batched(bse_handle h, int64_t count, const int64_t* n, const double* const* A,
                                        const double* const* B, int64_t k, int method, int prec, double* const* omega,
                                        double* const* X, double* const* Y, int64_t* status, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int64_t* dstat = nullptr;
  TRY(batched_enqueue(h, count, n, A, B, k, method, prec, omega, X, Y, &dstat, nullptr, s));
  if (count == 0) return BSE_OK;
  std::vector<int64_t> hs(2 * count);
  BSE_CUDA(cudaMemcpyAsync(hs.data(), dstat, 16 * count, cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  bse_status first = BSE_OK;
  for (int64_t i = 0; i < count; ++i) {
    if (status) status[i] = hs[2 * i];
    if (hs[2 * i] != 0 && first == BSE_OK) {
      first = (bse_status)hs[2 * i];
      char buf[128];
      snprintf(buf, sizeof buf, "batched instance %lld: status %lld (info %lld)", (long long)i, (long long)hs[2 * i],
               (long long)hs[2 * i + 1]);
      bse_internal_set_error(buf);
    }
  }
  return first;
}

// ---------------------------------------------------------------------------
extern "C" {

bse_status bse_create(bse_handle* out) {
  if (!out) return bse_internal_set_error("NULL output"), BSE_ERR_ARG;
  bse_context* h = new bse_context();
  BSE_CUDA(cudaGetDevice(&h->device));
  if (cudaMallocHost(&h->host_status, 4 * sizeof(int64_t)) != cudaSuccess) {  // code, info, err_est
    cudaGetLastError();
    delete h;
    return bse_internal_set_error("cudaMallocHost failed"), BSE_ERR_NOMEM;
  }
  h->prof = prof_new();
  BSE_CUDA(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device));
  *out = h;
  return BSE_OK;
}

bse_status bse_destroy(bse_handle h) {
  if (!h) return BSE_OK;
  prof_delete(h->prof);
  if (h->ws) cudaFree(h->ws);
  if (h->io) cudaFree(h->io);
  if (h->host_status) cudaFreeHost(h->host_status);
  if (h->bws) cudaFree(h->bws);
  if (h->bdesc_host) cudaFreeHost(h->bdesc_host);
  delete h;
  return BSE_OK;
}

const char* bse_last_error(void) { return g_err.c_str(); }

bse_status bse_workspace_size(int64_t n, int method, int prec, size_t* bytes) {
  if (!bytes || n < 0 || method < BSE_METHOD_CHOL || method > BSE_METHOD_TDA ||
      (prec != BSE_PREC_FP64 && prec != BSE_PREC_MIXED))
    return bse_internal_set_error("bad argument to bse_workspace_size"), BSE_ERR_ARG;
  *bytes = plan_bytes(n, n > 0 ? n : 1, method, prec);
  return BSE_OK;
}

bse_status bse_set_workspace(bse_handle h, void* ptr, size_t bytes) {
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  if (ptr && ((uintptr_t)ptr & 255)) return bse_internal_set_error("workspace must be 256-byte aligned"), BSE_ERR_ARG;
  h->user_ws = ptr;
  h->user_bytes = ptr ? bytes : 0;
  return BSE_OK;
}

bse_status bse_solve_chol(bse_handle h, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                          int64_t il, int64_t iu, int prec, double* omega, double* X, int64_t ldx, double* Y,
                          int64_t ldy, bse_info* info, void* stream) {
  bse_status r = check_common(h, n, A, lda, B, ldb, il, iu, prec, omega, X, ldx, Y, ldy);
  if (r != BSE_OK || n == 0) return r;
  return solve_chol_dev(h, n, (const cplx*)A, lda, (const cplx*)B, ldb, il, iu, prec, omega, (cplx*)X, ldx, (cplx*)Y,
                        ldy, info, (cudaStream_t)stream);
}

bse_status bse_solve_svd(bse_handle h, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                         int64_t il, int64_t iu, int prec, double* omega, double* X, int64_t ldx, double* Y,
                         int64_t ldy, bse_info* info, void* stream) {
  bse_status r = check_common(h, n, A, lda, B, ldb, il, iu, prec, omega, X, ldx, Y, ldy);
  if (r != BSE_OK || n == 0) return r;
  return solve_svd_dev(h, n, (const cplx*)A, lda, (const cplx*)B, ldb, il, iu, prec, omega, (cplx*)X, ldx, (cplx*)Y,
                       ldy, info, (cudaStream_t)stream);
}

bse_status bse_solve_sqrt(bse_handle h, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                          int64_t il, int64_t iu, int prec, double* omega, double* X, int64_t ldx, double* Y,
                          int64_t ldy, bse_info* info, void* stream) {
  bse_status r = check_common(h, n, A, lda, B, ldb, il, iu, prec, omega, X, ldx, Y, ldy);
  if (r != BSE_OK || n == 0) return r;
  return solve_sqrt_dev(h, n, (const cplx*)A, lda, (const cplx*)B, ldb, il, iu, prec, omega, (cplx*)X, ldx, (cplx*)Y,
                        ldy, info, (cudaStream_t)stream);
}

bse_status bse_solve_tda(bse_handle h, int64_t n, const double* A, int64_t lda, int64_t il, int64_t iu,
                         double* omega, double* X, int64_t ldx, bse_info* info, void* stream) {
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  if (n < 0) return bse_internal_set_error("n < 0"), BSE_ERR_ARG;
  if (n == 0) return BSE_OK;
  if (!A || !omega) return bse_internal_set_error("NULL A or omega"), BSE_ERR_ARG;
  if (lda < n) return bse_internal_set_error("lda < n"), BSE_ERR_ARG;
  if (il < 1 || iu > n || il > iu) return bse_internal_set_error("need 1 <= il <= iu <= n"), BSE_ERR_ARG;
  if (X && ldx < n) return bse_internal_set_error("ldx < n"), BSE_ERR_ARG;
  return solve_tda_dev(h, n, (const cplx*)A, lda, il, iu, omega, (cplx*)X, ldx, info, (cudaStream_t)stream);
}

bse_status bse_grad(bse_handle h, int64_t n, int64_t k, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                    const double* w, double* dA, int64_t ldda, double* dB, int64_t lddb, void* stream) {
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  if (n < 0 || k < 0) return bse_internal_set_error("n or k < 0"), BSE_ERR_ARG;
  if (n == 0) return BSE_OK;
  if (!dA || !dB || (k > 0 && (!X || !Y || !w))) return bse_internal_set_error("NULL pointer"), BSE_ERR_ARG;
  if (ldda < n || lddb < n || (k > 0 && (ldx < n || ldy < n))) return bse_internal_set_error("leading dimension < n"), BSE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  TuneGuard tgd(h);
  ProfGuard pgd(h, s);
  StageScope sc(8, s);
  TRY(grad_outer(s, n, k, (const cplx*)X, ldx, (const cplx*)Y, ldy, w, (cplx*)dA, ldda, (cplx*)dB, lddb));
  BSE_CUDA(cudaStreamSynchronize(s));
  return BSE_OK;
}

bse_status bse_solve_host(bse_handle h, int method, int64_t n, const double* A, int64_t lda, const double* B,
                          int64_t ldb, int64_t il, int64_t iu, int prec, double* omega, double* X, int64_t ldx,
                          double* Y, int64_t ldy, bse_info* info, void* stream) {
  if (method != BSE_METHOD_CHOL && method != BSE_METHOD_SVD && method != BSE_METHOD_SQRT)
    return bse_internal_set_error("unknown method"), BSE_ERR_ARG;
  bse_status r = check_common(h, n, A, lda, B, ldb, il, iu, prec, omega, X, ldx, Y, ldy);
  if (r != BSE_OK || n == 0) return r;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t k = iu - il + 1;
  Plan need(nullptr);
  need.take<cplx>((size_t)n * n);
  need.take<cplx>((size_t)n * n);
  need.take<double>(k);
  if (X) need.take<cplx>((size_t)n * k), need.take<cplx>((size_t)n * k);
  if (h->io_bytes < need.off + 256) {
    if (h->io) cudaFree(h->io);
    h->io = nullptr;
    h->io_bytes = 0;
    if (cudaMalloc(&h->io, need.off + 256) != cudaSuccess) {
      cudaGetLastError();
      return bse_internal_set_error("cudaMalloc of staging buffers failed"), BSE_ERR_NOMEM;
    }
    h->io_bytes = need.off + 256;
  }
  Plan pl(h->io);
  cplx* dA = pl.take<cplx>((size_t)n * n);
  cplx* dB = pl.take<cplx>((size_t)n * n);
  double* dom = pl.take<double>(k);
  cplx *dX = nullptr, *dY = nullptr;
  if (X) dX = pl.take<cplx>((size_t)n * k), dY = pl.take<cplx>((size_t)n * k);
  BSE_CUDA(cudaMemcpy2DAsync(dA, sizeof(cplx) * n, A, sizeof(cplx) * lda, sizeof(cplx) * n, n, cudaMemcpyHostToDevice, s));
  BSE_CUDA(cudaMemcpy2DAsync(dB, sizeof(cplx) * n, B, sizeof(cplx) * ldb, sizeof(cplx) * n, n, cudaMemcpyHostToDevice, s));
  r = method == BSE_METHOD_CHOL  ? solve_chol_dev(h, n, dA, n, dB, n, il, iu, prec, dom, dX, n, dY, n, info, s)
      : method == BSE_METHOD_SVD ? solve_svd_dev(h, n, dA, n, dB, n, il, iu, prec, dom, dX, n, dY, n, info, s)
                                 : solve_sqrt_dev(h, n, dA, n, dB, n, il, iu, prec, dom, dX, n, dY, n, info, s);
  if (r != BSE_OK) return r;
  BSE_CUDA(cudaMemcpyAsync(omega, dom, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  if (X) {
    BSE_CUDA(cudaMemcpy2DAsync(X, sizeof(cplx) * ldx, dX, sizeof(cplx) * n, sizeof(cplx) * n, k, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaMemcpy2DAsync(Y, sizeof(cplx) * ldy, dY, sizeof(cplx) * n, sizeof(cplx) * n, k, cudaMemcpyDeviceToHost, s));
  }
  BSE_CUDA(cudaStreamSynchronize(s));
  return BSE_OK;
}

bse_status bse_ooc_run(bse_handle h, int64_t nb, int64_t ntiles, void* const* host_tiles, int64_t nops,
                       const bse_ooc_op* ops, int64_t ntasks, const bse_ooc_task* tasks, int64_t budget,
                       bse_info* info, void* stream) {
  // the plan is checked on the host before anything else (no CUDA call)
  std::string why;
  const char* bad = ooc_validate(nb, ntiles, host_tiles, nops, ops, ntasks, tasks, budget, why);
  if (bad) return bse_internal_set_error(bad), BSE_ERR_ARG;
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  if (info) *info = bse_info{};
  if (nops == 0) return BSE_OK;
  cudaStream_t s = (cudaStream_t)stream;
  void* ws;
  TRY(ensure_ws(h, ooc_ws_bytes(nb, budget), &ws));
  int64_t* dstatus = nullptr;
  const bse_status r = ooc_execute(s, ws, nb, ntiles, host_tiles, nops, ops, tasks, budget, &dstatus);
  if (r != BSE_OK) {
    cudaStreamSynchronize(s);
    return r;
  }
  BSE_CUDA(cudaMemcpyAsync(h->host_status, dstatus, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  const int64_t code = h->host_status[0], row = h->host_status[2];
  if (code != 0) {
    const int64_t col = row >= 0 ? row * nb + h->host_status[1] : h->host_status[1];
    if (info) info->info = col;
    char buf[128];
    snprintf(buf, sizeof buf, "device status %lld (global column %lld)", (long long)code, (long long)col);
    bse_internal_set_error(buf);
  }
  return (bse_status)code;
}

int64_t bse_launch_count(bse_handle h) {
  (void)h;
  return (int64_t)bse_total_launches();
}

bse_status bse_set_option(bse_handle h, int option, int64_t value) {
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  if (option == BSE_OPT_TC_MIN_MNK) {
    if (value < 1) return bse_internal_set_error("BSE_OPT_TC_MIN_MNK must be >= 1"), BSE_ERR_ARG;
    h->oz_min = value;
    return BSE_OK;
  }
  if (option == BSE_OPT_TC_ENGINE) {
    if (value != 0 && value != 1) return bse_internal_set_error("BSE_OPT_TC_ENGINE must be 0 or 1"), BSE_ERR_ARG;
    h->oz_engine = (int)value;
    return BSE_OK;
  }
  if (option == BSE_OPT_TC_WAIT_CYCLES) {
    if (value < 0 || value > ((int64_t)1 << 36))
      return bse_internal_set_error("BSE_OPT_TC_WAIT_CYCLES must be in [0, 2^36]"), BSE_ERR_ARG;
    h->oz_wait = value;
    return BSE_OK;
  }
  if (option == BSE_OPT_HEMV_ITEM_TILES) {
    if (value < 0 || value > 16) return bse_internal_set_error("BSE_OPT_HEMV_ITEM_TILES must be in [0, 16]"), BSE_ERR_ARG;
    h->tune_hemv = (int)value;
    return BSE_OK;
  }
  if (option == BSE_OPT_SPLITK_MAX) {
    if (value < 0 || value > 8) return bse_internal_set_error("BSE_OPT_SPLITK_MAX must be in [0, 8]"), BSE_ERR_ARG;
    h->tune_splitk = (int)value;
    return BSE_OK;
  }
  if (option == BSE_OPT_BATCH_TEAM) {
    if (value != 1 && value != 2 && value != 4 && value != 8)
      return bse_internal_set_error("BSE_OPT_BATCH_TEAM must be 1, 2, 4 or 8"), BSE_ERR_ARG;
    h->batch_team = (int)value;
    return BSE_OK;
  }
  if (option == BSE_OPT_BATCH_TEAM_MIN_N) {
    if (value < 1) return bse_internal_set_error("BSE_OPT_BATCH_TEAM_MIN_N must be >= 1"), BSE_ERR_ARG;
    h->batch_team_min = value;
    return BSE_OK;
  }
  if (option == BSE_OPT_BATCH_CTAS_PER_SM) {
    if (value != 1 && value != 2) return bse_internal_set_error("BSE_OPT_BATCH_CTAS_PER_SM must be 1 or 2"), BSE_ERR_ARG;
    h->batch_cps = (int)value;
    return BSE_OK;
  }
  return bse_internal_set_error("unknown option"), BSE_ERR_ARG;
}

bse_status bse_profile_enable(bse_handle h, int enable) {
  if (!h) return bse_internal_set_error("NULL handle"), BSE_ERR_ARG;
  h->prof_on = enable ? 1 : 0;
  prof_set_fine(h->prof, enable >= 2);
  prof_reset(h->prof);
  return BSE_OK;
}

int64_t bse_profile_kernels(bse_handle h, char* buf, size_t len) {
  if (!h) return -1;
  return prof_kernel_summary(h->prof, buf, len);
}

bse_status bse_profile_read(bse_handle h, bse_profile_data* out) {
  if (!h || !out) return bse_internal_set_error("NULL argument"), BSE_ERR_ARG;
  prof_read(h->prof, out);
  return BSE_OK;
}

}  // extern "C"
