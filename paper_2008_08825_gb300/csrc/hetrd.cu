// Householder reduction of the Hermitian M of Alg. 2 to a real symmetric
// tridiagonal T = Q^H M Q (lower storage), and the back-transformation
// V_M = Q Z of the eigenvectors Z of T.
//
// Blocked in panels of NBT columns.  Within a panel the matrix is kept as
// panel-start A plus the correction -V W^H - W V^H (V: reflectors, W: their
// images); column j of the panel
//   1. receives the correction (tr_col_update) and the norm of its tail,
//   2. gets the reflector H_j = I - tau v v^H with H_j^H x = beta e_1,
//      beta real (tr_house), so T is real,
//   3. w = tau (A22 v - V (W^H v) - W (V^H v)) with A22 v from the lower
//      triangle, 64 x 64 tiles, each tile read once (tr_hemv_strip),
//   4. w += -tau/2 (w^H v) v  -- so that H_j^H A H_j = A - v w^H - w v^H.
// After the panel, the trailing lower triangle takes the rank-2*NBT update
// through the GEMM engine.  On GB300 step 3 is bound by the FP64 pipe, not by
// HBM (n'^2 complex MACs over n'^2 * 16 bytes needs 3.4 TFLOP/s to saturate
// 6.8 TB/s; the part delivers 1.2), so the one-stage reduction does the same
// FP64 work as a band reduction and saves its second back-transformation.
#include <atomic>
#include <cmath>

#include "kernels.cuh"
#include "prof.cuh"

constexpr int NBT = 32;    // panel width
constexpr int RB = 64;     // rows per CTA (and threads) of the per-column row kernels
constexpr int BTB = 128;   // reflectors per block in the back-transformation
constexpr int GSPLIT = 64;  // split-K layers of the Gram product V^H V of a block
constexpr int WSPLIT = 8;   // at most this many split-K layers of W1 = V^H Z

int hetrd_panel() { return NBT; }
int backtransform_block() { return BTB; }
size_t backtransform_tmp_elems(int64_t k) {
  return (size_t)(2 + GSPLIT) * BTB * BTB + (2 + WSPLIT) * (size_t)BTB * k;
}

// SM count of the current device (looked up once per device)
static int device_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> sms_of[kMaxDev];
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError(), dev = -1;
  if (dev >= 0 && dev < kMaxDev) sms = sms_of[dev].load(std::memory_order_relaxed);
  if (!sms) {
    if (dev < 0 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 152;  // GB300
    }
    if (dev >= 0 && dev < kMaxDev) sms_of[dev].store(sms, std::memory_order_relaxed);
  }
  return sms;
}

static thread_local LaunchTuning g_tuning = {0, 0};
void tuning_set_current(const LaunchTuning& t) { g_tuning = t; }
LaunchTuning tuning_current() { return g_tuning; }

// Split-K layers for a product whose tiles do not fill the GPU: the count
// s <= WSPLIT (or the tuned cap) that brings tiles * s closest to whole
// waves of `slots` CTAs.
static int split_layers(int64_t tiles, int slots) {
  if (tiles >= 4 * slots) return 1;
  const int cap = g_tuning.splitk_max > 0 && g_tuning.splitk_max < WSPLIT ? g_tuning.splitk_max : WSPLIT;
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= cap; ++s) {
    const double work = (double)tiles * s;
    const double eff = work / (slots * std::ceil(work / slots));
    if (eff > best_eff + 0.02) best = s, best_eff = eff;
  }
  return best;
}
constexpr int HR = 8;      // default: at most this many row tiles per work item of the strip matvec
// partial-sum slots of the matvec: one per 32-wide column strip (row
// products) plus one per chunk of row tiles (column products; at most one
// per strip)
static inline int64_t hemv_slots(int64_t n) {
  const int64_t nst = (n + 31) / 32;
  return 2 * nst;
}
// row tiles (64 x 32) per work item: up to HR, fewer while that leaves under
// ~4 items per CTA (ntr^2 tiles in all, two CTAs per SM)
static inline int hemv_chunk(int64_t ntr) {
  const int64_t cap = g_tuning.hemv_items > 0 ? g_tuning.hemv_items : HR;
  const int64_t c = ntr * ntr / 1216;
  return c < 1 ? 1 : (c > cap ? (int)cap : (int)c);
}
size_t hetrd_part_elems(int64_t n) {
  // partial-sum slots, norm and dot partials, and the matvec's per-column
  // work-queue counters (n ints)
  return (size_t)(hemv_slots(n) + 2) * (size_t)(n + 1) + 4 * (n / RB + 2) + 4 * NBT + 64 + (size_t)(n / 4 + 4);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < (blockDim.x >> 5)) t = red[threadIdx.x];
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;  // valid in thread 0
}

__device__ __forceinline__ cplx block_sum_c(cplx v, double* red) {
  const double a = block_sum(v.x, red);
  const double b = block_sum(v.y, red);
  return mkc(a, b);
}

// 1. column update + norm partial sums of rows >= j+2.  With nfin > 0 it
// also finishes the previous column's w (step 4 below, w += alpha v with
// alpha = -tau/2 (w^H v) from nfin partial sums): every CTA forms alpha, uses
// the finished w and stores it for its rows > j (row j is read by every CTA
// and needed by no later step, so it is left as it was).
__global__ void __launch_bounds__(RB) tr_col_update(int64_t n, int64_t p, int64_t j, cplx* __restrict__ A,
                                                    int64_t lda, const cplx* __restrict__ V, int64_t ldv,
                                                    cplx* __restrict__ W, int64_t ldw, double* __restrict__ d,
                                                    double* __restrict__ npart, const double* __restrict__ dpart,
                                                    int nfin, const cplx* __restrict__ tau, const int64_t* status) {
  __shared__ cplx vj[NBT], wj[NBT];
  __shared__ cplx falpha;
  __shared__ double red[32];
  if (*(volatile const int64_t*)status) return;
  const int jj = (int)(j - p);
  const bool fin = nfin > 0 && jj > 0;
  if (fin && threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nfin; ++i) a += dpart[2 * i], b += dpart[2 * i + 1];
    falpha = cscale(cmul(tau[j - 1], mkc(a, b)), -0.5);
  }
  __syncthreads();
  if (threadIdx.x < jj) {
    vj[threadIdx.x] = V[IDX2(j, p + threadIdx.x, ldv)];
    cplx w0 = W[IDX2(j, threadIdx.x, ldw)];
    if (fin && threadIdx.x == jj - 1) w0 = cadd(w0, cmul(falpha, V[IDX2(j, j - 1, ldv)]));
    wj[threadIdx.x] = w0;
  }
  __syncthreads();
  const int64_t r = j + (int64_t)blockIdx.x * RB + threadIdx.x;
  double nrm = 0.0;
  if (r < n) {
    cplx c = A[IDX2(r, j, lda)];
    for (int q = 0; q < jj; ++q) {
      // c -= V(r,q) conj(W(j,q)) + W(r,q) conj(V(j,q))
      const cplx vr = V[IDX2(r, p + q, ldv)];
      cplx wr = W[IDX2(r, q, ldw)];
      if (fin && q == jj - 1) {
        wr = cadd(wr, cmul(falpha, V[IDX2(r, j - 1, ldv)]));
        if (r > j) W[IDX2(r, q, ldw)] = wr;
      }
      const cplx a = cmul(vr, cconj(wj[q])), b = cmul(wr, cconj(vj[q]));
      c = csub(c, cadd(a, b));
    }
    if (r == j) {
      c.y = 0.0;
      d[j] = c.x;
    }
    A[IDX2(r, j, lda)] = c;
    if (r >= j + 2) nrm = cabs2(c);
  }
  const double s = block_sum(nrm, red);
  if (threadIdx.x == 0) npart[blockIdx.x] = s;
}

// Reflector from alpha = x_0 and ||x_{1:}||^2: H^H x = beta e_1 with beta real,
// H = I - tau v v^H, v_0 = 1, v_{1:} = x_{1:} / (alpha - beta).
struct House {
  cplx tau, scal;
  double beta;
};
__device__ __forceinline__ House make_house(cplx alpha, double xnorm2) {
  House h;
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

// 2. reflector for column j, v written into V(:, j) (rows >= j+1)
__global__ void __launch_bounds__(RB) tr_house(int64_t n, int64_t j, const cplx* __restrict__ A, int64_t lda,
                                               cplx* __restrict__ V, int64_t ldv, cplx* __restrict__ tau,
                                               double* __restrict__ e, const double* __restrict__ npart, int nparts,
                                               const int64_t* status) {
  __shared__ House hs;
  if (*(volatile const int64_t*)status) return;
  if (threadIdx.x == 0) {
    double x2 = 0.0;
    for (int i = 0; i < nparts; ++i) x2 += npart[i];
    hs = make_house(A[IDX2(j + 1, j, lda)], x2);
    if (blockIdx.x == 0) {
      tau[j] = hs.tau;
      e[j] = hs.beta;
    }
  }
  __syncthreads();
  const int64_t r = j + 1 + (int64_t)blockIdx.x * RB + threadIdx.x;
  if (r < n) V[IDX2(r, j, ldv)] = (r == j + 1) ? mkc(1.0, 0.0) : cmul(A[IDX2(r, j, lda)], hs.scal);
}

// 3. y = A22 v from the lower triangle in tiles of 64 rows x 32 columns:
// each tile is read once and gives both its row sums (A v) and, below the
// diagonal, its column sums (A^H v).
constexpr int HT = 64;            // rows per tile
constexpr int HS = 32;            // columns per tile (strip width)
constexpr int HEMV_THREADS = 256;  // two CTAs per SM
// dynamic shared memory: two prefetch stages of one tile (each thread's 8
// entries, [u][thread]), the column-partial transpose T[32][65] and the
// double-buffered row partials rs[2][4][64]
constexpr int HEMV_STAGE = 8 * HEMV_THREADS;  // complex entries per stage
constexpr int HEMV_SMEM = (int)sizeof(cplx) * (2 * HEMV_STAGE + HS * (HT + 1) + 2 * 4 * HT);  // 107,008 bytes

__device__ __forceinline__ void hemv_cp16(uint32_t dst, const void* src, bool in) {
  // 16-byte copy to shared memory, L2 only; zero fill when `in` is false
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(in ? 16 : 0) : "memory");
}

// Work items: column strip bj (32 columns) and chunk ch of its row tiles,
// bi in [bj/2 + ch hr, min(ntr, bj/2 + (ch+1) hr)), hr = hemv_chunk(ntr); items
// are numbered strip by strip, so the longest come first and the last ones
// are the short strips near the end of the matrix.  The grid is two CTAs per
// SM (plus the dot CTAs) and each CTA takes items from a per-column counter
// until none is left, which balances the triangular work across the SMs.
// Thread (row r, column quarter q) handles 8 entries of its row per tile; the
// tile after the current one is prefetched with cp.async into shared memory
// (each thread copies, and later reads, only its own 8 entries, so the
// prefetch needs no barrier).  The row products of a tile go to slot bj (one
// writer per row, double-buffered so one barrier per tile suffices); the
// column products accumulate in registers over the item's tiles and, after
// one shared-memory reduction, go to slot nst + ch.  Per entry: two complex
// multiply-adds.  (Two CTAs of 8 warps per SM keep the FP64 pipe busier
// than one CTA of 16 warps with 64-wide strips.)
// The first `ndots` CTAs compute the panel dots s1 = W^H v and
// s2 = V_panel^H v (over rows >= j+1) beside the matvec (jj > 0).
__global__ void __launch_bounds__(HEMV_THREADS, 2)
    tr_hemv_strip(int64_t n, int64_t j, const cplx* __restrict__ A, int64_t lda, const cplx* __restrict__ V,
                  int64_t ldv, cplx* __restrict__ part, int64_t ldpart, int hr, int64_t p, int jj,
                  const cplx* __restrict__ W, int64_t ldw, cplx* __restrict__ s12, int ndots, int* __restrict__ counter,
                  const int64_t* status) {
  extern __shared__ __align__(16) unsigned char hsm[];
  cplx* stage = (cplx*)hsm;              // [2][8][HEMV_THREADS]
  cplx* T = stage + 2 * HEMV_STAGE;       // column partials, T[c * (HT + 1) + r]
  cplx* rs = T + HS * (HT + 1);           // [2][4][HT]
  __shared__ cplx vc[HS];
  __shared__ double red[32];
  __shared__ int item_s[2];  // strip, chunk of the CTA's current item
  if (*(volatile const int64_t*)status) return;
  const int64_t base = j + 1, m = n - base;
  const int nst = (int)((m + HS - 1) / HS), ntr = (int)((m + HT - 1) / HT);
  if ((int)blockIdx.x < ndots) {
    for (int d = blockIdx.x; d < 2 * jj; d += ndots) {
      const int q = d % jj, which = d / jj;  // which 0: W, 1: V
      const cplx* col = which == 0 ? W + IDX2(0, q, ldw) : V + IDX2(0, p + q, ldv);
      cplx acc = mkc(0.0, 0.0);
      for (int64_t r = j + 1 + threadIdx.x; r < n; r += blockDim.x) cfma_cj(acc, col[r], V[IDX2(r, j, ldv)]);
      const cplx sv = block_sum_c(acc, red);
      if (threadIdx.x == 0) s12[which * NBT + q] = sv;
      __syncthreads();
    }
    return;
  }
  const int tid = threadIdx.x, r = tid & 63, q = tid >> 6;  // row, column quarter
  const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(stage);
  int cur_b = 0, cur_acc = 0;  // thread 0's decode cursor: items come in increasing order
  for (;;) {
    if (tid == 0) {
      // decode the next item (one thread, 32-bit arithmetic), continuing the
      // scan over the strips from the previous item
      const int item = atomicAdd(counter, 1);
      int c = 0;
      for (; cur_b < nst; ++cur_b) {
        const int nc = (ntr - (cur_b >> 1) + hr - 1) / hr;
        if (item < cur_acc + nc) {
          c = item - cur_acc;
          break;
        }
        cur_acc += nc;
      }
      item_s[0] = cur_b;
      item_s[1] = c;
    }
    __syncthreads();
    const int bj = item_s[0], ch = item_s[1];
    if (bj >= nst) break;  // uniform: every thread reads the same item
    const int bi0 = (bj >> 1) + ch * hr, bi1 = bi0 + hr < ntr ? bi0 + hr : ntr;
    const int64_t c0 = (int64_t)bj * HS;
    auto prefetch = [&](int bi, int st) {
      const int64_t gr = (int64_t)bi * HT + r;
      const cplx* Ar = A + IDX2(base + gr, base + c0, lda);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t gc = c0 + q * 8 + u;
        const bool in = gr < m && gc < m && gr >= gc;
        hemv_cp16(stage_s + (uint32_t)sizeof(cplx) * (st * HEMV_STAGE + u * HEMV_THREADS + tid),
                  in ? (const void*)(Ar + (int64_t)(q * 8 + u) * lda) : (const void*)A, in);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    if (tid < HS) vc[tid] = (c0 + tid < m) ? V[IDX2(base + c0 + tid, j, ldv)] : mkc(0.0, 0.0);
    prefetch(bi0, 0);
    __syncthreads();
    cplx colacc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) colacc[u] = mkc(0.0, 0.0);
    int t = 0;
    for (int bi = bi0; bi < bi1; ++bi, ++t) {
      if (bi + 1 < bi1) {
        prefetch(bi + 1, (t + 1) & 1);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
      const int64_t r0 = (int64_t)bi * HT, gr = r0 + r;
      const cplx vrr = gr < m ? V[IDX2(base + gr, j, ldv)] : mkc(0.0, 0.0);
      const cplx* sb = stage + (t & 1) * HEMV_STAGE + tid;
      cplx av[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = sb[u * HEMV_THREADS];
      cplx ra0 = mkc(0.0, 0.0), ra1 = mkc(0.0, 0.0);  // two chains of row products
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = q * 8 + u;
        cfma((u & 1) ? ra1 : ra0, av[u], vc[c]);
        if (gr > c0 + c) cfma_cj(colacc[u], av[u], vrr);
      }
      cplx* rsb = rs + (t & 1) * 4 * HT;
      rsb[q * HT + r] = cadd(ra0, ra1);
      __syncthreads();
      if (tid < HT && r0 + tid < m) {
        const cplx y = cadd(cadd(rsb[tid], rsb[HT + tid]), cadd(rsb[2 * HT + tid], rsb[3 * HT + tid]));
        part[r0 + tid + (int64_t)bj * ldpart] = y;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) T[(q * 8 + u) * (HT + 1) + r] = colacc[u];
    __syncthreads();
    {
      // column c: thread (c, eighth e) adds rows e*8 .. e*8+7, then the 8 eighths
      const int c = tid & 31, e = tid >> 5;
      cplx acc = mkc(0.0, 0.0);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = cadd(acc, T[c * (HT + 1) + e * 8 + u]);
      rs[e * HS + c] = acc;
    }
    __syncthreads();
    if (tid < HS && c0 + tid < m) {
      cplx y = rs[tid];
#pragma unroll
      for (int e = 1; e < 8; ++e) y = cadd(y, rs[e * HS + tid]);
      part[c0 + tid + (int64_t)(nst + ch) * ldpart] = y;
    }
    __syncthreads();
  }
}

// 3d. w = tau (y - V s1 - W s2), stored in W(:, jj); partial sums of w^H v.
// 64 rows per CTA, 4 threads per row (slots and panel columns split 4 ways).
constexpr int AR = 64;

__global__ void __launch_bounds__(256) tr_w_assemble(int64_t n, int64_t p, int64_t j, const cplx* __restrict__ V,
                                                     int64_t ldv, cplx* __restrict__ W, int64_t ldw,
                                                     const cplx* __restrict__ part, int64_t ldpart, int nch, int hr,
                                                     const cplx* __restrict__ s12, const cplx* __restrict__ tau,
                                                     double* __restrict__ dpart, const int64_t* status) {
  __shared__ cplx s1[NBT], s2[NBT];
  __shared__ cplx red4[4][AR];
  __shared__ double red[32];
  if (*(volatile const int64_t*)status) return;
  const int jj = (int)(j - p);
  if (threadIdx.x < jj) {
    s1[threadIdx.x] = s12[threadIdx.x];
    s2[threadIdx.x] = s12[NBT + threadIdx.x];
  }
  __syncthreads();
  const int64_t base = j + 1, m = n - base;
  const int rl = threadIdx.x & (AR - 1), qq = threadIdx.x / AR;
  const int64_t r = (int64_t)blockIdx.x * AR + rl;
  cplx y = mkc(0.0, 0.0);
  if (r < m) {
    // row products of the strips 0 .. 2 bi + 1 that meet row tile bi, column
    // products of the chunks of the row's own strip b (nch strips, their
    // row tiles in chunks of hr)
    const int bi = (int)(r / HT), b = (int)(r / HS);
    const int ntr = (nch + 1) / 2;
    const int last = 2 * bi + 1 < nch - 1 ? 2 * bi + 1 : nch - 1;
    const int nchk = (ntr - (b >> 1) + hr - 1) / hr;
    for (int c = qq; c <= last; c += 4) y = cadd(y, part[r + c * ldpart]);
    for (int c = qq; c < nchk; c += 4) y = cadd(y, part[r + (nch + c) * ldpart]);
    const int64_t gr = base + r;
    for (int q = qq; q < jj; q += 4) {
      y = csub(y, cmul(V[IDX2(gr, p + q, ldv)], s1[q]));
      y = csub(y, cmul(W[IDX2(gr, q, ldw)], s2[q]));
    }
  }
  red4[qq][rl] = y;
  __syncthreads();
  cplx dot = mkc(0.0, 0.0);
  if (qq == 0 && r < m) {
    y = cadd(cadd(red4[0][rl], red4[1][rl]), cadd(red4[2][rl], red4[3][rl]));
    y = cmul(tau[j], y);
    const int64_t gr = base + r;
    W[IDX2(gr, jj, ldw)] = y;
    dot = cmul(cconj(y), V[IDX2(gr, j, ldv)]);
  }
  const cplx sdot = block_sum_c(dot, red);
  if (threadIdx.x == 0) {
    dpart[2 * blockIdx.x] = sdot.x;
    dpart[2 * blockIdx.x + 1] = sdot.y;
  }
}

// 4. w += -tau/2 (w^H v) v
__global__ void __launch_bounds__(RB) tr_w_finish(int64_t n, int64_t p, int64_t j, const cplx* __restrict__ V,
                                                  int64_t ldv, cplx* __restrict__ W, int64_t ldw,
                                                  const cplx* __restrict__ tau, const double* __restrict__ dpart,
                                                  int nparts, const int64_t* status) {
  __shared__ cplx alpha;
  if (*(volatile const int64_t*)status) return;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nparts; ++i) a += dpart[2 * i], b += dpart[2 * i + 1];
    alpha = cscale(cmul(tau[j], mkc(a, b)), -0.5);
  }
  __syncthreads();
  const int jj = (int)(j - p);
  const int64_t r = j + 1 + (int64_t)blockIdx.x * RB + threadIdx.x;
  if (r < n) W[IDX2(r, jj, ldw)] = cadd(W[IDX2(r, jj, ldw)], cmul(alpha, V[IDX2(r, j, ldv)]));
}

__global__ void tr_last_diag(int64_t n, const cplx* A, int64_t lda, double* d, const int64_t* status) {
  if (*(volatile const int64_t*)status) return;
  d[n - 1] = A[IDX2(n - 1, n - 1, lda)].x;
}

#define LAUNCH(kern, grid, blk, ...)                 \
  do {                                               \
    prof_launch_begin(s);                            \
    kern<<<(grid), (blk), 0, s>>>(__VA_ARGS__);      \
    prof_launch_end(s, #kern);                       \
    bse_count_launch();                              \
    BSE_LAUNCH_CHECK();                              \
  } while (0)

bse_status hetrd_lower(cudaStream_t s, int64_t n, cplx* A, int64_t lda, const HetrdWork& w,
                       const int64_t* status) {
  if (n <= 0) return BSE_OK;
  {
    const bse_status r = set_smem_attr((const void*)tr_hemv_strip, HEMV_SMEM);
    if (r) return r;
  }
  const int64_t ldv = n, ldw = n;
  BSE_CUDA(cudaMemsetAsync(w.V, 0, sizeof(cplx) * n * n, s));
  const int64_t ldpart = n + 1;
  cplx* part = w.part;  // hemv_slots(n) columns of length ldpart
  const int64_t slots = hemv_slots(n);
  double* npart = (double*)(w.part + slots * ldpart);
  double* dpart = npart + (n / RB + 2);
  int* counters = (int*)(dpart + 2 * (n / AR + 4));  // one work-queue counter per column
  BSE_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * n, s));
  const int64_t sms = device_sms();
  cplx* s12 = w.small;
  const cplx one = mkc(1.0, 0.0), mone = mkc(-1.0, 0.0);
  for (int64_t p = 0; p < n - 1; p += NBT) {
    const int64_t bs = (n - 1 - p) < NBT ? (n - 1 - p) : NBT;
    int nfin = 0;  // partial sums of the previous column's w^H v still to fold in
    for (int64_t j = p; j < p + bs; ++j) {
      const int64_t m = n - j - 1;  // length of the reflector
      const unsigned g1 = ceil_div_u(n - j, RB);
      LAUNCH(tr_col_update, g1, RB, n, p, j, A, lda, w.V, ldv, w.W, ldw, w.d, npart, dpart, nfin, w.tau, status);
      const unsigned g2 = ceil_div_u(m, RB);
      LAUNCH(tr_house, g2, RB, n, j, A, lda, w.V, ldv, w.tau, w.e, npart, (int)g1, status);
      const int64_t nst = (m + HS - 1) / HS, ntr = (m + HT - 1) / HT;  // strips, row tiles
      const int hr = hemv_chunk(ntr);
      {
        prof_launch_begin(s);
        const int jj = (int)(j - p);
        int64_t nitems = 0;
        for (int64_t bj = 0; bj < nst; ++bj) nitems += (ntr - bj / 2 + hr - 1) / hr;
        const int ndots = jj > 0 ? (2 * jj < 16 ? 2 * jj : 16) : 0;
        const unsigned hg = (unsigned)(ndots + (nitems < 2 * sms ? nitems : 2 * sms));
        tr_hemv_strip<<<hg, HEMV_THREADS, HEMV_SMEM, s>>>(n, j, A, lda, w.V, ldv, part, ldpart, hr, p, jj, w.W, ldw,
                                                           s12, ndots, counters + j, status);
        prof_launch_end(s, "tr_hemv_strip");
        bse_count_launch();
        BSE_LAUNCH_CHECK();
      }
      const unsigned ga = ceil_div_u(m, AR);
      LAUNCH(tr_w_assemble, ga, 256, n, p, j, w.V, ldv, w.W, ldw, part, ldpart, (int)nst, hr, s12, w.tau, dpart,
             status);
      if (j + 1 < p + bs) {
        nfin = (int)ga;  // the next column update finishes this w
      } else {
        LAUNCH(tr_w_finish, g2, RB, n, p, j, w.V, ldv, w.W, ldw, w.tau, dpart, (int)ga, status);
      }
    }
    const int64_t t0 = p + bs, mt = n - t0;
    if (mt > 0 && p + 2 * bs <= n) {
      // A22 -= V W^H + W V^H as ONE product of depth 2 bs: [W V_p] [V_p W]^H,
      // with W parked in the (still zero) columns p+bs .. p+2bs-1 of V for the
      // second operand and [W V_p] assembled in S2; the parked columns are
      // zeroed again before the next panel writes its reflectors there
      cplx* A22 = A + IDX2(t0, t0, lda);
      const size_t rowb = sizeof(cplx) * (size_t)mt;
      BSE_CUDA(cudaMemcpy2DAsync(w.V + IDX2(t0, p + bs, ldv), sizeof(cplx) * ldv, w.W + IDX2(t0, 0, ldw),
                                 sizeof(cplx) * ldw, rowb, bs, cudaMemcpyDeviceToDevice, s));
      BSE_CUDA(cudaMemcpy2DAsync(w.S2, sizeof(cplx) * n, w.W + IDX2(t0, 0, ldw), sizeof(cplx) * ldw, rowb, bs,
                                 cudaMemcpyDeviceToDevice, s));
      BSE_CUDA(cudaMemcpy2DAsync(w.S2 + IDX2(0, bs, n), sizeof(cplx) * n, w.V + IDX2(t0, p, ldv), sizeof(cplx) * ldv,
                                 rowb, bs, cudaMemcpyDeviceToDevice, s));
      GemmParams<cplx> g = gemm_params<cplx>(mt, mt, 2 * bs, OPN, w.S2, n, OPC, w.V + IDX2(t0, p, ldv), ldv, mone,
                                             one, A22, lda);
      g.lowerC = 1;
      g.status = status;
      bse_status r = gemm_z(s, g);
      if (r) return r;
      BSE_CUDA(cudaMemset2DAsync(w.V + IDX2(t0, p + bs, ldv), sizeof(cplx) * ldv, 0, rowb, bs, s));
    } else if (mt > 0) {
      // A22 -= V W^H + W V^H  (lower triangle of rows/cols >= t0)
      cplx* A22 = A + IDX2(t0, t0, lda);
      GemmParams<cplx> g1 = gemm_params<cplx>(mt, mt, bs, OPN, w.V + IDX2(t0, p, ldv), ldv, OPC,
                                              w.W + IDX2(t0, 0, ldw), ldw, mone, one, A22, lda);
      g1.lowerC = 1;
      g1.status = status;
      bse_status r = gemm_z(s, g1);
      if (r) return r;
      GemmParams<cplx> g2p = gemm_params<cplx>(mt, mt, bs, OPN, w.W + IDX2(t0, 0, ldw), ldw, OPC,
                                               w.V + IDX2(t0, p, ldv), ldv, mone, one, A22, lda);
      g2p.lowerC = 1;
      g2p.status = status;
      r = gemm_z(s, g2p);
      if (r) return r;
    }
  }
  LAUNCH(tr_last_diag, 1, 1, n, A, lda, w.d, status);
  return BSE_OK;
}

// ---------------------------------------------------------------------------
// Block reflector application (columnwise, forward order):
//   H_c0 ... H_{c0+bs-1} = I - Vp T Vp^H,  T upper triangular with
//   T(i,i) = tau_i,  T(0:i, i) = -tau_i T(0:i, 0:i) (Vp(:, 0:i)^H v_i).
__global__ void larft_kernel(int bs, const cplx* __restrict__ G, int ldg, const cplx* __restrict__ tau,
                             cplx* __restrict__ T, int ldt, const int64_t* status) {
  if (*(volatile const int64_t*)status) return;
  const int r = threadIdx.x;
  for (int e = r; e < bs * bs; e += blockDim.x) T[(e % bs) + (e / bs) * ldt] = mkc(0.0, 0.0);
  __syncthreads();
  for (int i = 0; i < bs; ++i) {
    if (r < i) {
      cplx acc = mkc(0.0, 0.0);
      for (int q = r; q < i; ++q) cfma(acc, T[r + q * ldt], G[q + i * ldg]);
      T[r + i * ldt] = cmul(cscale(tau[i], -1.0), acc);
    } else if (r == i) {
      T[i + i * ldt] = tau[i];
    }
    __syncthreads();
  }
}

// out[e] = sum of the nl layers of `len` elements
__global__ void sum_layers_kernel(int64_t len, int nl, const cplx* __restrict__ layers, cplx* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= len) return;
  cplx acc = layers[e];
  for (int z = 1; z < nl; ++z) acc = cadd(acc, layers[e + z * len]);
  out[e] = acc;
}

bse_status apply_block_reflector(cudaStream_t s, int64_t n, int64_t k, const cplx* Vbuf, int64_t ldvb, int64_t c0,
                                 int64_t bs, int64_t r0, const cplx* tau, cplx* Vout, int64_t ldv, cplx* tmp,
                                 const int64_t* status) {
  if (bs <= 0 || k <= 0 || r0 >= n) return BSE_OK;
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0), mone = mkc(-1.0, 0.0);
  const int64_t m = n - r0;
  const cplx* Vp = Vbuf + IDX2(r0, c0, ldvb);
  cplx* G = tmp;                 // bs x bs
  cplx* T = G + bs * bs;         // bs x bs
  cplx* W1 = T + bs * bs;        // bs x k
  cplx* W2 = W1 + bs * k;        // bs x k
  cplx* Gl = W2 + bs * k;        // GSPLIT layers of bs x bs
  // G = V^H V: a bs x bs output over the m rows of the block; as one GEMM it
  // would run on (bs/64)^2 = 4 CTAs, so the k range is split into up to
  // GSPLIT layers (DFMA engine, both precisions: it is ~0.1% of the flops)
  // and the layers are added
  const int64_t kc = ((m + GSPLIT - 1) / GSPLIT + 63) / 64 * 64;
  const int nl = (int)((m + kc - 1) / kc);
  GemmParams<cplx> pg = gemm_params<cplx>(bs, bs, m, OPC, Vp, ldvb, OPN, Vp, ldvb, one, zero, Gl, bs);
  pg.status = status;
  pg.kchunk = kc;
  pg.cstride = bs * bs;
  bse_status r = gemm_z(s, pg);
  if (r) return r;
  sum_layers_kernel<<<ceil_div_u(bs * bs, 256), 256, 0, s>>>(bs * bs, nl, Gl, G);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  const int lt = (int)((bs + 31) / 32 * 32);
  larft_kernel<<<1, lt, 0, s>>>((int)bs, G, (int)bs, tau + c0, T, (int)bs, status);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  GemmParams<cplx> p1 = gemm_params<cplx>(bs, k, m, OPC, Vp, ldvb, OPN, Vout + r0, ldv, one, zero, W1, bs);
  p1.status = status;
  // W1 = V^H Z is a thin output of depth m: split k so that the tiles fill
  // whole waves -- (bs/64) x (k/64) tiles over 2 CTAs per SM on the DFMA
  // engine, (bs/128) x (2k/64) tiles over the persistent tensor-core
  // engine's one CTA per SM
  const OzWork oz = oz_current();
  const bool on_tc = oz.ptr && oz.engine == OZ_ENGINE_TCGEN05 && (double)bs * k * m >= (double)oz.min_mnk;
  const int ws = on_tc ? split_layers(((bs + 127) / 128) * ((2 * k + 63) / 64), device_sms())
                       : split_layers(((bs + 63) / 64) * ((k + 63) / 64), 2 * device_sms());
  if (ws > 1 && m >= 64 * ws) {
    cplx* Wl = Gl + (size_t)GSPLIT * bs * bs;  // ws layers of bs x k
    p1.C = Wl;
    p1.kchunk = ((m + ws - 1) / ws + 63) / 64 * 64;
    p1.cstride = bs * k;
    if ((r = gemm_z(s, p1))) return r;
    const int nl = (int)((m + p1.kchunk - 1) / p1.kchunk);
    sum_layers_kernel<<<ceil_div_u(bs * k, 256), 256, 0, s>>>(bs * k, nl, Wl, W1);
    bse_count_launch();
    BSE_LAUNCH_CHECK();
  } else if ((r = gemm_z(s, p1))) {
    return r;
  }
  GemmParams<cplx> p2 = gemm_params<cplx>(bs, k, bs, OPN, T, bs, OPN, W1, bs, one, zero, W2, bs);
  p2.triA = TRI_UP;
  p2.status = status;
  if ((r = gemm_z(s, p2))) return r;
  GemmParams<cplx> p3 = gemm_params<cplx>(m, k, bs, OPN, Vp, ldvb, OPN, W2, bs, mone, one, Vout + r0, ldv);
  p3.status = status;
  return gemm_z(s, p3);
}

bse_status hetrd_backtransform(cudaStream_t s, int64_t n, int64_t k, const HetrdWork& w, cplx* Vout, int64_t ldv,
                               cplx* tmp, const int64_t* status) {
  if (n <= 1) return BSE_OK;
  const int64_t npan = (n - 1 + BTB - 1) / BTB;
  for (int64_t b = npan - 1; b >= 0; --b) {
    const int64_t p = b * BTB;
    const int64_t bs = (n - 1 - p) < BTB ? (n - 1 - p) : BTB;
    bse_status r = apply_block_reflector(s, n, k, w.V, n, p, bs, p + 1, w.tau, Vout, ldv, tmp, status);
    if (r) return r;
  }
  return BSE_OK;
}
