// FP64-accurate complex GEMM on the BF16 tensor cores by exact operand
// splitting (the Ozaki scheme): C = alpha op(A) op(B) + beta C, the same
// contract as the DFMA engine (triangular operands, lower-only output, the
// fused X/Y epilogue), for the large products of the solver.
//
// Complex operands enter as their real 2x2 embedding, interleaved so that a
// lane's accumulator pair (c0, c1) is (Re, Im) of one complex entry:
//   A'(i, 2kk) = Re a(i,kk),  A'(i, 2kk+1) = Im a(i,kk)
//   B''(2kk, 2j) = Re b,  B''(2kk+1, 2j) = -Im b,  B''(2kk, 2j+1) = Im b,  B''(2kk+1, 2j+1) = Re b
// so Re c(i,j) = C'(i, 2j) and Im c(i,j) = C'(i, 2j+1) with C' = A' B''.
//
// Splitting (per row of A', per column pair of B''): with 2^e the smallest
// power of two above the row's (column's) largest |Re|, |Im|, every entry
// v = 2^e sum_{t=1..S} 2^{-7t} q_t with integers |q_1| <= 128, |q_t| <= 64
// (round to nearest at each step, exact in FP64).  Slice t is stored as the
// BF16 number q_t 2^{-7(t-1)} -- exact (<= 8 significant bits).  The product
// keeps the pairs t + u <= S + 1; a pair's BF16 products at level l = t + u
// carry the common factor 2^{-7(l-2)}, so the FP32 tensor-core accumulation
// of one level is exact while its integer partial sum stays below 2^24
// (guaranteed for 512 consecutive k' at every level).  Levels 2..6 therefore
// accumulate separately and exactly and are added into FP64 accumulators
// every 512 k'; levels >= 7 share one FP32 accumulator (their rounding is
// below 2^-53 of the result).  The dropped pairs (t + u > S + 1) are below
// 2^-7S of the row/column scale, the same order as FP64 rounding for S = 8.
#include <cuda.h>
#include <stdint.h>

#include <atomic>

#include "kernels.cuh"
#include "prof.cuh"

namespace {

constexpr int OZ_BM = 64, OZ_BN = 64, OZ_BK = 32;  // real rows, real cols, real k per tile
constexpr int OZ_ROWB = 80;                          // smem bytes per tile row (64 data + 16 pad)
constexpr int OZ_FOLD = 16;                          // k-tiles per FP64 fold (512 k')
constexpr int OZ_NSETS = 6;                          // levels 2..6 separate, >= 7 combined

__device__ __forceinline__ uint16_t bf16_bits_exact(float v) {
  // v has <= 8 significant bits: truncation of the FP32 encoding is exact
  return (uint16_t)(__float_as_uint(v) >> 16);
}

// Slices of v (|v| < 2^e): v 2^(7 - e) = sum_t q_t 2^(-7(t-1)) with integers
// |q_1| <= 128, |q_t| <= 64 (t >= 2), each digit rounded to nearest in turn
// and the tail below the last digit rounded, returned as the exact FP32 (and
// BF16) numbers q_t 2^(-7(t-1)).  Integer arithmetic on the bit pattern only:
// FP64 is the slowest unit of this part.  A NaN or Inf entry gives NaN slices.
__device__ __forceinline__ void split_value(double v, int e, int S, float* out) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef == 0x7FF) {
    for (int t = 0; t < S; ++t) out[t] = __int_as_float(0x7FC00000);
    return;
  }
  uint64_t M = b & 0xFFFFFFFFFFFFFull;  // v = +-M 2^E
  const int E = ef ? ef - 1075 : -1074;
  if (ef) M |= 1ull << 52;
  // R = round(|v| 2^(7S - e)): the digits' common integer scale; sh <= 7S - 53
  // because M < 2^53 and M 2^E < 2^e
  const int sh = E + 7 * S - e;
  int64_t R = 0;
  if (M && sh > -64) R = sh >= 0 ? (int64_t)(M << sh) : (int64_t)((M + (1ull << (-sh - 1))) >> (-sh));
  if (b >> 63) R = -R;
  for (int t = 0; t < S - 1; ++t) {
    const int sd = 7 * (S - 1 - t);
    const int64_t q = (R + (1ll << (sd - 1))) >> sd;  // nearest (ties up)
    R -= q * (1ll << sd);
    out[t] = (float)(int)q * __int_as_float((127 - 7 * t) << 23);
  }
  out[S - 1] = (float)(int)R * __int_as_float((127 - 7 * (S - 1)) << 23);
}

// frexp exponent of x (|x| = m 2^e, 1/2 <= m < 1) from its bit pattern; -4096 for 0
__device__ __forceinline__ int fexp_bits(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0) return -4096;
  const int ef = (int)(b >> 52);
  return ef ? ef - 1022 : -1010 - __clzll((long long)b);
}

// ---- scales -----------------------------------------------------------------
// ea[i] = 2048 + e_i for row i of op(A) (0 = all-zero row); fb[j] likewise for
// column j of op(B).  Logical element (r, c) of op(X) with triangular mask.
__device__ __forceinline__ bool op_elem(const cplx* X, int64_t ldx, int op, int tri, int64_t r, int64_t c,
                                        int64_t R, int64_t C, cplx* out) {
  if (r >= R || c >= C) return false;
  if (tri == TRI_LO && c > r) return false;
  if (tri == TRI_UP && c < r) return false;
  cplx v = (op == OPN) ? X[r + c * ldx] : X[c + r * ldx];
  if (op == OPC) v = cconj(v);
  *out = v;
  return true;
}

// rows of op(A) (m x k): one warp per row chunk; atomicMax on biased exponents
__global__ void oz_rowexp_kernel(int64_t m, int64_t k, const cplx* A, int64_t lda, int op, int tri, int* ea) {
  // tile of 32 rows x 32 columns, coalesced along the stored leading dimension
  __shared__ int mx[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int q = ty; q < 32; q += 8) {
    int64_t r, c;
    if (op == OPN) r = r0 + tx, c = c0 + q;  // consecutive tx -> consecutive rows (stored contiguous)
    else r = r0 + q, c = c0 + tx;
    cplx v;
    int a = -4096;
    if (op_elem(A, lda, op, tri, r, c, m, k, &v)) a = max(fexp_bits(v.x), fexp_bits(v.y));
    if (op == OPN) mx[tx][q] = a; else mx[q][tx] = a;
  }
  __syncthreads();
  if (ty == 0) {
    int a = -4096;
    for (int q = 0; q < 32; ++q) a = max(a, mx[tx][q]);
    if (a > -4096 && r0 + tx < m) atomicMax(ea + r0 + tx, 2048 + a);
  }
}

__global__ void oz_colexp_kernel(int64_t k, int64_t n, const cplx* B, int64_t ldb, int op, int tri, int* fb) {
  __shared__ int mx[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;  // c: column j of op(B), r: kk
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    int64_t r, c;
    if (op == OPN) r = r0 + tx, c = c0 + q;  // op(B) = B: rows kk contiguous
    else r = r0 + q, c = c0 + tx;
    cplx v;
    int a = -4096;
    if (op_elem(B, ldb, op, tri, r, c, k, n, &v)) a = max(fexp_bits(v.x), fexp_bits(v.y));
    if (op == OPN) mx[q][tx] = a; else mx[tx][q] = a;  // mx[col][row]
  }
  __syncthreads();
  if (ty == 0) {
    int a = -4096;
    for (int q = 0; q < 32; ++q) a = max(a, mx[tx][q]);
    if (a > -4096 && c0 + tx < n) atomicMax(fb + c0 + tx, 2048 + a);
  }
}

// ---- slices -----------------------------------------------------------------
// As: [S][Mp][Kp] bf16 (Kp = padded 2k, row-major, k' contiguous); every entry
// of the padded extent is written (zeros outside op(A) and its triangle).
template <int S>
__global__ void oz_split_a_kernel(int64_t m, int64_t k, const cplx* A, int64_t lda, int op, int tri, const int* ea,
                                  int64_t Mp, int64_t Kp, uint32_t* As) {
  __shared__ cplx tile[32][33];  // tile[row][kk]
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    int64_t r, c;
    if (op == OPN) r = r0 + tx, c = c0 + q;
    else r = r0 + q, c = c0 + tx;
    cplx v = mkc(0.0, 0.0);
    op_elem(A, lda, op, tri, r, c, m, k, &v);
    if (op == OPN) tile[tx][q] = v; else tile[q][tx] = v;
  }
  __syncthreads();
  const int64_t Kc = Kp / 2;  // complex columns of the padded extent
  for (int q = ty; q < 32; q += 8) {
    const int64_t r = r0 + q, c = c0 + tx;  // write along kk (contiguous)
    if (r >= Mp || c >= Kc) continue;
    const cplx v = tile[q][tx];
    const int eb = (r < m) ? ea[r] : 0;
    float sr[S], si[S];
    const int e = eb ? eb - 2048 : 0;
    split_value(v.x, e, S, sr);
    split_value(v.y, e, S, si);
    for (int t = 0; t < S; ++t) {
      const uint32_t w = (uint32_t)bf16_bits_exact(sr[t]) | ((uint32_t)bf16_bits_exact(si[t]) << 16);
      As[((int64_t)t * Mp + r) * Kc + c] = w;  // (k' = 2c, 2c+1)
    }
  }
}

// Bs: [S][Np][Kp] bf16 with Np = padded 2n; column j of op(B) gives rows 2j
// (Re b, -Im b) and 2j+1 (Im b, Re b) at k' = 2kk, 2kk+1.
template <int S>
__global__ void oz_split_b_kernel(int64_t k, int64_t n, const cplx* B, int64_t ldb, int op, int tri, const int* fb,
                                  int64_t Np, int64_t Kp, uint32_t* Bs) {
  __shared__ cplx tile[32][33];  // tile[j][kk]
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;  // j, kk
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    int64_t r, c;
    if (op == OPN) r = r0 + tx, c = c0 + q;
    else r = r0 + q, c = c0 + tx;
    cplx v = mkc(0.0, 0.0);
    op_elem(B, ldb, op, tri, r, c, k, n, &v);
    if (op == OPN) tile[q][tx] = v; else tile[tx][q] = v;  // tile[j][kk]
  }
  __syncthreads();
  const int64_t Kc = Kp / 2, Nc = Np / 2;
  for (int q = ty; q < 32; q += 8) {
    const int64_t j = c0 + q, kk = r0 + tx;
    if (j >= Nc || kk >= Kc) continue;
    const cplx v = tile[q][tx];
    const int eb = (j < n) ? fb[j] : 0;
    float sr[S], si[S];
    const int e = eb ? eb - 2048 : 0;
    split_value(v.x, e, S, sr);
    split_value(v.y, e, S, si);
    for (int t = 0; t < S; ++t) {
      const uint32_t w0 = (uint32_t)bf16_bits_exact(sr[t]) | ((uint32_t)bf16_bits_exact(-si[t]) << 16);
      const uint32_t w1 = (uint32_t)bf16_bits_exact(si[t]) | ((uint32_t)bf16_bits_exact(sr[t]) << 16);
      Bs[((int64_t)t * Np + 2 * j) * Kc + kk] = w0;
      Bs[((int64_t)t * Np + 2 * j + 1) * Kc + kk] = w1;
    }
  }
}

// ---- the tensor-core product -------------------------------------------------
template <typename T>
struct OzArgs {
  GemmParams<T> p;
  const uint32_t* As;
  const uint32_t* Bs;
  const int* ea;
  const int* fb;
  int64_t Mp, Np, Kp;
  long long wait;       // tcgen05 engine: limit of its pipeline waits (cycles)
  int64_t ncols_real;   // tcgen05 engine: real output columns (a multiple of 64)
};

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// not volatile: ordered by its data dependences only, so the scheduler can
// overlap the next ldmatrix with the MMAs in flight
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// T = cplx: complex product through the real 2x2 embedding (k' = 2k, two
// real columns per complex column); T = double: real product (k' = k).
template <int S, typename T>
__global__ void __launch_bounds__(256, 1) oz_mma_kernel(const OzArgs<T> z) {
  extern __shared__ __align__(128) unsigned char osm[];
  constexpr bool CPLX = sizeof(T) == sizeof(cplx);
  constexpr int XF = CPLX ? 2 : 1;  // real rows/cols of k' and n' per logical index
  const GemmParams<T>& p = z.p;
  // grouped rasterisation: consecutive CTAs walk down groups of 8 tile rows so
  // that the slices of 8 row panels and of a few column panels stay in L2
  const int64_t gx = gridDim.x, gy = gridDim.y;
  const int64_t lin = (int64_t)blockIdx.x + (int64_t)blockIdx.y * gx;
  const int64_t grp = lin / (8 * gx), first = grp * 8;
  const int64_t rows = (gy - first) < 8 ? (gy - first) : 8;
  const int64_t loc = lin % (8 * gx);
  const int64_t ty = first + loc % rows, tx = loc / rows;
  const int64_t i0 = ty * OZ_BM;                         // real rows = complex rows
  const int64_t jr0 = tx * OZ_BN;                        // real columns
  const int64_t jc0 = jr0 / XF;                          // logical columns
  if (i0 >= p.m || jc0 >= p.n) return;
  if (p.lowerC && jc0 > i0 + OZ_BM - 1) return;
  if (p.status && *(volatile const int64_t*)p.status) return;
  // k-range from the triangular structure (complex), then real k' tiles
  int64_t kb = 0, ke = p.k;
  if (p.triA == TRI_LO) ke = min(ke, i0 + OZ_BM);
  if (p.triA == TRI_UP) kb = max(kb, i0);
  if (p.triB == TRI_LO) kb = max(kb, jc0);
  if (p.triB == TRI_UP) ke = min(ke, jc0 + OZ_BN / XF);
  int64_t kb2 = (XF * kb / OZ_BK) * OZ_BK, ke2 = XF * ke;
  const int64_t ntile = ke2 > kb2 ? (ke2 - kb2 + OZ_BK - 1) / OZ_BK : 0;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, warp tile 32 x 16
  const int g = lane >> 2, tg = lane & 3;

  constexpr int SLICE_BYTES = OZ_BM * OZ_ROWB;           // 64 rows x 80 B
  constexpr int STAGE_BYTES = 2 * S * SLICE_BYTES;       // A and B
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(osm);
  const int64_t Kc = z.Kp / 2;  // 32-bit words per slice row

  auto issue = [&](int64_t kt, int stage) {
    const int64_t kw = (kb2 + kt * OZ_BK) / 2;  // word offset of the tile in a row
    const uint32_t st = sbase + stage * STAGE_BYTES;
    // A: S slices x 64 rows x 4 chunks; B: S x 64 x 4
    for (int c = tid; c < 2 * S * 256; c += 256) {
      const int which = c / (S * 256);
      const int rem = c % (S * 256);
      const int t = rem / 256, row = (rem % 256) / 4, ch = rem % 4;
      const uint32_t* src;
      if (which == 0) src = z.As + ((int64_t)t * z.Mp + i0 + row) * Kc + kw + ch * 4;
      else src = z.Bs + ((int64_t)t * z.Np + jr0 + row) * Kc + kw + ch * 4;
      const uint32_t dst = st + (which * S + t) * SLICE_BYTES + row * OZ_ROWB + ch * 16;
      cp_async16(dst, src);
    }
  };

  double acc64[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc64[q] = 0.0;
  float acc[OZ_NSETS][16];
#pragma unroll
  for (int s = 0; s < OZ_NSETS; ++s)
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[s][q] = 0.f;

  if (ntile > 0) {
    issue(0, 0);
    cp_commit();
  }
  for (int64_t kt = 0; kt < ntile; ++kt) {
    const int stage = (int)(kt & 1);
    if (kt + 1 < ntile) issue(kt + 1, stage ^ 1);
    cp_commit();
    cp_wait1();
    __syncthreads();
    const uint32_t st = sbase + stage * STAGE_BYTES;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
      for (int t = 0; t < S; ++t) {
        uint32_t a[2][4];
        const uint32_t abase = st + t * SLICE_BYTES;
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
          const int row = wm * 32 + mi * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
          const int col = ks * 16 + (lane >> 4) * 8;  // bf16 index
          ldsm_x4(abase + row * OZ_ROWB + col * 2, a[mi][0], a[mi][1], a[mi][2], a[mi][3]);
        }
        const int nrow = wn * 16 + (lane & 7) + (lane >> 4) * 8;
        const int kcol = ks * 16 + ((lane >> 3) & 1) * 8;
        const uint32_t boff = nrow * OZ_ROWB + kcol * 2;
        uint32_t bc[4], bn[4];
        ldsm_x4(st + S * SLICE_BYTES + boff, bc[0], bc[1], bc[2], bc[3]);
#pragma unroll
        for (int u = 0; u < S - t; ++u) {  // u index 0-based: level (t+1)+(u+1) = t + u + 2 <= S + 1
          if (u + 1 < S - t) ldsm_x4(st + (S + u + 1) * SLICE_BYTES + boff, bn[0], bn[1], bn[2], bn[3]);
          const int lev = t + u;  // 0-based level (l - 2)
          const int set = lev < OZ_NSETS - 1 ? lev : OZ_NSETS - 1;
#pragma unroll
          for (int mi = 0; mi < 2; ++mi) {
            mma_bf16(&acc[set][(mi * 2 + 0) * 4], a[mi], bc[0], bc[1]);
            mma_bf16(&acc[set][(mi * 2 + 1) * 4], a[mi], bc[2], bc[3]);
          }
#pragma unroll
          for (int x = 0; x < 4; ++x) bc[x] = bn[x];
        }
      }
    }
    if ((kt + 1) % OZ_FOLD == 0 || kt + 1 == ntile) {
#pragma unroll
      for (int s = 0; s < OZ_NSETS; ++s)
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          acc64[q] += (double)acc[s][q];
          acc[s][q] = 0.f;
        }
    }
    __syncthreads();
  }
  cp_wait0();

  // epilogue: complex -- (c0, c1) / (c2, c3) of tile (mi, ni) are Re/Im of
  // one entry; real -- they are two adjacent columns
  if constexpr (CPLX) {
    const bool use_beta = p.beta.x != 0.0 || p.beta.y != 0.0;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t i = i0 + wm * 32 + mi * 16 + g + 8 * h;
          const int64_t j = jc0 + wn * 8 + ni * 4 + tg;
          if (i >= p.m || j >= p.n) continue;
          if (p.lowerC && i < j) continue;
          const int q = (mi * 2 + ni) * 4 + 2 * h;
          const int ei = z.ea[i], fj = z.fb[j];
          double re = 0.0, im = 0.0;
          if (ei && fj) {
            const int sc = (ei - 2048) + (fj - 2048) - 14;
            re = ldexp(acc64[q], sc);
            im = ldexp(acc64[q + 1], sc);
          }
          cplx v = cmul(p.alpha, mkc(re, im));
          if (p.epi == EPI_XY) {
            const cplx v1 = p.P[i + j * p.ldp];
            const double s1 = p.c1[j], s2 = p.c2[j];
            const cplx x1 = cscale(v1, 0.5 * s1), x2 = cscale(v, 0.5 * s2);
            p.C[i + j * p.ldc] = cadd(x1, x2);
            p.Y[i + j * p.ldy] = csub(x2, x1);
          } else {
            if (use_beta) v = cadd(v, cmul(p.beta, p.C[i + j * p.ldc]));
            p.C[i + j * p.ldc] = v;
          }
        }
  } else {
    const bool use_beta = p.beta != 0.0;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int64_t i = i0 + wm * 32 + mi * 16 + g + 8 * h;
            const int64_t j = jc0 + wn * 16 + ni * 8 + 2 * tg + e;
            if (i >= p.m || j >= p.n) continue;
            if (p.lowerC && i < j) continue;
            const int q = (mi * 2 + ni) * 4 + 2 * h + e;
            const int ei = z.ea[i], fj = z.fb[j];
            double v = 0.0;
            if (ei && fj) v = ldexp(acc64[q], (ei - 2048) + (fj - 2048) - 14);
            v *= p.alpha;
            if (use_beta) v += p.beta * p.C[i + j * p.ldc];
            p.C[i + j * p.ldc] = v;
          }
  }
}

// ---- the tcgen05 product (5th-generation tensor cores, TMEM accumulators) ------
// Same arithmetic as oz_mma_kernel, tile 128 real rows x 64 real columns:
//   warp 0      TMA producer: per stage, ONE 3-D bulk-tensor copy brings all S
//               slices of the A tile (S x 128 rows x 32 k') and one all S
//               slices of the B tile (S x 64 x 32), 64-byte swizzled;
//   warp 1      MMA issuer (one thread): per stage and per 16-wide k step, the
//               36 slice pairs t + u <= S + 1 as tcgen05.mma kind::f16
//               (BF16 x BF16 -> FP32, M = 128) into TMEM level sets of 64
//               columns: sets 0..4 hold levels 2..6, sets 5 and 6 share the
//               levels >= 7.  The pairs (t, u) and (t, u + 1) always land in
//               adjacent sets, so they go as ONE N = 128 instruction whose B
//               operand is the two consecutive B slices (16 N = 128 and 4
//               N = 64 instructions per k step instead of 36 N = 64: an N = 64
//               instruction costs ~55 cycles, an N = 128 one 64 cycles, the
//               rate of the math);
//   warp 2      allocates / frees the 512 TMEM columns;
//   warps 4-11  zero the sets first; every 512 k' (the exactness bound of the
//               FP32 level sums) read the seven sets (tcgen05.ld; a thread
//               owns one row and 32 of the 64 columns), zero them again and
//               add them into int64 registers; then the epilogue (scales,
//               alpha/beta, the fused X/Y setup) straight from registers.
//               Pre-zeroed sets let every MMA accumulate, so a paired
//               instruction never mixes a fresh and a running set.
// Two smem stages of 96 KB; mbarriers full/empty per stage and tmem_full /
// tmem_empty per fold.  Every wait is bounded: on timeout the CTA records
// BSE_ERR_TIMEOUT in the status word (when given), stops issuing, drains what
// it started and frees its TMEM.
// Stage shape: two stages of 32 k' (rows of 64 bytes, 64-byte swizzle).  Four
// stages of 16 k' (32-byte rows and swizzle; UM_BK = 16, UM_STAGES = 4) measured
// the same speed on this part, so the refill latency is not what bounds it.
constexpr int UM_BM = 128, UM_BN = 64, UM_BK = 32, UM_STAGES = 2;
constexpr int UM_SLICE_A = UM_BM * UM_BK * 2, UM_SLICE_B = UM_BN * UM_BK * 2;  // 8 KB, 4 KB
constexpr int UM_FOLD = 512 / UM_BK;  // k-tiles per fold (512 k', the exactness bound)
constexpr int UM_ROWB = UM_BK * 2;    // bytes per k-major tile row
constexpr long long UM_WAIT_CYCLES = 2000000000LL;  // default wait limit, about 1 s; drains always use it

template <int S>
struct UmLayout {
  static constexpr int A_BYTES = S * UM_SLICE_A, B_BYTES = S * UM_SLICE_B;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = UM_STAGES * STAGE + 1024 + 256;  // + alignment, barriers
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// (-1)^neg (hi 2^17 + lo) 2^e as the nearest double (one rounding, ties to
// even), with integer instructions only: the exact 128-bit value is
// normalised and rounded on its bit pattern (FP64 instructions are the
// slowest unit of this part).  Results outside the normal range take ldexp.
__device__ __forceinline__ double um_to_double(int64_t hi, int32_t lo, int e, bool neg) {
  uint64_t vl = ((uint64_t)hi << 17) | (uint64_t)(uint32_t)lo;  // 128-bit two's complement
  uint64_t vh = (uint64_t)(hi >> 47);
  if ((int64_t)vh < 0) {  // magnitude
    vl = ~vl + 1;
    vh = ~vh + (vl == 0 ? 1 : 0);
    neg = !neg;
  }
  if (vh == 0 && vl == 0) return 0.0;
  int t = vh ? 127 - __clzll((long long)vh) : 63 - __clzll((long long)vl);  // top bit
  uint64_t mant;
  if (t <= 52) {
    mant = vl << (52 - t);
  } else {
    const int sh = t - 52;  // 1 .. 75
    uint64_t rb, st;
    if (sh < 64) {
      mant = (vl >> sh) | (vh << (64 - sh));
      rb = (vl >> (sh - 1)) & 1;
      st = vl & ((1ull << (sh - 1)) - 1);
    } else if (sh == 64) {
      mant = vh;
      rb = vl >> 63;
      st = vl & ~(1ull << 63);
    } else {
      mant = vh >> (sh - 64);
      rb = (vh >> (sh - 65)) & 1;
      st = (vh & ((1ull << (sh - 65)) - 1)) | vl;
    }
    if (rb && (st || (mant & 1))) ++mant;
    if (mant >> 53) mant >>= 1, ++t;
  }
  const int be = t + e + 1023;
  if (be <= 0 || be >= 2047) {
    const double d = ldexp((double)mant, t - 52 + e);
    return neg ? -d : d;
  }
  return __longlong_as_double((long long)(((uint64_t)neg << 63) | ((uint64_t)be << 52) | (mant & ((1ull << 52) - 1))));
}

// bounded wait on an mbarrier phase; false on timeout (which sets the abort
// flag) or, when abort_flag is given, as soon as another role has aborted
__device__ __forceinline__ bool um_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                        volatile int* timeout_flag, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (abort_flag && *abort_flag) return false;
    if (clock64() - t0 > limit) {
      *timeout_flag = 1;
      return false;
    }
  }
}

// K-major operand tile in shared memory, swizzled rows of UM_ROWB bytes (32:
// layout 6, 64: layout 4), 8-row groups 8 UM_ROWB bytes apart (stride byte
// offset); the leading byte offset is unused for swizzled K-major tiles;
// descriptor version 1.
__device__ __forceinline__ uint64_t um_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * UM_ROWB) >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)(UM_ROWB == 64 ? 4 : 6) << 61);
}

// instruction descriptors: FP32 accumulate, BF16 A and B, both K-major, N, M
__host__ __device__ constexpr uint32_t um_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(UM_BM >> 4) << 24);
}
constexpr int UM_NSETS = 7;  // levels 2..6, then two sets for the levels >= 7

// Geometry of one output tile of the persistent kernel (all roles compute it
// the same way from the linear tile index L): 128 real rows x 64 real
// columns, grouped rasterisation in bands of 8 tile rows, and with split-K
// (p.kchunk > 0) layer tz = L / (tiles per layer) of the k range.
struct UmTile {
  int64_t i0, jr0, jc0, kb2, tz;
  int ntile, nfold;
  bool valid;
};

// Every role of every CTA evaluates this for each tile it visits, so it uses
// 32-bit arithmetic (three 32-bit divisions; the tile count stays below 2^31,
// checked at launch): with 64-bit divisions the 20 warps of a CTA spent as
// many instructions here as in the folds and the epilogue of a thin product.
template <typename T>
__device__ __forceinline__ UmTile um_tile(const GemmParams<T>& p, uint32_t L, uint32_t ntx, uint32_t nty) {
  constexpr int XF = sizeof(T) == sizeof(cplx) ? 2 : 1;
  UmTile t;
  const uint32_t per = ntx * nty, band = 8u * ntx;
  const uint32_t tz = L / per;
  const uint32_t lin = L - tz * per;
  const uint32_t grp = lin / band, first = grp * 8u;
  const uint32_t rows = (nty - first) < 8u ? (nty - first) : 8u;
  const uint32_t loc = lin - grp * band;
  const uint32_t q = loc / rows;
  const uint32_t ty = first + (loc - q * rows), tx = q;
  t.tz = tz;
  t.i0 = (int64_t)ty * UM_BM, t.jr0 = (int64_t)tx * UM_BN, t.jc0 = t.jr0 / XF;
  t.valid = t.i0 < p.m && t.jc0 < p.n && !(p.lowerC && t.jc0 > t.i0 + UM_BM - 1);
  int64_t kb = 0, ke = p.k;
  if (p.triA == TRI_LO) ke = min(ke, t.i0 + UM_BM);
  if (p.triA == TRI_UP) kb = max(kb, t.i0);
  if (p.triB == TRI_LO) kb = max(kb, t.jc0);
  if (p.triB == TRI_UP) ke = min(ke, t.jc0 + UM_BN / XF);
  if (p.kchunk > 0) kb = max(kb, t.tz * p.kchunk), ke = min(ke, (t.tz + 1) * p.kchunk);
  t.kb2 = (XF * kb / UM_BK) * UM_BK;
  const int64_t ke2 = XF * ke;
  t.ntile = ke2 > t.kb2 ? (int)((ke2 - t.kb2 + UM_BK - 1) / UM_BK) : 0;
  t.nfold = (t.ntile + UM_FOLD - 1) / UM_FOLD;
  return t;
}

// Persistent form: one CTA per SM walks the tiles L = blockIdx.x,
// blockIdx.x + gridDim.x, ...  The stage ring, the MMA issue and the folds
// run on global counters across tiles, so the producer streams the next
// tile's slices while the current one finishes, and the fold warps write a
// tile's result (from registers, after its last fold has cleared the TMEM
// sets) while the MMAs of the next tile already run.
constexpr int UM_FOLD_WARPS = 16;                       // warps 4 .. 19
constexpr int UM_THREADS = 32 * (4 + UM_FOLD_WARPS);    // 640
template <int S, typename T>
__global__ void __launch_bounds__(UM_THREADS, 1) oz_umma_kernel(const OzArgs<T> z,
                                                                 const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ __align__(1024) unsigned char usm[];
  using L = UmLayout<S>;
  constexpr bool CPLX = sizeof(T) == sizeof(cplx);
  const GemmParams<T>& p = z.p;
  if (p.status && *(volatile const int64_t*)p.status) return;
  const uint32_t ntx = (uint32_t)((z.ncols_real + UM_BN - 1) / UM_BN), nty = (uint32_t)((z.Mp + UM_BM - 1) / UM_BM);
  const uint32_t ntiles = ntx * nty * (uint32_t)(p.kchunk > 0 ? (p.k + p.kchunk - 1) / p.kchunk : 1);

  unsigned char* base = (unsigned char*)(((uintptr_t)usm + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + UM_STAGES * L::STAGE);  // full[S] empty[S] tfull tempty drain
  uint32_t* tslot = (uint32_t*)(bars + 2 * UM_STAGES + 4);
  int* abort_flag = (int*)(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + UM_STAGES);
  const uint32_t tfull = smem_u32(bars + 2 * UM_STAGES), tempty = smem_u32(bars + 2 * UM_STAGES + 1);
  const uint32_t drain = smem_u32(bars + 2 * UM_STAGES + 2);
  if (threadIdx.x == 0) {
    for (int q = 0; q < UM_STAGES; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full0 + 8 * q));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty0 + 8 * q));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tfull));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tempty), "r"(UM_FOLD_WARPS));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(drain));
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  volatile int* ab = abort_flag;

  uint32_t issued = 0;  // producer: loads issued (global over the CTA's tiles)
  if (warp == 0 && lane == 0) {
    // producer
    bool ok = true;
    for (uint32_t Lt = blockIdx.x; Lt < ntiles && ok; Lt += gridDim.x) {
      const UmTile t = um_tile(p, Lt, ntx, nty);
      if (!t.valid) continue;
      for (int kt = 0; kt < t.ntile; ++kt, ++issued) {
        const uint32_t st = issued % UM_STAGES;
        if (issued >= UM_STAGES && !um_wait(empty0 + 8 * st, ((issued / UM_STAGES) - 1) & 1, ab, ab, z.wait)) {
          ok = false;
          break;
        }
        const uint32_t fb = full0 + 8 * st;
        const uint32_t da = smem_u32(base + st * L::STAGE), db = da + L::A_BYTES;
        const int x = (int)(t.kb2 + (int64_t)kt * UM_BK);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(L::STAGE) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];\n" ::"r"(da),
            "l"(&tmA), "r"(x), "r"((int)t.i0), "r"(0), "r"(fb)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];\n" ::"r"(db),
            "l"(&tmB), "r"(x), "r"((int)t.jr0), "r"(0), "r"(fb)
            : "memory");
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    bool ok = true;
    uint32_t g = 0, F = 0;  // k-tiles consumed, folds issued (global)
    for (uint32_t Lt = blockIdx.x; Lt < ntiles && ok; Lt += gridDim.x) {
      const UmTile t = um_tile(p, Lt, ntx, nty);
      if (!t.valid) continue;
      for (int kt = 0; kt < t.ntile; ++kt, ++g) {
        const uint32_t st = g % UM_STAGES;
        if (kt % UM_FOLD == 0) {  // the sets are zero (initially, or read and cleared by the last fold)
          ok = um_wait(tempty, F & 1, ab, ab, z.wait);
          if (!ok) break;
        }
        ok = um_wait(full0 + 8 * st, (g / UM_STAGES) & 1, ab, ab, z.wait);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t da = smem_u32(base + st * L::STAGE), db = da + L::A_BYTES;
#pragma unroll
        for (int ks = 0; ks < UM_BK / 16; ++ks) {
#pragma unroll
          for (int ts = 0; ts < S; ++ts) {
            const uint64_t ad = um_desc(da + ts * UM_SLICE_A + ks * 32);
#pragma unroll
            for (int u = 0; u < S - ts; u += 2) {
              // pair (ts, u) [+ (ts, u + 1)]: level ts + u (0-based) -> column min(ts + u, 5) * 64
              const int lev = ts + u;
              const uint32_t col = (uint32_t)((lev < 5 ? lev : 5) * UM_BN);
              const uint64_t bd = um_desc(db + u * UM_SLICE_B + ks * 32);
              const uint32_t idesc = (u + 1 < S - ts) ? um_idesc(2 * UM_BN) : um_idesc(UM_BN);
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + col),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(1u));
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         empty0 + 8 * st)
                     : "memory");
        if ((kt + 1) % UM_FOLD == 0 || kt + 1 == t.ntile) {
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(tfull)
                       : "memory");
          ++F;
        }
      }
    }
  } else if (warp >= 4) {
    // folds, all in integers: per column, levels 2..6 are exact FP32
    // integers in their own units 2^-7(l-2) and combine exactly by Horner's
    // rule into units of 2^-28 (below 2^52 per fold); the two sets of levels
    // >= 7 round to units of 2^-45, i.e. 2^-59 of the largest product (an
    // integer part at 2^-38 plus the rounded remainder, below 2^35 per fold).
    // No FP64 work until the epilogue.  A non-finite level sum (non-finite
    // input) marks its column, which ends as NaN.  Every fold clears the sets
    // it read, so the next tile's MMAs start from zero.  16 fold warps: warp w
    // reads TMEM lanes 32 (w % 4) .. + 31 (the quarter its SM sub-partition may
    // access) and 16 of the 64 columns of every set.
    constexpr int EC = UM_BN / 4;  // columns per fold/epilogue thread
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int col0 = ((warp - 4) >> 2) * EC;
    const uint32_t zero = 0;
    auto clear_sets = [&](int c0) {
#pragma unroll
      for (int set = 0; set < UM_NSETS; ++set)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(
                         tmem + lane_base + set * UM_BN + col0 + c0),
                     "r"(zero));
    };
    auto release_sets = [&]() {
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tempty) : "memory");
    };
#pragma unroll
    for (int c0 = 0; c0 < EC; c0 += 8) clear_sets(c0);
    release_sets();
    uint32_t F = 0;  // folds consumed (global)
    bool ok = true;
    for (uint32_t Lt = blockIdx.x; Lt < ntiles && ok; Lt += gridDim.x) {
      const UmTile t = um_tile(p, Lt, ntx, nty);
      if (!t.valid) continue;
      // a column's value = hi 2^-28 + lo 2^-45 in units of the level-2
      // products; after each fold lo keeps only the remainder 0 <= lo < 2^17
      // (its multiples of 2^17 move into hi exactly), so it stays 32-bit
      int64_t hi[EC];
      int32_t lo[EC];
#pragma unroll
      for (int q = 0; q < EC; ++q) hi[q] = 0, lo[q] = 0;
      uint32_t nanmask = 0;
      for (int f = 0; f < t.nfold; ++f, ++F) {
        const bool got = um_wait(tfull, F & 1, ab, ab, z.wait);
        if (!__all_sync(0xffffffffu, got)) {  // warp-uniform: the loads below are .sync.aligned
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
        for (int c0 = 0; c0 < EC; c0 += 4) {
          int64_t tot[4], low[4];
#pragma unroll
          for (int set = 0; set < UM_NSETS; ++set) {
            uint32_t v[4];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                         : "r"(tmem + lane_base + set * UM_BN + col0 + c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float x = __uint_as_float(v[q]);
              if (set < 5) {
                const int iv = __float2int_rn(x * (float)(1 << (7 * set)));  // exact
                tot[q] = set == 0 ? (int64_t)iv : tot[q] * 128 + iv;
              } else {
                if (!(fabsf(x) <= 3.0e38f)) nanmask |= 1u << (c0 + q);
                const float y = x * 274877906944.0f;  // 2^38, exact
                const float yi = rintf(y);
                const int64_t iv = (int64_t)(int)yi * 128 + __float2int_rn((y - yi) * 128.0f);  // units 2^-45
                low[q] = set == 5 ? iv : low[q] + iv;
              }
            }
          }
          if ((c0 & 7) == 4) clear_sets(c0 - 4);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int64_t l = (int64_t)lo[c0 + q] + low[q];
            hi[c0 + q] += tot[q] + (l >> 17);
            lo[c0 + q] = (int32_t)(l & 0x1FFFF);
          }
        }
        release_sets();
      }
      if (!ok) break;
      // epilogue: thread = one row of the tile and columns [col0, col0 + 32)
      // of its 64 real columns; complex -- real columns (2j, 2j+1) are (Re,
      // Im) of logical column jc0 + col0/2 + j; real -- column jc0 + col0 + q
      const int64_t i = t.i0 + (warp & 3) * 32 + lane;
      if (i >= p.m) continue;
      T* C = p.C + (p.kchunk > 0 ? t.tz * p.cstride : 0);
      const int ei = z.ea[i];
      const double qnan = __longlong_as_double(0x7ff8000000000000LL);
      // value of column q = (hi 2^17 + lo) 2^(sc - 45); alpha = -1 folds into
      // the sign for free
      auto value = [&](int q, int sc, bool neg) -> double {
        if ((nanmask >> q) & 1u) return qnan;
        return um_to_double(hi[q], lo[q], sc - 45, neg);
      };
      if constexpr (CPLX) {
        const bool use_beta = p.beta.x != 0.0 || p.beta.y != 0.0;
        // alpha = +-1 and beta in {0, 1} (every product but the fused X/Y
        // setup): no FP64 work but the one add of C
        const bool fast = p.epi != EPI_XY && p.alpha.y == 0.0 && (p.alpha.x == 1.0 || p.alpha.x == -1.0) &&
                          p.beta.y == 0.0 && (p.beta.x == 0.0 || p.beta.x == 1.0);
        const bool aneg = p.alpha.x < 0.0;
        if (fast) {
#pragma unroll
          for (int jj = 0; jj < EC / 2; ++jj) {
            const int64_t j = t.jc0 + col0 / 2 + jj;
            if (j >= p.n) break;
            if (p.lowerC && i < j) break;
            const int fj = z.fb[j];
            double re = 0.0, im = 0.0;
            if (ei && fj) {
              const int sc = (ei - 2048) + (fj - 2048) - 14;
              re = value(2 * jj, sc, aneg);
              im = value(2 * jj + 1, sc, aneg);
            }
            cplx v = mkc(re, im);
            if (use_beta) v = cadd(v, C[i + j * p.ldc]);
            C[i + j * p.ldc] = v;
          }
          continue;
        }
#pragma unroll
        for (int jj = 0; jj < EC / 2; ++jj) {
          const int64_t j = t.jc0 + col0 / 2 + jj;
          if (j >= p.n) break;
          if (p.lowerC && i < j) break;
          const int fj = z.fb[j];
          double re = 0.0, im = 0.0;
          if (ei && fj) {
            const int sc = (ei - 2048) + (fj - 2048) - 14;
            re = value(2 * jj, sc, false);
            im = value(2 * jj + 1, sc, false);
          }
          cplx v = cmul(p.alpha, mkc(re, im));
          if (p.epi == EPI_XY) {
            const cplx v1 = p.P[i + j * p.ldp];
            const double s1 = p.c1[j], s2 = p.c2[j];
            const cplx x1 = cscale(v1, 0.5 * s1), x2 = cscale(v, 0.5 * s2);
            C[i + j * p.ldc] = cadd(x1, x2);
            p.Y[i + j * p.ldy] = csub(x2, x1);
          } else {
            if (use_beta) v = cadd(v, cmul(p.beta, C[i + j * p.ldc]));
            C[i + j * p.ldc] = v;
          }
        }
      } else {
        const bool use_beta = p.beta != 0.0;
        const bool fast = (p.alpha == 1.0 || p.alpha == -1.0) && (p.beta == 0.0 || p.beta == 1.0);
#pragma unroll
        for (int jj = 0; jj < EC; ++jj) {
          const int64_t j = t.jc0 + col0 + jj;
          if (j >= p.n) break;
          if (p.lowerC && i < j) break;
          const int fj = z.fb[j];
          double v = 0.0;
          if (ei && fj) v = value(jj, (ei - 2048) + (fj - 2048) - 14, fast && p.alpha < 0.0);
          if (!fast) v *= p.alpha;
          if (use_beta) v = fast ? v + C[i + j * p.ldc] : v + p.beta * C[i + j * p.ldc];
          C[i + j * p.ldc] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  const bool failed = *ab != 0;
  if (warp == 1 && lane == 0) {
    // every MMA this thread issued has completed once `drain` flips (bounded)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(drain)
                 : "memory");
    um_wait(drain, 0, nullptr, ab, UM_WAIT_CYCLES);
  }
  if (failed && warp == 0 && lane == 0) {
    // the copies still in flight land before the CTA leaves (bounded)
    for (uint32_t g = issued > UM_STAGES ? issued - UM_STAGES : 0; g < issued; ++g)
      um_wait(full0 + 8 * (g % UM_STAGES), (g / UM_STAGES) & 1, nullptr, ab, UM_WAIT_CYCLES);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
  }
  if (failed && threadIdx.x == 0 && p.status) dev_fail((int64_t*)p.status, BSE_ERR_TIMEOUT, 0);
}

// ---- real operands -------------------------------------------------------------
__device__ __forceinline__ bool op_elem_d(const double* X, int64_t ldx, int op, int tri, int64_t r, int64_t c,
                                          int64_t R, int64_t C, double* out) {
  if (r >= R || c >= C) return false;
  if (tri == TRI_LO && c > r) return false;
  if (tri == TRI_UP && c < r) return false;
  *out = (op == OPN) ? X[r + c * ldx] : X[c + r * ldx];
  return true;
}

// exponents of rows (rowsx = 1) of op(A) or of columns (rowsx = 0) of op(B)
__global__ void oz_exp_d_kernel(int64_t R, int64_t C, const double* X, int64_t ldx, int op, int tri, int rowsx,
                                int* ex) {
  __shared__ int mx[32][33];
  const int64_t b0 = (int64_t)blockIdx.y * 32, b1 = (int64_t)blockIdx.x * 32;  // (row block, col block)
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    int64_t r, c;
    if (op == OPN) r = b0 + tx, c = b1 + q;
    else r = b0 + q, c = b1 + tx;
    double v = 0.0;
    int a = -4096;
    if (op_elem_d(X, ldx, op, tri, r, c, R, C, &v)) a = fexp_bits(v);
    const int lr = (int)(r - b0), lc = (int)(c - b1);
    if (rowsx) mx[lr][lc] = a; else mx[lc][lr] = a;
  }
  __syncthreads();
  if (ty == 0) {
    int a = -4096;
    for (int q = 0; q < 32; ++q) a = max(a, mx[tx][q]);
    const int64_t idx = (rowsx ? b0 : b1) + tx;
    if (a > -4096 && idx < (rowsx ? R : C)) atomicMax(ex + idx, 2048 + a);
  }
}

// slices: rows of op(A) (trans = 0) or columns of op(B) (trans = 1) become the
// slice rows; Xs[t][rows_p][Kp] bf16, every padded entry written
template <int S>
__global__ void oz_split_d_kernel(int64_t R, int64_t C, const double* X, int64_t ldx, int op, int tri, int trans,
                                  const int* ex, int64_t Rp, int64_t Kp, uint16_t* Xs) {
  __shared__ double tile[32][33];  // tile[slice row][k]
  const int64_t b0 = (int64_t)blockIdx.y * 32, b1 = (int64_t)blockIdx.x * 32;  // slice-row block, k block
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    // logical element: trans = 0 -> (row b0+., k b1+.) of op(X); trans = 1 -> (k b1+., col b0+.)
    int64_t r, c;
    const bool contig_first = (op == OPN);  // stored contiguous along the logical row index
    int sr, sk;
    if (trans == 0) {
      if (contig_first) r = b0 + tx, c = b1 + q, sr = tx, sk = q;
      else r = b0 + q, c = b1 + tx, sr = q, sk = tx;
    } else {
      if (contig_first) r = b1 + tx, c = b0 + q, sr = q, sk = tx;
      else r = b1 + q, c = b0 + tx, sr = tx, sk = q;
    }
    double v = 0.0;
    op_elem_d(X, ldx, op, tri, r, c, R, C, &v);
    tile[sr][sk] = v;
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int64_t rr = b0 + q, kk = b1 + tx;
    if (rr >= Rp || kk >= Kp) continue;
    const int64_t nrows = trans ? C : R;
    const int eb = (rr < nrows) ? ex[rr] : 0;
    float sl[S];
    split_value(tile[q][tx], eb ? eb - 2048 : 0, S, sl);
    for (int t = 0; t < S; ++t) Xs[((int64_t)t * Rp + rr) * Kp + kk] = bf16_bits_exact(sl[t]);
  }
}

}  // namespace

// Workspace (thread-current, set by the solve entry points)
static thread_local OzWork g_oz = {nullptr, 0, 0, OZ_ENGINE_TCGEN05, 0};
void oz_set_current(const OzWork& w) { g_oz = w; }
OzWork oz_current() { return g_oz; }

size_t oz_work_bytes(int64_t maxdim, int slices) {
  const int64_t Mp = (maxdim + OZ_BM - 1) / OZ_BM * OZ_BM;
  const int64_t Np = (2 * maxdim + OZ_BN - 1) / OZ_BN * OZ_BN;
  const int64_t Kp = (2 * maxdim + OZ_BK - 1) / OZ_BK * OZ_BK;
  return (size_t)slices * 2 * (size_t)Kp * (size_t)(Mp + Np) + (size_t)(Mp + Np) * 4 + 1024;
}

// ---- tcgen05 engine: tensor maps and launch ------------------------------------
// SM count of the current device (looked up once per device)
static int64_t oz_device_sms() {
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
    else
      cudaGetLastError();
  }
  return fn;
}

// slices [S][rows][Kp] bf16 as a 3-D tensor (k', row, slice); box (UM_BK, box_rows, S), swizzled as
// the descriptors expect
static bool slice_map(CUtensorMap* m, const void* base, int S, int64_t rows, int64_t Kp, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)S};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
  const cuuint32_t box[3] = {(cuuint32_t)UM_BK, (cuuint32_t)box_rows, (cuuint32_t)S};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, UM_ROWB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S, typename T>
static bse_status umma_launch(cudaStream_t s, const OzArgs<T>& z, int64_t ncols_real, double flops) {
  CUtensorMap ta, tb;
  if (!slice_map(&ta, z.As, S, z.Mp, z.Kp, UM_BM) || !slice_map(&tb, z.Bs, S, z.Np, z.Kp, UM_BN)) {
    bse_internal_set_error("tensor-core GEMM: cuTensorMapEncodeTiled failed");
    return BSE_ERR_CUDA;
  }
  {
    const bse_status r = set_smem_attr((const void*)oz_umma_kernel<S, T>, UmLayout<S>::SMEM);
    if (r) return r;
  }
  // persistent: one CTA per SM (its shared memory allows no second one), or
  // one per tile when there are fewer
  OzArgs<T> za = z;
  za.ncols_real = ncols_real;
  const int64_t layers = z.p.kchunk > 0 ? (z.p.k + z.p.kchunk - 1) / z.p.kchunk : 1;
  const int64_t tiles = ((ncols_real + UM_BN - 1) / UM_BN) * ((z.Mp + UM_BM - 1) / UM_BM) * layers;
  if (tiles >= ((int64_t)1 << 31)) {
    bse_internal_set_error("tensor-core GEMM: more than 2^31 tiles");
    return BSE_ERR_ARG;
  }
  const int64_t sms = oz_device_sms();
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  prof_tc_begin(s);
  prof_launch_begin(s);
  oz_umma_kernel<S, T><<<grid, UM_THREADS, UmLayout<S>::SMEM, s>>>(za, ta, tb);
  prof_launch_end(s, "oz_umma_kernel");
  prof_tc_end(s, flops);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

template <int S>
static bse_status oz_run(cudaStream_t s, const GemmParams<cplx>& p, double flops) {
  const int64_t Mp = (p.m + OZ_BM - 1) / OZ_BM * OZ_BM;
  const int64_t Np = (2 * p.n + OZ_BN - 1) / OZ_BN * OZ_BN;
  const int64_t Kp = (2 * p.k + OZ_BK - 1) / OZ_BK * OZ_BK;
  const size_t need = (size_t)S * 2 * (size_t)Kp * (size_t)(Mp + Np) + (size_t)(Mp + Np) * 4 + 1024;
  if (!g_oz.ptr || g_oz.bytes < need) {
    bse_internal_set_error("tensor-core GEMM workspace too small");
    return BSE_ERR_NOMEM;
  }
  char* base = (char*)g_oz.ptr;
  uint32_t* As = (uint32_t*)base;
  uint32_t* Bs = (uint32_t*)(base + (size_t)S * Mp * Kp * 2);
  int* ea = (int*)(base + (size_t)S * (Mp + Np) * Kp * 2);
  int* fb = ea + Mp;
  prof_launch_begin(s);
  BSE_CUDA(cudaMemsetAsync(ea, 0, sizeof(int) * (Mp + Np / 2), s));
  dim3 tb(32, 8);
  oz_rowexp_kernel<<<dim3(ceil_div_u(p.k, 32), ceil_div_u(p.m, 32)), tb, 0, s>>>(p.m, p.k, p.A, p.lda, p.opA, p.triA, ea);
  oz_colexp_kernel<<<dim3(ceil_div_u(p.n, 32), ceil_div_u(p.k, 32)), tb, 0, s>>>(p.k, p.n, p.B, p.ldb, p.opB, p.triB, fb);
  oz_split_a_kernel<S><<<dim3(ceil_div_u(Kp / 2, 32), ceil_div_u(Mp, 32)), tb, 0, s>>>(p.m, p.k, p.A, p.lda, p.opA,
                                                                                       p.triA, ea, Mp, Kp, As);
  oz_split_b_kernel<S><<<dim3(ceil_div_u(Np / 2, 32), ceil_div_u(Kp / 2, 32)), tb, 0, s>>>(p.k, p.n, p.B, p.ldb,
                                                                                           p.opB, p.triB, fb, Np, Kp, Bs);
  prof_launch_end(s, "oz_split (exponents, slices)");
  bse_count_launch(4);
  BSE_LAUNCH_CHECK();
  OzArgs<cplx> z;
  z.p = p, z.As = As, z.Bs = Bs, z.ea = ea, z.fb = fb, z.Mp = Mp, z.Np = Np, z.Kp = Kp;
  z.wait = g_oz.wait_cycles > 0 ? (long long)g_oz.wait_cycles : UM_WAIT_CYCLES;
  if (g_oz.engine == OZ_ENGINE_TCGEN05) return umma_launch<S, cplx>(s, z, Np, flops);
  const int smem = 2 * 2 * S * OZ_BM * OZ_ROWB;
  {
    const bse_status r = set_smem_attr((const void*)oz_mma_kernel<S, cplx>, smem);
    if (r) return r;
  }
  dim3 grid((unsigned)(Np / OZ_BN), (unsigned)(Mp / OZ_BM));
  prof_tc_begin(s);
  oz_mma_kernel<S, cplx><<<grid, 256, smem, s>>>(z);
  prof_tc_end(s, flops);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

bse_status gemm_z_oz_raw(cudaStream_t s, const GemmParams<cplx>& p, double fp64_flops) {
  if (p.m <= 0 || p.n <= 0) return BSE_OK;
  if (p.opA == OPT || p.opB == OPT) {
    bse_internal_set_error("tensor-core GEMM: transpose without conjugate is not supported");
    return BSE_ERR_ARG;
  }
  return oz_run<8>(s, p, fp64_flops);
}

template <int S>
static bse_status oz_run_d(cudaStream_t s, const GemmParams<double>& p, double flops) {
  const int64_t Mp = (p.m + OZ_BM - 1) / OZ_BM * OZ_BM;
  const int64_t Np = (p.n + OZ_BN - 1) / OZ_BN * OZ_BN;
  const int64_t Kp = (p.k + OZ_BK - 1) / OZ_BK * OZ_BK;
  const size_t need = (size_t)S * 2 * (size_t)Kp * (size_t)(Mp + Np) + (size_t)(Mp + Np) * 4 + 1024;
  if (!g_oz.ptr || g_oz.bytes < need) {
    bse_internal_set_error("tensor-core GEMM workspace too small");
    return BSE_ERR_NOMEM;
  }
  char* base = (char*)g_oz.ptr;
  uint16_t* As = (uint16_t*)base;
  uint16_t* Bs = (uint16_t*)(base + (size_t)S * Mp * Kp * 2);
  int* ea = (int*)(base + (size_t)S * (Mp + Np) * Kp * 2);
  int* fb = ea + Mp;
  prof_launch_begin(s);
  BSE_CUDA(cudaMemsetAsync(ea, 0, sizeof(int) * (Mp + Np), s));
  dim3 tb(32, 8);
  oz_exp_d_kernel<<<dim3(ceil_div_u(p.k, 32), ceil_div_u(p.m, 32)), tb, 0, s>>>(p.m, p.k, p.A, p.lda, p.opA, p.triA, 1, ea);
  oz_exp_d_kernel<<<dim3(ceil_div_u(p.n, 32), ceil_div_u(p.k, 32)), tb, 0, s>>>(p.k, p.n, p.B, p.ldb, p.opB, p.triB, 0, fb);
  oz_split_d_kernel<S><<<dim3(ceil_div_u(Kp, 32), ceil_div_u(Mp, 32)), tb, 0, s>>>(p.m, p.k, p.A, p.lda, p.opA,
                                                                                    p.triA, 0, ea, Mp, Kp, As);
  oz_split_d_kernel<S><<<dim3(ceil_div_u(Kp, 32), ceil_div_u(Np, 32)), tb, 0, s>>>(p.k, p.n, p.B, p.ldb, p.opB,
                                                                                    p.triB, 1, fb, Np, Kp, Bs);
  prof_launch_end(s, "oz_split (exponents, slices)");
  bse_count_launch(4);
  BSE_LAUNCH_CHECK();
  OzArgs<double> z;
  z.p = p, z.As = (const uint32_t*)As, z.Bs = (const uint32_t*)Bs, z.ea = ea, z.fb = fb, z.Mp = Mp, z.Np = Np,
  z.Kp = Kp;
  z.wait = g_oz.wait_cycles > 0 ? (long long)g_oz.wait_cycles : UM_WAIT_CYCLES;
  if (g_oz.engine == OZ_ENGINE_TCGEN05) return umma_launch<S, double>(s, z, Np, flops);
  const int smem = 2 * 2 * S * OZ_BM * OZ_ROWB;
  {
    const bse_status r = set_smem_attr((const void*)oz_mma_kernel<S, double>, smem);
    if (r) return r;
  }
  dim3 grid((unsigned)(Np / OZ_BN), (unsigned)(Mp / OZ_BM));
  prof_tc_begin(s);
  oz_mma_kernel<S, double><<<grid, 256, smem, s>>>(z);
  prof_tc_end(s, flops);
  bse_count_launch();
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

bse_status gemm_d_oz_raw(cudaStream_t s, const GemmParams<double>& p, double fp64_flops) {
  if (p.m <= 0 || p.n <= 0) return BSE_OK;
  if (p.opA == OPC || p.opB == OPC) {
    bse_internal_set_error("tensor-core real GEMM: conjugate transpose is not meaningful");
    return BSE_ERR_ARG;
  }
  return oz_run_d<8>(s, p, fp64_flops);
}
