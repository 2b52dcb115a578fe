// Out-of-core tile executor: runs a plan of tile copies and tile tasks for
// the BLAS3 stages of Alg. 2 (forming A +- B, step 1's Cholesky factorisation
// of A - B and step 2's congruence M = L^H (A + B) L) with the matrices in
// host memory.  Section 4 puts real exciton problems at n ~ 1e5, where one
// complex128 matrix is 160 GB: A, B, L and M together do not fit in HBM, so
// they move through the device in nb x nb tiles (Grace memory over
// NVLink-C2C on a GB300 node).
//
// The plan (from the package's planner) is a sequence of LOAD / ALLOC /
// COMPUTE / STORE / FREE operations; this file validates it on the host,
// then issues copies on a copy stream and tasks on three compute streams
// (the caller's and two more).  Every device slot records its last writer
// and the reads since as events; each operation waits only for the accesses
// it conflicts with, so copies of the next tiles run under the current tasks
// (limited only by the free slots) and independent tile tasks overlap.
//
// Tasks use the FP64 GEMM engine and the blocked Cholesky of potrf.cu.  The
// tile TRSM (X L^H = A) multiplies by the tile's inverse conjugate
// transpose, computed once per POTRF with the L^H solve of potrf.cu; its
// product goes to a spare slot that then takes the tile's place.
#include <string>
#include <vector>

#include "kernels.cuh"

__global__ void ooc_form_kernel(int64_t count, const cplx* __restrict__ X, const cplx* __restrict__ Y, double sgn,
                                cplx* __restrict__ out, const int64_t* status) {
  if (*(volatile const int64_t*)status) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < count) {
    const cplx x = X[e], y = Y[e];
    out[e] = mkc(x.x + sgn * y.x, x.y + sgn * y.y);
  }
}

// strict upper part := 0 (the blocked Cholesky leaves it untouched outside
// its 64 x 64 diagonal blocks)
__global__ void ooc_zero_upper_kernel(int64_t nb, cplx* __restrict__ T, const int64_t* status) {
  if (*(volatile const int64_t*)status) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nb * nb) {
    const int64_t i = e % nb, j = e / nb;
    if (i < j) T[e] = mkc(0.0, 0.0);
  }
}

__global__ void ooc_identity_kernel(int64_t nb, cplx* __restrict__ X) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nb * nb) X[e] = mkc((e % nb) == (e / nb) ? 1.0 : 0.0, 0.0);
}

// The first time the status word is set, remember the tile row of the POTRF
// task just issued (every later kernel returns at once, so the first POTRF
// after which the word is nonzero is the failing one).
__global__ void ooc_mark_kernel(const int64_t* status, int64_t* mark, int64_t row) {
  if (*(volatile const int64_t*)status != 0 && *mark < 0) *mark = row;
}

static unsigned ooc_blocks(int64_t count) { return ceil_div_u(count, 256); }

constexpr int OOC_STREAMS = 3;  // compute streams (the caller's and two more)

#define OOC_LAUNCH_CHECK()                                      \
  do {                                                          \
    bse_count_launch();                                         \
    BSE_LAUNCH_CHECK();                                         \
  } while (0)

size_t ooc_ws_bytes(int64_t nb, int64_t budget) {
  const size_t tile = sizeof(cplx) * (size_t)nb * (size_t)nb;
  const size_t al = 256;
  auto up = [&](size_t b) { return (b + al - 1) / al * al; };
  return up(tile) * (size_t)(budget + 1)      // slots, one spare
         + (1 + OOC_STREAMS) * up(tile)       // inverse, a Hermitian expansion per compute stream
         + up(sizeof(cplx) * chol_linv_elems(nb))  // diagonal-block inverses
         + up(4 * sizeof(int64_t))            // status word, failing tile row
         + al;
}

static bool task_needs(int kind, int which) {
  // which 0: in0, 1: in1
  switch (kind) {
    case BSE_OOC_FORM_SUM:
    case BSE_OOC_FORM_DIFF:
    case BSE_OOC_GEMM_SUB:
    case BSE_OOC_GEMM_ACC:
      return true;
    case BSE_OOC_TRSM:
    case BSE_OOC_HERK:
      return which == 0;
    default:
      return false;
  }
}

const char* ooc_validate(int64_t nb, int64_t ntiles, void* const* host_tiles, int64_t nops, const bse_ooc_op* ops,
                         int64_t ntasks, const bse_ooc_task* tasks, int64_t budget, std::string& why) {
  if (nb < 1 || nb > 4096) return "nb must be in [1, 4096]";
  if (ntiles < 0 || nops < 0 || ntasks < 0) return "negative count";
  if (budget < 1) return "budget must be >= 1";
  if ((nops && !ops) || (ntasks && !tasks) || (ntiles && !host_tiles)) return "NULL plan array";
  std::vector<char> res((size_t)ntiles, 0);
  int64_t nres = 0, last_potrf = -1;
  auto fail = [&](int64_t i, const char* what) {
    why = "op " + std::to_string((long long)i) + ": " + what;
    return why.c_str();
  };
  for (int64_t i = 0; i < nops; ++i) {
    const int kind = ops[i].kind;
    const int64_t a = ops[i].arg;
    if (kind == BSE_OOC_COMPUTE) {
      if (a < 0 || a >= ntasks) return fail(i, "task index out of range");
      const bse_ooc_task& t = tasks[a];
      if (t.kind < BSE_OOC_FORM_SUM || t.kind > BSE_OOC_GEMM_ACC) return fail(i, "unknown task kind");
      const int64_t ids[3] = {t.out, t.in0, t.in1};
      for (int w = 0; w < 3; ++w) {
        const bool need = w == 0 || task_needs(t.kind, w - 1);
        if (!need) continue;
        if (ids[w] < 0 || ids[w] >= ntiles) return fail(i, "task tile out of range");
        if (!res[(size_t)ids[w]]) return fail(i, "task tile not resident");
      }
      if ((task_needs(t.kind, 0) && t.in0 == t.out) || (task_needs(t.kind, 1) && t.in1 == t.out))
        return fail(i, "task output aliases an input");
      if (t.kind == BSE_OOC_POTRF) last_potrf = t.out;
      if (t.kind == BSE_OOC_TRSM && t.in0 != last_potrf) return fail(i, "TRSM tile is not the latest POTRF's");
      continue;
    }
    if (a < 0 || a >= ntiles) return fail(i, "tile index out of range");
    switch (kind) {
      case BSE_OOC_LOAD:
      case BSE_OOC_ALLOC:
        if (res[(size_t)a]) return fail(i, "tile already resident");
        if (kind == BSE_OOC_LOAD && !host_tiles[a]) return fail(i, "LOAD of a tile without host memory");
        res[(size_t)a] = 1;
        if (++nres > budget) return fail(i, "more tiles resident than the budget");
        break;
      case BSE_OOC_STORE:
        if (!res[(size_t)a]) return fail(i, "STORE of a tile that is not resident");
        if (!host_tiles[a]) return fail(i, "STORE of a tile without host memory");
        break;
      case BSE_OOC_FREE:
        if (!res[(size_t)a]) return fail(i, "FREE of a tile that is not resident");
        res[(size_t)a] = 0;
        --nres;
        break;
      default:
        return fail(i, "unknown op kind");
    }
  }
  return nullptr;
}

namespace {

// Events made during one run, destroyed at its end (recorded work may still
// be pending then; CUDA releases such an event once its work completes).
struct EventPool {
  std::vector<cudaEvent_t> all;
  cudaError_t make(cudaEvent_t* e) {
    const cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    if (r == cudaSuccess) all.push_back(*e);
    return r;
  }
  ~EventPool() {
    for (cudaEvent_t e : all) cudaEventDestroy(e);
  }
};

// Streams created for one run are drained and destroyed before the executor
// returns, on every path: host tiles are not touched after the call returns.
struct StreamSet {
  std::vector<cudaStream_t> v;
  ~StreamSet() {
    for (cudaStream_t x : v) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  }
};

// One device buffer's accesses in flight: its last writer and the reads
// issued since that write.
struct Hazard {
  cudaEvent_t wr = nullptr;
  std::vector<cudaEvent_t> rd;
};

}  // namespace

// Issues the plan and returns once the created streams have drained (the
// caller's stream waits for them; the caller synchronises it and reads the
// status word at `status`, the failing tile row at `status + 2`).
//
// Tasks are dealt round-robin to OOC_STREAMS compute streams, copies go to
// one copy stream; every ordering the plan implies is an event wait: a task
// waits for the last writer of each tile it touches and, for the tile it
// writes, for the reads issued since; a LOAD into a slot waits for the last
// writer and readers of the slot's previous tile.  Independent tile tasks
// then overlap, which fills the SMs that one tile product leaves idle.
bse_status ooc_execute(cudaStream_t s, void* ws, int64_t nb, int64_t ntiles, void* const* host_tiles, int64_t nops,
                       const bse_ooc_op* ops, const bse_ooc_task* tasks, int64_t budget, int64_t** status_out) {
  const size_t al = 256;
  auto up = [&](size_t b) { return (b + al - 1) / al * al; };
  const size_t tile_b = sizeof(cplx) * (size_t)nb * (size_t)nb;
  char* p = (char*)(((uintptr_t)ws + al - 1) / al * al);
  const int nslots = (int)budget + 1;
  std::vector<cplx*> slot((size_t)nslots);
  for (int i = 0; i < nslots; ++i) {
    slot[(size_t)i] = (cplx*)p;
    p += up(tile_b);
  }
  cplx* Xinv = (cplx*)p;  // L^{-H} of the latest POTRF tile
  p += up(tile_b);
  cplx* F[OOC_STREAMS];  // Hermitian expansion, one per compute stream
  for (int i = 0; i < OOC_STREAMS; ++i) {
    F[i] = (cplx*)p;
    p += up(tile_b);
  }
  cplx* Linv = (cplx*)p;
  p += up(sizeof(cplx) * chol_linv_elems(nb));
  int64_t* status = (int64_t*)p;  // [0] code, [1] info, [2] failing tile row
  *status_out = status;
  BSE_CUDA(cudaMemsetAsync(status, 0, 2 * sizeof(int64_t), s));
  BSE_CUDA(cudaMemsetAsync(status + 2, 0xff, sizeof(int64_t), s));

  EventPool evp;
  StreamSet made;
  cudaStream_t cst[OOC_STREAMS];
  cst[0] = s;
  for (int i = 0; i < OOC_STREAMS; ++i) {  // OOC_STREAMS - 1 compute streams and the copy stream
    cudaStream_t x;
    BSE_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    made.v.push_back(x);
    if (i + 1 < OOC_STREAMS) cst[i + 1] = x;
  }
  cudaStream_t cs = made.v.back();
  // every stream starts after the caller's earlier work and the status reset
  // (earlier work on s may still use this workspace)
  cudaEvent_t start;
  BSE_CUDA(evp.make(&start));
  BSE_CUDA(cudaEventRecord(start, s));
  for (cudaStream_t x : made.v) BSE_CUDA(cudaStreamWaitEvent(x, start, 0));

  std::vector<Hazard> hz((size_t)nslots);
  Hazard inv;  // Xinv and Linv
  auto wait_write = [&](cudaStream_t st, const Hazard& h) -> cudaError_t {
    return h.wr ? cudaStreamWaitEvent(st, h.wr, 0) : cudaSuccess;
  };
  auto wait_all = [&](cudaStream_t st, const Hazard& h) -> cudaError_t {
    cudaError_t r = wait_write(st, h);
    for (cudaEvent_t e : h.rd)
      if (r == cudaSuccess) r = cudaStreamWaitEvent(st, e, 0);
    return r;
  };

  std::vector<int> free_slots;
  for (int i = nslots - 2; i >= 0; --i) free_slots.push_back(i);
  int spare = nslots - 1;
  std::vector<int> slot_of((size_t)ntiles, -1);
  const cplx one = mkc(1.0, 0.0), mone = mkc(-1.0, 0.0);
  const int64_t nn = nb * nb;
  int turn = 0;

  for (int64_t i = 0; i < nops; ++i) {
    const int kind = ops[i].kind;
    const int64_t a = ops[i].arg;
    if (kind == BSE_OOC_LOAD || kind == BSE_OOC_ALLOC) {
      const int q = free_slots.back();
      free_slots.pop_back();
      slot_of[(size_t)a] = q;
      BSE_CUDA(wait_all(cs, hz[(size_t)q]));
      if (kind == BSE_OOC_LOAD)
        BSE_CUDA(cudaMemcpyAsync(slot[(size_t)q], host_tiles[a], tile_b, cudaMemcpyHostToDevice, cs));
      else
        BSE_CUDA(cudaMemsetAsync(slot[(size_t)q], 0, tile_b, cs));
      cudaEvent_t e;
      BSE_CUDA(evp.make(&e));
      BSE_CUDA(cudaEventRecord(e, cs));
      hz[(size_t)q].wr = e;
      hz[(size_t)q].rd.clear();
    } else if (kind == BSE_OOC_STORE) {
      const int q = slot_of[(size_t)a];
      BSE_CUDA(wait_write(cs, hz[(size_t)q]));
      BSE_CUDA(cudaMemcpyAsync(host_tiles[a], slot[(size_t)q], tile_b, cudaMemcpyDeviceToHost, cs));
      cudaEvent_t e;
      BSE_CUDA(evp.make(&e));
      BSE_CUDA(cudaEventRecord(e, cs));
      hz[(size_t)q].rd.push_back(e);
    } else if (kind == BSE_OOC_FREE) {
      free_slots.push_back(slot_of[(size_t)a]);
      slot_of[(size_t)a] = -1;
    } else {  // COMPUTE
      const bse_ooc_task& t = tasks[a];
      const int si = turn;
      turn = (turn + 1) % OOC_STREAMS;
      cudaStream_t st = cst[si];
      const int qo = slot_of[(size_t)t.out];
      const int q0 = t.in0 >= 0 && task_needs(t.kind, 0) ? slot_of[(size_t)t.in0] : -1;
      const int q1 = t.in1 >= 0 && task_needs(t.kind, 1) ? slot_of[(size_t)t.in1] : -1;
      const bool trsm = t.kind == BSE_OOC_TRSM, potrf = t.kind == BSE_OOC_POTRF;
      // the tile written: out, or for TRSM the spare slot that takes its place
      const int qw = trsm ? spare : qo;
      BSE_CUDA(wait_all(st, hz[(size_t)qw]));
      if (trsm) BSE_CUDA(wait_write(st, hz[(size_t)qo]));
      for (int q : {q0, q1})
        if (q >= 0) BSE_CUDA(wait_write(st, hz[(size_t)q]));
      if (potrf) BSE_CUDA(wait_all(st, inv));
      if (trsm) BSE_CUDA(wait_write(st, inv));
      cplx* O = slot[(size_t)qo];
      const cplx* I0 = q0 >= 0 ? slot[(size_t)q0] : nullptr;
      const cplx* I1 = q1 >= 0 ? slot[(size_t)q1] : nullptr;
      switch (t.kind) {
        case BSE_OOC_FORM_SUM:
        case BSE_OOC_FORM_DIFF:
          ooc_form_kernel<<<ooc_blocks(nn), 256, 0, st>>>(nn, I0, I1, t.kind == BSE_OOC_FORM_SUM ? 1.0 : -1.0, O,
                                                          status);
          OOC_LAUNCH_CHECK();
          break;
        case BSE_OOC_POTRF: {
          bse_status r = potrf_lower(st, nb, O, nb, Linv, status, BSE_ERR_NOT_PD_AMINUSB);
          if (r) return r;
          ooc_mark_kernel<<<1, 1, 0, st>>>(status, status + 2, BSE_OOC_ROW(t.flags));
          OOC_LAUNCH_CHECK();
          ooc_zero_upper_kernel<<<ooc_blocks(nn), 256, 0, st>>>(nb, O, status);
          OOC_LAUNCH_CHECK();
          ooc_identity_kernel<<<ooc_blocks(nn), 256, 0, st>>>(nb, Xinv);
          OOC_LAUNCH_CHECK();
          r = trsm_lower_conjtrans(st, nb, nb, O, nb, Linv, Xinv, nb, status);  // Xinv = L^{-H}
          if (r) return r;
          break;
        }
        case BSE_OOC_TRSM: {
          // spare = out L^{-H} (upper triangular factor); spare then takes out's place
          GemmParams<cplx> g = gemm_params<cplx>(nb, nb, nb, OPN, O, nb, OPN, Xinv, nb, one, mkc(0.0, 0.0),
                                                 slot[(size_t)spare], nb);
          g.triB = TRI_UP;
          g.status = status;
          bse_status r = gemm_z(st, g);
          if (r) return r;
          break;
        }
        case BSE_OOC_HERK: {
          GemmParams<cplx> g = gemm_params<cplx>(nb, nb, nb, OPN, I0, nb, OPC, I0, nb, mone, one, O, nb);
          g.lowerC = 1;
          g.status = status;
          bse_status r = gemm_z(st, g);
          if (r) return r;
          break;
        }
        case BSE_OOC_GEMM_SUB: {
          GemmParams<cplx> g = gemm_params<cplx>(nb, nb, nb, OPN, I0, nb, OPC, I1, nb, mone, one, O, nb);
          g.status = status;
          bse_status r = gemm_z(st, g);
          if (r) return r;
          break;
        }
        case BSE_OOC_GEMM_ACC: {
          const cplx* Aop = I0;
          int opA = (t.flags & BSE_OOC_IN0_CONJT) ? OPC : OPN;
          int triA = TRI_NONE;
          if (t.flags & BSE_OOC_IN0_HERM) {
            BSE_CUDA(cudaMemcpyAsync(F[si], I0, tile_b, cudaMemcpyDeviceToDevice, st));
            bse_status r = hermitian_fill_upper(st, nb, F[si], nb);
            if (r) return r;
            Aop = F[si];
          } else if (t.flags & BSE_OOC_IN0_LOWER) {
            triA = opA == OPN ? TRI_LO : TRI_UP;  // structure of op(in0)
          }
          GemmParams<cplx> g = gemm_params<cplx>(nb, nb, nb, opA, Aop, nb, OPN, I1, nb, one, one, O, nb);
          g.triA = triA;
          g.triB = (t.flags & BSE_OOC_IN1_LOWER) ? TRI_LO : TRI_NONE;
          g.status = status;
          bse_status r = gemm_z(st, g);
          if (r) return r;
          break;
        }
        default:
          break;
      }
      cudaEvent_t e;
      BSE_CUDA(evp.make(&e));
      BSE_CUDA(cudaEventRecord(e, st));
      hz[(size_t)qw].wr = e;
      hz[(size_t)qw].rd.clear();
      for (int q : {q0, q1})
        if (q >= 0) hz[(size_t)q].rd.push_back(e);
      if (potrf) {
        inv.wr = e;
        inv.rd.clear();
      }
      if (trsm) {
        hz[(size_t)qo].rd.push_back(e);
        inv.rd.push_back(e);
        slot_of[(size_t)t.out] = spare;
        spare = qo;
      }
    }
  }
  // the caller's stream ends after every other stream's last operation
  for (cudaStream_t x : made.v) {
    cudaEvent_t e;
    BSE_CUDA(evp.make(&e));
    BSE_CUDA(cudaEventRecord(e, x));
    BSE_CUDA(cudaStreamWaitEvent(s, e, 0));
  }
  return BSE_OK;
}
