// Event-based profiler (see prof.cuh).
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "prof.cuh"

long long bse_total_launches();

struct Profiler {
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int kind;  // 0 stage, 1 gemm, 2 named launch, 3 tensor-core product kernel
    int stage;
    double flops;
    cudaEvent_t a, b;
    const char* name;
  };
  int fine = 0;
  cudaEvent_t launch_a = nullptr;
  std::map<std::string, std::pair<long long, double>> per_kernel;
  std::vector<Rec> open_stage[BSE_NSTAGES];
  std::vector<Rec> done;
  bse_profile_data acc;
  long long launches0 = 0;
  cudaEvent_t gemm_a = nullptr;
  cudaEvent_t tc_a = nullptr;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
};

static thread_local Profiler* g_cur = nullptr;

Profiler* prof_new() {
  Profiler* p = new Profiler();
  prof_reset(p);
  return p;
}

void prof_delete(Profiler* p) {
  if (!p) return;
  for (auto e : p->pool) cudaEventDestroy(e);
  for (auto& r : p->done) cudaEventDestroy(r.a), cudaEventDestroy(r.b);
  delete p;
}

void prof_reset(Profiler* p) {
  memset(&p->acc, 0, sizeof(p->acc));
  p->per_kernel.clear();
  p->launches0 = bse_total_launches();
}

void prof_set_current(Profiler* p) { g_cur = p; }
Profiler* prof_current() { return g_cur; }

void prof_stage_begin(int stage, cudaStream_t s) {
  Profiler* p = g_cur;
  if (!p) return;
  Profiler::Rec r{0, stage, 0.0, p->get(), nullptr, nullptr};
  if (r.a) cudaEventRecord(r.a, s);
  p->open_stage[stage].push_back(r);
}

void prof_stage_end(int stage, cudaStream_t s) {
  Profiler* p = g_cur;
  if (!p || p->open_stage[stage].empty()) return;
  Profiler::Rec r = p->open_stage[stage].back();
  p->open_stage[stage].pop_back();
  r.b = p->get();
  if (r.b) cudaEventRecord(r.b, s);
  p->done.push_back(r);
}

void prof_gemm_begin(cudaStream_t s) {
  Profiler* p = g_cur;
  if (!p) return;
  p->gemm_a = p->get();
  if (p->gemm_a) cudaEventRecord(p->gemm_a, s);
}

void prof_gemm_end(cudaStream_t s, double flops) {
  Profiler* p = g_cur;
  if (!p || !p->gemm_a) return;
  Profiler::Rec r{1, 0, flops, p->gemm_a, p->get(), nullptr};
  if (r.b) cudaEventRecord(r.b, s);
  p->gemm_a = nullptr;
  p->done.push_back(r);
}

void prof_tc_begin(cudaStream_t s) {
  Profiler* p = g_cur;
  if (!p) return;
  p->tc_a = p->get();
  if (p->tc_a) cudaEventRecord(p->tc_a, s);
}

void prof_tc_end(cudaStream_t s, double flops) {
  Profiler* p = g_cur;
  if (!p || !p->tc_a) return;
  Profiler::Rec r{3, 0, flops, p->tc_a, p->get(), nullptr};
  if (r.b) cudaEventRecord(r.b, s);
  p->tc_a = nullptr;
  p->done.push_back(r);
}

bool prof_fine() { return g_cur && g_cur->fine; }
void prof_set_fine(Profiler* p, int fine) { p->fine = fine; }

void prof_launch_begin(cudaStream_t s) {
  Profiler* p = g_cur;
  if (!p || !p->fine) return;
  p->launch_a = p->get();
  if (p->launch_a) cudaEventRecord(p->launch_a, s);
}

void prof_launch_end(cudaStream_t s, const char* name) {
  Profiler* p = g_cur;
  if (!p || !p->fine || !p->launch_a) return;
  Profiler::Rec r{2, 0, 0.0, p->launch_a, p->get(), name};
  if (r.b) cudaEventRecord(r.b, s);
  p->launch_a = nullptr;
  p->done.push_back(r);
}

int prof_kernel_summary(Profiler* p, char* buf, size_t len) {
  std::string out;
  for (auto& kv : p->per_kernel) {
    char line[256];
    snprintf(line, sizeof line, "%s %lld %.4f\n", kv.first.c_str(), kv.second.first, kv.second.second);
    out += line;
  }
  if (buf && len) {
    const size_t nb = out.size() < len - 1 ? out.size() : len - 1;
    memcpy(buf, out.data(), nb);
    buf[nb] = 0;
  }
  return (int)out.size();
}

void prof_flush(Profiler* p) {
  if (!p) return;
  for (auto& r : p->done) {
    float ms = 0.f;
    if (r.a && r.b && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      if (r.kind == 2) {
        auto& e = p->per_kernel[r.name];
        e.first += 1;
        e.second += ms;
      } else if (r.kind == 0) {
        p->acc.stage_ms[r.stage] += ms;
        p->acc.stage_calls[r.stage] += 1;
      } else if (r.kind == 3) {
        p->acc.tc_ms += ms;
        p->acc.tc_flops += r.flops;
        p->acc.tc_launches += 1;
      } else {
        p->acc.gemm_ms += ms;
        p->acc.gemm_flops += r.flops;
        p->acc.gemm_launches += 1;
      }
    } else {
      cudaGetLastError();
    }
    if (r.a) p->pool.push_back(r.a);
    if (r.b) p->pool.push_back(r.b);
  }
  p->done.clear();
}

void prof_read(Profiler* p, bse_profile_data* out) {
  *out = p->acc;
  out->launches = bse_total_launches() - p->launches0;
}
