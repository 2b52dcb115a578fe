// Event-based profiler behind bse_profile_enable / bse_profile_read.  The
// solve entry points make a handle's profiler current for the calling host
// thread; stage guards and the GEMM engine record CUDA events on the solve's
// stream while one is current, and prof_flush turns them into times after
// the stream has been synchronised.
#pragma once
#include "common.cuh"

struct Profiler;
Profiler* prof_new();
void prof_delete(Profiler* p);
void prof_reset(Profiler* p);
void prof_set_current(Profiler* p);  // NULL: profiling off for this thread
Profiler* prof_current();
void prof_stage_begin(int stage, cudaStream_t s);
void prof_stage_end(int stage, cudaStream_t s);
void prof_gemm_begin(cudaStream_t s);
void prof_gemm_end(cudaStream_t s, double flops);
// the tensor-core product kernel inside a split-operand product
void prof_tc_begin(cudaStream_t s);
void prof_tc_end(cudaStream_t s, double flops);
// fine level: every wrapped launch timed and accumulated under its name
bool prof_fine();
void prof_launch_begin(cudaStream_t s);
void prof_launch_end(cudaStream_t s, const char* name);
void prof_set_fine(Profiler* p, int fine);
int prof_kernel_summary(Profiler* p, char* buf, size_t len);
void prof_flush(Profiler* p);  // after the stream is synchronised
void prof_read(Profiler* p, bse_profile_data* out);

struct StageScope {
  int stage;
  cudaStream_t s;
  StageScope(int st, cudaStream_t ss) : stage(st), s(ss) { prof_stage_begin(stage, s); }
  ~StageScope() { prof_stage_end(stage, s); }
};
