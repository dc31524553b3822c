// Per-kernel timing of the library's launches with CUDA events (host side, off by default).
//
// When enabled (tmamg_profile_enable), every instrumented launch site records a pair of events
// on the stream it launches on; tmamg_profile_report synchronises those events and returns, per
// kernel name, the number of launches and their summed device time. The events order with the
// launches on the same stream, so the times are the kernels' own durations plus the (small)
// event gaps between them; nothing is recorded while profiling is off.
#pragma once
#include <cuda_runtime.h>

namespace tmamg {

bool profile_on();
void profile_begin(cudaStream_t st, const char* name, cudaEvent_t* ev);
void profile_end(cudaStream_t st, const char* name, cudaEvent_t ev);

struct ProfScope {
  cudaStream_t st;
  const char* name;
  cudaEvent_t ev = nullptr;
  ProfScope(cudaStream_t s, const char* n) : st(s), name(n) {
    if (profile_on()) profile_begin(st, name, &ev);
  }
  ~ProfScope() {
    if (ev) profile_end(st, name, ev);
  }
};

}  // namespace tmamg

#define TM_PROF(st, name) ::tmamg::ProfScope _tm_prof_scope_(st, name)
