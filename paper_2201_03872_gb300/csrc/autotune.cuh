// Launch-shape autotuner (host side).
//
// A kernel family offers several launch variants that compute identical results (the same
// per-thread arithmetic under different CTA shapes and register budgets). The first call for a
// problem key (lattice volume and system count) times every variant on that call's own data
// with CUDA events on the call's stream, keeps the fastest and uses it from then on; the
// choices are kept per device for the life of the process. Only idempotent launches are tuned
// (each variant overwrites the same output from unchanged inputs).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

namespace tmamg {

bool autotune_on();
// the variant every tuned family is held to (tmamg_autotune_force), or -1
int tune_forced();
// the variant chosen for (family, key) on the current device, or -1 if not tuned yet
int tune_lookup(const char* family, int64_t key);
// times variants 0..nvar-1 (launch(v) enqueues variant v on st; one warm-up and two timed launches
// each), records the fastest for (family, key) and returns it
int tune_run(const char* family, int64_t key, int nvar, const std::function<void(int)>& launch, cudaStream_t st);

// the variant to use: tuned on first use when tuning is on, else variant 0
inline int tune_pick(const char* family, int64_t key, int nvar, const std::function<void(int)>& launch,
                     cudaStream_t st) {
  const int f = tune_forced();
  if (f >= 0) return f < nvar ? f : 0;
  if (!autotune_on() || nvar < 2) return 0;
  const int v = tune_lookup(family, key);
  return v >= 0 ? v : tune_run(family, key, nvar, launch, st);
}

}  // namespace tmamg
