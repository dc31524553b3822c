// Per-kernel CUDA-event timing of the library's launches (see profile.cuh).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace tmamg {

namespace {
std::atomic<bool> g_on{false};
std::mutex g_mu;
struct Pending {
  std::string name;
  cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;  // recycled events
struct Total {
  long long count = 0;
  double ms = 0.0;
};
std::map<std::string, Total> g_total;

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// fold completed event pairs into the totals (the caller holds g_mu); with wait, every pair
void drain(bool wait) {
  size_t keep = 0;
  for (size_t i = 0; i < g_pending.size(); ++i) {
    Pending& p = g_pending[i];
    if (!wait && cudaEventQuery(p.b) != cudaSuccess) {
      g_pending[keep++] = p;
      continue;
    }
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      Total& t = g_total[p.name];
      t.count += 1;
      t.ms += ms;
    }
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.resize(keep);
}
}  // namespace

bool profile_on() { return g_on.load(std::memory_order_relaxed); }

void profile_begin(cudaStream_t st, const char* name, cudaEvent_t* ev) {
  std::lock_guard<std::mutex> lk(g_mu);
  (void)name;
  *ev = take_event();
  cudaEventRecord(*ev, st);
}

void profile_end(cudaStream_t st, const char* name, cudaEvent_t ev) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st);
  g_pending.push_back(Pending{name, ev, b});
  if (g_pending.size() > 4096) drain(false);
}

}  // namespace tmamg

using namespace tmamg;

extern "C" {

int tmamg_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain(true);
  g_total.clear();
  g_on.store(on != 0);
  return TMAMG_OK;
}

int tmamg_profile_report(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain(true);
  std::string s = "{";
  bool first = true;
  for (const auto& kv : g_total) {
    char item[256];
    snprintf(item, sizeof(item), "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.count,
             kv.second.ms);
    s += item;
    first = false;
  }
  s += "}";
  if (!buf || len < s.size() + 1) return TMAMG_ERR_ARG;
  memcpy(buf, s.c_str(), s.size() + 1);
  return (int)s.size();
}

}  // extern "C"
