// Launch-shape autotuner (see autotune.cuh).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "autotune.cuh"
#include "common.cuh"

namespace tmamg {

namespace {
std::atomic<bool> g_on{true};
std::atomic<int> g_force{-1};
std::mutex g_mu;
struct Entry {
  int choice = -1;
  std::vector<float> ms;  // mean time of each variant
};
std::map<std::tuple<int, std::string, int64_t>, Entry> g_table;

int device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}
}  // namespace

bool autotune_on() { return g_on.load(std::memory_order_relaxed); }

int tune_forced() { return g_force.load(std::memory_order_relaxed); }

int tune_lookup(const char* family, int64_t key) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(std::make_tuple(device(), std::string(family), key));
  return it == g_table.end() ? -1 : it->second.choice;
}

int tune_run(const char* family, int64_t key, int nvar, const std::function<void(int)>& launch, cudaStream_t st) {
  std::vector<float> ms(nvar, 0.f);
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return 0;
  }
  int best = 0;
  for (int v = 0; v < nvar; ++v) {
    launch(v);  // warm-up (first launch of the variant's kernel)
    cudaEventRecord(a, st);
    launch(v);
    launch(v);
    cudaEventRecord(b, st);
    float t = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess) t = 1e30f;
    ms[v] = 0.5f * t;
    if (ms[v] < ms[best]) best = v;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::lock_guard<std::mutex> lk(g_mu);
  Entry& e = g_table[std::make_tuple(device(), std::string(family), key)];
  e.choice = best;
  e.ms = ms;
  return best;
}

}  // namespace tmamg

using namespace tmamg;

extern "C" {

int tmamg_autotune_force(int variant) {
  g_force.store(variant < 0 ? -1 : variant);
  return TMAMG_OK;
}

int tmamg_autotune(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
  g_on.store(on != 0);
  return TMAMG_OK;
}

int tmamg_autotune_report(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::string s = "{";
  bool first = true;
  for (const auto& kv : g_table) {
    char head[160];
    snprintf(head, sizeof(head), "%s\"%s/dev%d/%lld\": {\"choice\": %d, \"ms\": [", first ? "" : ", ",
             std::get<1>(kv.first).c_str(), std::get<0>(kv.first), (long long)std::get<2>(kv.first),
             kv.second.choice);
    s += head;
    for (size_t i = 0; i < kv.second.ms.size(); ++i) {
      char v[32];
      snprintf(v, sizeof(v), "%s%.4f", i ? ", " : "", kv.second.ms[i]);
      s += v;
    }
    s += "]}";
    first = false;
  }
  s += "}";
  if (!buf || len < s.size() + 1) return TMAMG_ERR_ARG;
  memcpy(buf, s.c_str(), s.size() + 1);
  return (int)s.size();
}

}  // extern "C"
