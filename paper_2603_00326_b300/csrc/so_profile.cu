// so_profile.cu -- per-stage CUDA-event timers and the kernel-launch counter.
//
// When enabled, every launch group records a start / stop event pair on its
// stream; so_profile_read() waits for the recorded pairs, sums the elapsed
// time per stage name and resets.  The launch counter is always on.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "so_internal.h"

namespace sof {
namespace {
struct Pair {
  int stage;
  cudaEvent_t a, b;
};
struct Stage {
  std::string name;
  long long launches = 0;
  double ms = 0.0;
};
std::atomic<long long> g_launches{0};
std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<Pair> g_pending;
std::vector<cudaEvent_t> g_pool;
std::vector<Stage> g_stages;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
int stage_id(const char* name) {
  for (size_t i = 0; i < g_stages.size(); ++i)
    if (g_stages[i].name == name) return (int)i;
  g_stages.push_back(Stage{name, 0, 0.0});
  return (int)g_stages.size() - 1;
}
}  // namespace

bool profiling_on() { return g_on.load(std::memory_order_relaxed) != 0; }

ProfScope::ProfScope(const char* name, cudaStream_t st, int launches) : st_(st) {
  g_launches.fetch_add(launches, std::memory_order_relaxed);
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  stage_ = stage_id(name);
  g_stages[stage_].launches += launches;
  a_ = get_event();
  b_ = get_event();
  if (a_ && b_) cudaEventRecord(a_, st);
}

ProfScope::~ProfScope() {
  if (stage_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (a_ && b_) {
    cudaEventRecord(b_, st_);
    g_pending.push_back(Pair{stage_, a_, b_});
  }
}

}  // namespace sof

using namespace sof;

extern "C" {

void so_profile_enable(int on) { g_on.store(on ? 1 : 0); }

long long so_launch_count(void) { return g_launches.load(); }

int so_profile_read(so_profile_entry* out, int max_entries) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (const Pair& p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
      g_stages[p.stage].ms += ms;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
  int k = 0;
  for (const Stage& s : g_stages) {
    if (k >= max_entries) break;
    memset(out[k].name, 0, sizeof(out[k].name));
    strncpy(out[k].name, s.name.c_str(), sizeof(out[k].name) - 1);
    out[k].launches = s.launches;
    out[k].total_ms = s.ms;
    ++k;
  }
  g_stages.clear();
  return k;
}

}  // extern "C"
