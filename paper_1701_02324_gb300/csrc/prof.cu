// prof.cu -- launch counter and event-based phase timing (see prof.cuh).
#include <atomic>
#include <mutex>
#include <vector>

#include "kf_internal.cuh"
#include "prof.cuh"

namespace {
struct Rec {
  int phase;
  cudaEvent_t a, b;
};
std::mutex g_mu;
std::atomic<long long> g_launches{0};
std::atomic<int> g_on{0};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
thread_local cudaEvent_t t_open = nullptr;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void kf_prof_begin(int, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  t_open = get_event();
  cudaEventRecord(t_open, s);
}

void kf_prof_end(int phase, cudaStream_t s) {
  if (!g_on.load(std::memory_order_relaxed) || !t_open) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  cudaEventRecord(b, s);
  g_recs.push_back({phase, t_open, b});
  t_open = nullptr;
}

extern "C" {

int64_t kf_launch_count(void) { return g_launches.load(); }

kf_status kf_profile_enable(int32_t on) {
  g_on.store(on ? 1 : 0);
  return KF_OK;
}

kf_status kf_profile_read(double* ms, int64_t* launches, int32_t nphase) {
  if (!ms || !launches || nphase < KF_PH_COUNT) return KF_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < nphase; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  kf_status st = KF_OK;
  for (auto& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) st = KF_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) st = KF_ECUDA;
    ms[r.phase] += t;
    launches[r.phase] += 1;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  cudaGetLastError();
  return st;
}

}  // extern "C"
