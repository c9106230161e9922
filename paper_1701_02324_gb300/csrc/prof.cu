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
  cudaStream_t s;
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

// Inside a stream capture a plain event record only expresses a dependency;
// an external record becomes a node of the graph, so launches in the batched
// graphs are timed too.
void record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}
}  // namespace

void kf_prof_begin(int, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  t_open = get_event();
  record(t_open, s);
}

void kf_prof_end(int phase, cudaStream_t s) {
  if (!g_on.load(std::memory_order_relaxed) || !t_open) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  record(b, s);
  g_recs.push_back({phase, t_open, b, s});
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

kf_status kf_profile_timeline(double* t0_ms, double* t1_ms, int32_t* phase, int32_t* stream, int64_t cap,
                              int64_t* n) {
  if (!t0_ms || !t1_ms || !phase || !stream || !n || cap < 0) return KF_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  *n = (int64_t)g_recs.size();
  if (g_recs.empty()) return KF_OK;
  kf_status st = KF_OK;
  std::vector<cudaStream_t> seen;
  for (int64_t q = 0; q < (int64_t)g_recs.size() && q < cap; ++q) {
    const Rec& r = g_recs[q];
    if (cudaEventSynchronize(r.b) != cudaSuccess) st = KF_ECUDA;
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, g_recs[0].a, r.a) != cudaSuccess) st = KF_ECUDA;
    if (cudaEventElapsedTime(&b, g_recs[0].a, r.b) != cudaSuccess) st = KF_ECUDA;
    t0_ms[q] = a;
    t1_ms[q] = b;
    phase[q] = r.phase;
    int si = 0;
    while (si < (int)seen.size() && seen[si] != r.s) ++si;
    if (si == (int)seen.size()) seen.push_back(r.s);
    stream[q] = si;
  }
  cudaGetLastError();
  return st;
}

}  // extern "C"
