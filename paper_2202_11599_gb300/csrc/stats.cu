// Instrumentation behind nys_stats_enable / nys_stats_read: a process-wide count
// of kernel launches and, while enabled, CUDA-event timing of every fused A-pass
// launch on the stream it is launched on.
#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "nys_internal.cuh"

namespace nys {
namespace {
struct EvRec {
  cudaEvent_t start, stop;
  double bytes;
  int dtype;
  int slot;
};
std::atomic<long long> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
std::vector<EvRec> g_recs;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_free;
constexpr size_t kMaxRecords = 1 << 20;
int* g_flags = nullptr;      // device: one "executed" flag per record slot
size_t g_next_slot = 0;
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool stats_enabled() { return g_enabled.load(std::memory_order_relaxed); }

cudaError_t stats_event_pair(cudaEvent_t* a, cudaEvent_t* b, int** executed) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_recs.size() >= kMaxRecords || g_next_slot >= kMaxRecords) return cudaErrorNotReady;
  if (!g_flags) {
    cudaError_t e = cudaMalloc(&g_flags, kMaxRecords * sizeof(int));
    if (e != cudaSuccess) {
      g_flags = nullptr;
      return e;
    }
    e = cudaMemset(g_flags, 0, kMaxRecords * sizeof(int));
    if (e != cudaSuccess) return e;
  }
  *executed = g_flags + g_next_slot;
  if (!g_free.empty()) {
    *a = g_free.back().first;
    *b = g_free.back().second;
    g_free.pop_back();
    return cudaSuccess;
  }
  cudaError_t e = cudaEventCreate(a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(b);
  if (e != cudaSuccess) cudaEventDestroy(*a);
  return e;
}

void stats_record_apass(cudaEvent_t start, cudaEvent_t stop, double bytes, int dtype, int* executed) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({start, stop, bytes, dtype, (int)(executed - g_flags)});
  g_next_slot = g_recs.size();
}

}  // namespace nys

extern "C" {

void nys_stats_enable(int32_t on) {
  using namespace nys;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) g_free.emplace_back(r.start, r.stop);
  if (g_flags && !g_recs.empty()) cudaMemset(g_flags, 0, g_recs.size() * sizeof(int));
  g_recs.clear();
  g_next_slot = 0;
  g_launches.store(0);
  g_enabled.store(on != 0);
}

nys_status nys_stats_read(nys_stats* out) {
  using namespace nys;
  if (!out) return NYS_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int k = 0; k < 3; ++k) {
    out->apass_launches[k] = 0;
    out->apass_ms[k] = 0.0;
    out->apass_bytes[k] = 0.0;
  }
  std::vector<int> ran(g_recs.size(), 0);
  if (!g_recs.empty() &&
      cudaMemcpy(ran.data(), g_flags, g_recs.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return NYS_ECUDA;
  for (size_t i = 0; i < g_recs.size(); ++i) {
    const EvRec& r = g_recs[i];
    if (!ran[r.slot]) continue;  // skipped pass (PCG already converged): no work, not counted
    if (cudaEventSynchronize(r.stop) != cudaSuccess) return NYS_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) return NYS_ECUDA;
    const int k = (r.dtype >= 0 && r.dtype < 3) ? r.dtype : 0;
    out->apass_launches[k] += 1;
    out->apass_ms[k] += t;
    out->apass_bytes[k] += r.bytes;
  }
  out->launches = g_launches.load();
  return NYS_OK;
}

}  // extern "C"
