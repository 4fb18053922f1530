// Instrumentation behind nys_stats_enable / nys_stats_read: a process-wide count
// of kernel launches and, while enabled, CUDA-event timing of every fused A-pass
// launch on the stream it is launched on.
#include <atomic>
#include <mutex>
#include <utility>
#include <vector>
#include <algorithm>

#include "device_util.cuh"
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
constexpr int kTimerCap = 1 << 18;
DevTimer g_timer;            // device buffers of the in-kernel timer (allocated on first enable)
bool g_timer_on = false;
}  // namespace

thread_local bool g_count_suspended = false;
void count_launch() {
  if (!g_count_suspended) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_launch_suspend(bool on) { g_count_suspended = on; }
bool launch_capturing() { return g_count_suspended; }
void count_launch_add(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool stats_enabled() { return g_enabled.load(std::memory_order_relaxed); }

DevTimer stats_device_timer() {
  if (!g_timer_on) return DevTimer{};
  return g_timer;
}

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
  if (on && !g_timer.count) {
    const size_t cap = kTimerCap;
    bool ok = cudaMalloc(&g_timer.start, cap * 8) == cudaSuccess && cudaMalloc(&g_timer.end, cap * 8) == cudaSuccess &&
              cudaMalloc(&g_timer.bytes, cap * 8) == cudaSuccess && cudaMalloc(&g_timer.dtype, cap * 4) == cudaSuccess &&
              cudaMalloc(&g_timer.count, 8) == cudaSuccess;
    if (ok) {
      g_timer.done = g_timer.count + 1;
      g_timer.cap = kTimerCap;
    } else {
      g_timer = DevTimer{};
    }
  }
  if (g_timer.count) {
    cudaMemset(g_timer.start, 0xff, (size_t)g_timer.cap * 8);
    cudaMemset(g_timer.end, 0, (size_t)g_timer.cap * 8);
    cudaMemset(g_timer.count, 0, 8);
  }
  g_timer_on = on != 0 && g_timer.count != nullptr;
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
  for (int k = 0; k < 4; ++k) {
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
    const int k = (r.dtype >= 0 && r.dtype < 4) ? r.dtype : 0;
    out->apass_launches[k] += 1;
    out->apass_ms[k] += t;
    out->apass_bytes[k] += r.bytes;
  }
  out->launches = g_launches.load();
  for (int k = 0; k < 4; ++k) {
    out->dev_launches[k] = 0;
    out->dev_ms[k] = 0.0;
    out->dev_bytes[k] = 0.0;
  }
  if (g_timer.count) {
    int cnt = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return NYS_ECUDA;
    if (cudaMemcpy(&cnt, g_timer.count, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NYS_ECUDA;
    cnt = std::min(cnt, g_timer.cap);
    std::vector<unsigned long long> t0(cnt), t1(cnt);
    std::vector<double> by(cnt);
    std::vector<int> dt(cnt);
    if (cnt > 0 &&
        (cudaMemcpy(t0.data(), g_timer.start, cnt * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(t1.data(), g_timer.end, cnt * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(by.data(), g_timer.bytes, cnt * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(dt.data(), g_timer.dtype, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess))
      return NYS_ECUDA;
    for (int i = 0; i < cnt; ++i) {
      const int k = (dt[i] >= 0 && dt[i] < 4) ? dt[i] : 0;
      if (t1[i] < t0[i]) continue;
      out->dev_launches[k] += 1;
      out->dev_ms[k] += (double)(t1[i] - t0[i]) * 1e-6;
      out->dev_bytes[k] += by[i];
    }
  }
  return NYS_OK;
}

// Diagnostic: one CTA whose thread 0 waits, with the bounded mbarrier wait every kernel of
// the library uses, on a barrier that expects two arrivals and receives one, so the wait
// must run out; the kernel then reports NYS_ETIMEOUT the way the passes do.
__global__ void wait_bound_check_kernel(long long cycles, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    nys::mbar_init(&bar, 2);
    nys::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(nys::smem_u32(&bar)) : "memory");
    const bool ok = nys::mbar_wait_bounded(&bar, 0u, cycles);
    *status = ok ? (int)NYS_OK : (int)NYS_ETIMEOUT;
  }
}

nys_status nys_check_wait_bound(double wait_us, void* stream) {
  if (!(wait_us > 0.0) || wait_us > 5e6) return NYS_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NYS_ECUDA;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) {
    cudaGetLastError();
    khz = 2000000;  // the bound is in clock ticks; ~2 GHz when the rate is not reported
  }
  const long long cycles = (long long)(wait_us * 1e-3 * khz);
  int* d_status = nullptr;
  if (cudaMallocAsync(&d_status, sizeof(int), st) != cudaSuccess) return NYS_ENOMEM;
  int h = -1;
  nys::count_launch();
  wait_bound_check_kernel<<<1, 32, 0, st>>>(cycles, d_status);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d_status, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return NYS_ECUDA;
  return (nys_status)h;
}

}  // extern "C"
