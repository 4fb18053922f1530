// Per-device runtime state of the library.
//
// One process may drive several GPUs (one host thread per device, or one thread
// that switches devices).  Every attribute, cache and stream the library keeps
// across calls is therefore keyed by the device that is current at the call:
// kernel attributes are per (kernel, device), SM counts per device, and the
// private capture streams per (host thread, device).
#include <mutex>
#include <set>
#include <utility>

#include "nys_internal.cuh"
#include "solver.cuh"

namespace nys {
namespace {
std::mutex g_rt_mu;
std::set<std::pair<const void*, int>> g_attr_done;   // (kernel, device) with the smem attribute set
int g_sms[kMaxDevices] = {};
}  // namespace

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return dev;
}

int sm_count() {
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return 1;
  std::lock_guard<std::mutex> lk(g_rt_mu);
  if (g_sms[dev] <= 0) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 1;
    g_sms[dev] = c;
  }
  return g_sms[dev];
}

cudaError_t ensure_max_dyn_smem(const void* fn, int bytes) {
  const int dev = current_device();
  if (dev < 0) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_rt_mu);
  const auto key = std::make_pair(fn, dev);
  if (g_attr_done.count(key)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_attr_done.insert(key);
  return e;
}

cudaStream_t capture_stream() {
  static thread_local cudaStream_t streams[kMaxDevices] = {};
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev] = nullptr;
  return streams[dev];
}

cudaStream_t side_stream() {
  static thread_local cudaStream_t streams[kMaxDevices] = {};
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev] = nullptr;
  return streams[dev];
}

ShardComm& shard_comm() {
  static thread_local ShardComm c;
  return c;
}

nys_status shard_sum(void* buf, int64_t count, int dtype, cudaStream_t st) {
  const ShardComm& c = shard_comm();
  if (!c.fn || count <= 0) return NYS_OK;
  return (nys_status)c.fn(buf, count, dtype, reinterpret_cast<void*>(st), c.ctx);
}

ShardScope::ShardScope(const nys_opts* o) : saved(shard_comm()) {
  shard_comm().fn = o ? o->allreduce : nullptr;
  shard_comm().ctx = o ? o->allreduce_ctx : nullptr;
}
ShardScope::~ShardScope() { shard_comm() = saved; }

}  // namespace nys
