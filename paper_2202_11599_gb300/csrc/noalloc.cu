// nys_hmatvec_noalloc: the fused H-matvec with its scratch memory in a file-scope
// device array instead of a per-call allocation.
//
// Scratch = the per-CTA partial sums of A^T phi(A p) (grid x padded d values of the
// compute type) followed by one status word.  The array is a static __device__
// object: it exists on every GPU that loads this library, for the life of the
// process.  Host code cannot use the array's name as a device address, so the
// address is resolved once per device with cudaGetSymbolAddress (with that device
// current) on the first call made on that device.
#include <mutex>

#include "nys_internal.cuh"

namespace nys {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr size_t kStatusBytes = 256;                          // status word slot

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes + kStatusBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace nys

extern "C" nys_status nys_hmatvec_noalloc(const nys_matrix* A, const double* D, double rho, const void* p,
                                          void* y, void* stream) {
  using namespace nys;
  const nys_status chk = check_hmatvec_args(A, rho, p, y);   // the checks of nys_hmatvec
  if (chk != NYS_OK) return chk;
  ApassPlan plan;
  if (!apass_plan(A, &plan)) return NYS_EINVAL;
  const size_t need = apass_partial_bytes(A, plan);
  if (need > kNoAllocScratchBytes) return NYS_EINVAL;   // larger than the fixed scratch
  unsigned char* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return NYS_ECUDA;
  int* dstat = reinterpret_cast<int*>(scratch + kNoAllocScratchBytes);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(dstat, 0, sizeof(int), st) != cudaSuccess) return NYS_ECUDA;
  ApassArgs a;
  a.A = A->data;
  a.n = A->n;
  a.d = A->d;
  a.ld = A->ld;
  a.dtype = A->dtype;
  a.col_scale = A->col_scale;
  a.p = p;
  a.D = D;
  a.b = nullptr;
  a.D_out = nullptr;
  a.t_out = nullptr;
  a.mode = D ? MODE_DIAG : MODE_ID;
  if (apass_run(a, plan, scratch, nullptr, dstat, st, /*allow_stats=*/false) != cudaSuccess) return NYS_ECUDA;
  if (apass_reduce(a, plan, scratch, rho, y, nullptr, 0, st) != cudaSuccess) return NYS_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return NYS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NYS_ECUDA;
  return h ? (nys_status)h : NYS_OK;
}
