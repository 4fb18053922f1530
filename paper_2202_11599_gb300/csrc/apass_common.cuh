// Device-side pieces shared by the fused A-pass kernels (apass.cu, apass_ws.cu):
// the kernel argument block, the in-kernel launch timer, the per-row modes phi and
// the unpacking of 16-byte vectors of stored elements.
#pragma once
#include <cuda_fp8.h>

#include "device_util.cuh"
#include "nys_internal.cuh"

namespace nys {

constexpr int kMaxStages = 8;
constexpr int kRMax = 4;
constexpr int kSmemBudget = 200 * 1024;
constexpr int kWsGroupWarps = 8;   // warp-specialised float pass: dot warps = update warps
constexpr int kWs64DotWarps = 8;   // warp-specialised FP64 pass: dot warps (update warps: twice as many)

struct ApassKArgs {
  const unsigned char* A;
  int64_t n, d, ld;
  const void* p;
  const double* D;
  const double* b;
  double* D_out;
  double* t_out;
  int mode;
  int R;          // rows per stage (<= kRMax)
  int S;          // stages
  int64_t dpad;   // partial stride
  void* partial;
  double* loss_part;
  int* status;
  const int* skip;
  int* executed;  // instrumentation: set to 1 by CTA 0 when the pass ran (not skipped)
  DevTimer tm;    // instrumentation: in-kernel launch timing (null pointers when off)
  double bytes_alg;
  const float* col_scale;  // FP8: p is read as col_scale o p (the reduce scales the sums)
  // warp-specialised float pass: CTA c takes rows [row_split[c], row_split[c + 1]) (null: the
  // equal split n c / grid); cta_time (null when off): start and end %globaltimer of CTA c
  // at [2 c] and [2 c + 1], for the row-split calibration
  const int64_t* row_split;
  unsigned long long* cta_time;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int timer_begin(const ApassKArgs& a) {
  int slot = -1;
  if (a.tm.count && threadIdx.x == 0) {
    const int c = *(volatile int*)a.tm.count;
    if (c < a.tm.cap) {
      slot = c;
      atomicMin(&a.tm.start[c], gtimer());
    }
  }
  return slot;
}
// called by every thread of the CTA at the end of a pass that completed
__device__ __forceinline__ void timer_end(const ApassKArgs& a, int slot, int dtype) {
  if (!a.tm.count) return;
  __syncthreads();
  if (threadIdx.x == 0 && slot >= 0) {
    atomicMax(&a.tm.end[slot], gtimer());
    if (blockIdx.x == 0) {
      a.tm.bytes[slot] = a.bytes_alg;
      a.tm.dtype[slot] = dtype;
    }
    __threadfence();
    if (atomicAdd(a.tm.done, 1) == (int)gridDim.x - 1) {
      *a.tm.done = 0;
      __threadfence();
      *(volatile int*)a.tm.count = slot + 1;
    }
  }
}

__device__ __forceinline__ double sigmoid_d(double t) {
  // stable logistic function
  if (t >= 0) {
    const double e = exp(-t);
    return 1.0 / (1.0 + e);
  }
  const double e = exp(t);
  return e / (1.0 + e);
}


// Two consecutive stored elements (pair q of a 16-byte vector) as FP32 values.
template <int DT>
__device__ __forceinline__ float2 unpack_pair(const uint4& r, int q);
template <>
__device__ __forceinline__ float2 unpack_pair<NYS_F32>(const uint4& r, int q) {
  return q == 0 ? make_float2(__uint_as_float(r.x), __uint_as_float(r.y))
                : make_float2(__uint_as_float(r.z), __uint_as_float(r.w));
}
template <>
__device__ __forceinline__ float2 unpack_pair<NYS_BF16>(const uint4& r, int q) {
  const unsigned w = q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// FP8 E4M3: 16-bit half (q & 1) of word q / 2 holds elements 2q and 2q + 1 (the per-column
// scales are folded into p and into the final sum, so only the codes are decoded here).
template <>
__device__ __forceinline__ float2 unpack_pair<NYS_FP8E4M3>(const uint4& r, int q) {
  const unsigned w = (q >> 1) == 0 ? r.x : ((q >> 1) == 1 ? r.y : ((q >> 1) == 2 ? r.z : r.w));
  const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((q & 1) ? (w >> 16) : (w & 0xffffu));
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
  return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

// Zero the stored elements of a 16-byte vector from element index `keep` on.
template <int DT>
__device__ __forceinline__ void mask_tail(uint4& r, int keep) {
  constexpr int ESZ = Stor<DT>::ESZ;
  unsigned* w = reinterpret_cast<unsigned*>(&r);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int first = i * 4 / ESZ;  // first element index held by word i
    if (ESZ == 4) {
      if (first >= keep) w[i] = 0u;
    } else if (ESZ == 1) {  // four 8-bit elements per word
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (first + b >= keep) w[i] &= ~(0xffu << (8 * b));
    } else {  // two 16-bit elements per word
      if (first >= keep) w[i] = 0u;
      else if (first + 1 >= keep) w[i] &= 0x0000ffffu;
    }
  }
}

__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}

// The per-row input of the pass's mode (D_i or b_i), loaded at the start of a step so
// that its latency overlaps the dot products instead of sitting between the barriers.
__device__ __forceinline__ double row_input(const ApassKArgs& a, int64_t i) {
  if (a.mode == MODE_ID) return 0.0;
  if (a.mode == MODE_DIAG) return a.D[i];
  return a.b[i];
}

// Row modes of the pass, applied by the warp that finishes row i: returns u_i.
// `in` is row_input(a, i).
__device__ __forceinline__ float row_phi(const ApassKArgs& a, int64_t i, float t, double in, double& loss) {
  switch (a.mode) {
    case MODE_CONST: return (float)in;
    case MODE_ID: return t;
    case MODE_DIAG: return (float)(in * (double)t);
    case MODE_RESID: {
      const double rr = (double)t - in;
      loss += 0.5 * rr * rr;
      return (float)rr;
    }
    case MODE_LGRAD: {
      const double td = (double)t;
      const double sg = sigmoid_d(td);
      const double b01 = 0.5 * (1.0 + in);
      loss += fmax(td, 0.0) + log1p(exp(-fabs(td))) - b01 * td;
      return (float)(sg - b01);
    }
    default: {  // MODE_LOGIT
      const double td = (double)t;
      const double sg = sigmoid_d(td);
      const double wv = sg * (1.0 - sg);
      const double b01 = 0.5 * (1.0 + in);
      if (a.D_out) a.D_out[i] = wv;
      loss += fmax(td, 0.0) + log1p(exp(-fabs(td))) - b01 * td;
      return (float)(wv * td + b01 - sg);
    }
  }
}


// row_phi in FP64 compute (the FP64 passes): u_i = phi(t_i).
__device__ __forceinline__ double row_phi_d(const ApassKArgs& a, int64_t i, double t, double in, double& loss) {
  switch (a.mode) {
    case MODE_CONST: return in;
    case MODE_ID: return t;
    case MODE_DIAG: return in * t;
    case MODE_RESID: {
      const double rr = t - in;
      loss += 0.5 * rr * rr;
      return rr;
    }
    case MODE_LGRAD: {
      const double sg = sigmoid_d(t);
      const double b01 = 0.5 * (1.0 + in);
      loss += fmax(t, 0.0) + log1p(exp(-fabs(t))) - b01 * t;
      return sg - b01;
    }
    default: {  // MODE_LOGIT
      const double sg = sigmoid_d(t);
      const double wv = sg * (1.0 - sg);
      const double b01 = 0.5 * (1.0 + in);
      if (a.D_out) a.D_out[i] = wv;
      loss += fmax(t, 0.0) + log1p(exp(-fabs(t))) - b01 * t;
      return wv * t + b01 - sg;
    }
  }
}

// Warp-uniform bounded wait: every lane waits on the barrier and the warp agrees on the
// outcome, so a bound that runs out on one lane only cannot split the warp.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
  return __all_sync(0xffffffffu, mbar_wait_bounded(bar, parity)) != 0;
}

// Warp-specialised pass (apass_ws.cu): threads and column vectors per thread of a group for
// a matrix of this storage type and width (false if no instantiation fits), and the launch.
bool apass_ws_layout(int dtype, int64_t d, int* threads, int* vpt);
cudaError_t apass_ws_launch(const ApassKArgs& k, const ApassPlan& plan, int dtype, cudaStream_t st,
                            bool prepare_only);

}  // namespace nys
