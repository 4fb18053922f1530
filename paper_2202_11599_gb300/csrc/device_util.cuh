// Device helpers: storage traits, mbarrier / TMA bulk-copy wrappers with bounded
// waits, warp and block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nys_internal.cuh"

namespace nys {

// Upper bound on any device-side wait (cycles of clock64, ~2 s at 2 GHz).
constexpr long long kWaitCycles = 4000000000LL;

template <int DT> struct Stor;
template <> struct Stor<NYS_F64> {
  using C = double;
  static constexpr int VEC = 2;
  static constexpr int ESZ = 8;
};
template <> struct Stor<NYS_F32> {
  using C = float;
  static constexpr int VEC = 4;
  static constexpr int ESZ = 4;
};
template <> struct Stor<NYS_BF16> {
  using C = float;
  static constexpr int VEC = 8;
  static constexpr int ESZ = 2;
};
template <> struct Stor<NYS_FP8E4M3> {
  using C = float;
  static constexpr int VEC = 16;
  static constexpr int ESZ = 1;
};

// Unpack one 16-byte vector of stored elements into compute values.
template <int DT>
__device__ __forceinline__ void unpack16(const uint4 r, typename Stor<DT>::C* o);
template <>
__device__ __forceinline__ void unpack16<NYS_F64>(const uint4 r, double* o) {
  o[0] = __hiloint2double((int)r.y, (int)r.x);
  o[1] = __hiloint2double((int)r.w, (int)r.z);
}
template <>
__device__ __forceinline__ void unpack16<NYS_F32>(const uint4 r, float* o) {
  o[0] = __uint_as_float(r.x);
  o[1] = __uint_as_float(r.y);
  o[2] = __uint_as_float(r.z);
  o[3] = __uint_as_float(r.w);
}
template <>
__device__ __forceinline__ void unpack16<NYS_BF16>(const uint4 r, float* o) {
  o[0] = __uint_as_float(r.x << 16);
  o[1] = __uint_as_float(r.x & 0xffff0000u);
  o[2] = __uint_as_float(r.y << 16);
  o[3] = __uint_as_float(r.y & 0xffff0000u);
  o[4] = __uint_as_float(r.z << 16);
  o[5] = __uint_as_float(r.z & 0xffff0000u);
  o[6] = __uint_as_float(r.w << 16);
  o[7] = __uint_as_float(r.w & 0xffff0000u);
}

// Load element j of a stored row as a compute value (scalar path for tails / GEMMs).
template <int DT>
__device__ __forceinline__ typename Stor<DT>::C load_elem(const void* base, int64_t idx);
template <>
__device__ __forceinline__ double load_elem<NYS_F64>(const void* base, int64_t idx) {
  return __ldg(reinterpret_cast<const double*>(base) + idx);
}
template <>
__device__ __forceinline__ float load_elem<NYS_F32>(const void* base, int64_t idx) {
  return __ldg(reinterpret_cast<const float*>(base) + idx);
}
template <>
__device__ __forceinline__ float load_elem<NYS_BF16>(const void* base, int64_t idx) {
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short*>(base) + idx);
  return __uint_as_float(((unsigned)h) << 16);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Plain arrive (release at CTA scope): publishes the arriving thread's prior writes.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// 1-D TMA bulk copy global -> shared, completion signalled on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 policy for data streamed once (the rows of A in the fused pass): evict first, so
// that the small vectors and U the other kernels of an iteration reuse stay in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// tma_load_1d with an L2 cache-policy hint
__device__ __forceinline__ void tma_load_1d_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
      "%4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: returns false if the phase did not complete within `cycles` clock64 ticks
// (default kWaitCycles).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long cycles = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > cycles) return false;
  }
  return true;
}

// Grid-wide barrier of a co-resident grid (cooperative launch): an arrival counter and a
// generation word in global memory.  The last block to arrive resets the counter and
// advances the generation; the others wait for the generation to change, at most
// `cycles` clock64 ticks.  Thread 0 arrives with an acquire-release atomic after the block's
// __syncthreads (which orders the block's writes before it) and waits with acquire loads,
// so no full memory fence is needed (measured: 2.4 -> 1.6 us per barrier on 40 blocks).  Every thread of every block calls it; returns false (in every
// thread of the block) when the wait ran out.  Data another block wrote before the barrier
// is read after it through L2 (__ldcg / .cg loads): this SM's L1 may still hold the line
// from before (measured: plain loads returned stale values).
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks,
                                             long long cycles = kWaitCycles) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    unsigned g, old;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gen) : "memory");
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(count), "r"(1u) : "memory");
    if (old == nblocks - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" :: "l"(count), "r"(0u) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(gen), "r"(1u) : "memory");
    } else {
      const long long t0 = clock64();
      for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(gen) : "memory");
        if (v != g) break;
        if (clock64() - t0 > cycles) {
          ok = 0;
          break;
        }
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}

// Grid barrier on one monotonic counter: every block adds 1 and waits until the counter
// reaches `target` (= blocks x barriers passed so far, kept by the caller; the counter
// starts at 0 and wraps harmlessly).  One release add per block and acquire polls (no reset
// write), so it costs about one L2 round trip less than grid_barrier.  Same memory rules: data that
// other blocks wrote before the barrier is read through L2 (__ldcg) after it.
// `sleep_ns` > 0 spaces the polls: blocks that arrive long before the last one (the end of an
// A-pass) would otherwise keep one L2 line busy while the others still stream A.
__device__ __forceinline__ bool grid_barrier_mono(unsigned* count, unsigned target, long long cycles = kWaitCycles,
                                                  unsigned sleep_ns = 0) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(count), "r"(1u) : "memory");
    const long long t0 = clock64();
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if ((int)(v - target) >= 0) break;
      if (sleep_ns) __nanosleep(sleep_ns);
      if (clock64() - t0 > cycles) {
        ok = 0;
        break;
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in fixed order (deterministic), result in thread 0 only: the other threads
// skip the final cross-warp adds (the FP64 pipe is narrow: one warp instruction occupies it
// for many cycles).  Thread 0 adds in the order of block_sum, so the value is the same.
template <int NT>
__device__ __forceinline__ double block_sum_t0(double v, double* sh /* >= NT/32 */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += sh[i];
  }
  return s;
}

// Block-wide sum in fixed order (deterministic); every thread gets the result.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh /* >= NT/32 */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s += sh[i];
  return s;
}

// Loads a thread keeps in flight in the batched sums below: 256 bytes of registers.
template <typename T>
constexpr int kLoadBatch = sizeof(T) == 4 ? 64 : 32;

// sum_{g < n} a[g * stride + j] added in increasing g (the order of a plain loop), the loads
// issued kLoadBatch at a time so that a thread keeps that many reads in flight.  CG: read
// through L2, for data written by other blocks of the running kernel.
template <bool CG, typename T>
__device__ __forceinline__ T sum_strided_fixed(const T* a, int n, int64_t stride, int64_t j, T s) {
  constexpr int B = kLoadBatch<T>;
  for (int g = 0; g < n; g += B) {
    T v[B];
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (g + q < n) {
        const T* ptr = a + (int64_t)(g + q) * stride + j;
        v[q] = CG ? __ldcg(ptr) : *ptr;
      }
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (g + q < n) s += v[q];
  }
  return s;
}

// acc + sum_{i < s} U[i * d + j] g[i] as one fma chain in increasing i (the row of U g, for
// y = w + U g), the loads of U issued kLoadBatch at a time.
template <typename C>
__device__ __forceinline__ C urow_dot(const C* __restrict__ U, int64_t d, int64_t j, int s, const C* g, C acc) {
  constexpr int B = kLoadBatch<C>;
  for (int i = 0; i < s; i += B) {
    C u[B];
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (i + q < s) u[q] = U[(int64_t)(i + q) * d + j];
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (i + q < s) acc = fma(u[q], g[i + q], acc);
  }
  return acc;
}

}  // namespace nys
