// Gaussian test matrix Omega ~ N(0,1) (App. B: Alg. Randomized Nystrom Approximation draws
// Omega with independent standard normal entries), generated on the device by the
// counter-based generator Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011) and the Box-Muller transform.
//
// Element e = i + j d of the column-major d x s panel is member e mod 2 of pair m = e / 2:
//   counter (lo32(m), hi32(m), 0, 0), key (lo32(seed), hi32(seed)) -> words w0..w3,
//   u1 = (((w0 2^32 + w1) >> 11) + 1) 2^-53 in (0, 1],  u2 = ((w2 2^32 + w3) >> 11) 2^-53 in [0, 1),
//   element 2m = sqrt(-2 ln u1) cos(2 pi u2), element 2m + 1 = sqrt(-2 ln u1) sin(2 pi u2).
// Every element is a pure function of (seed, e): any thread order gives the same panel.
#include <algorithm>

#include "nys_internal.cuh"

namespace nys {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   // round multipliers
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   // key-schedule increments
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

__global__ void gaussian_panel_kernel(uint64_t seed, int64_t n, double* __restrict__ out) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const int64_t pairs = (n + 1) / 2;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < pairs; m += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)m, (uint32_t)((uint64_t)m >> 32), 0u, 0u), key);
    const uint64_t a = (((uint64_t)w.x << 32) | w.y) >> 11;
    const uint64_t b = (((uint64_t)w.z << 32) | w.w) >> 11;
    const double u1 = (double)(a + 1) * 0x1p-53;
    const double u2 = (double)b * 0x1p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[2 * m] = r * cs;
    if (2 * m + 1 < n) out[2 * m + 1] = r * sn;
  }
}

cudaError_t gaussian_panel(uint64_t seed, int64_t d, int s, double* Omega, cudaStream_t st) {
  const int64_t n = d * (int64_t)s;
  const int64_t pairs = (n + 1) / 2;
  const int blocks = (int)std::min<int64_t>((pairs + 255) / 256, 8 * (int64_t)sm_count());
  count_launch();
  gaussian_panel_kernel<<<std::max(1, blocks), 256, 0, st>>>(seed, n, Omega);
  return cudaGetLastError();
}

}  // namespace nys
