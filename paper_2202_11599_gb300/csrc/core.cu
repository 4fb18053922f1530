// Sketch GEMMs and the FP64 Nystrom core (App. B, Alg. Randomized Nystrom
// Approximation): Y = A^T D (A Omega), the shift nu = shift_scale * eps(||Y||_2),
// C = chol(Omega^T Y_nu), B = Y_nu C^{-1}, the thin SVD of B through the
// symmetric eigendecomposition of B^T B (parallel cyclic Jacobi), U = B V Sigma^{-1}
// and lam = max(0, Sigma^2 - nu).  Also CholQR2 for the thin QR of Omega.
//
// All s x s work is FP64.  GEMM reductions are split into fixed chunks whose
// partials are summed in a fixed order, so every result is run-to-run
// deterministic.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cuda_fp8.h>

#include "device_util.cuh"
#include "nys_internal.cuh"

#include <algorithm>
#include <vector>

namespace nys {

// ------------------------------------------------------------------ generic small GEMM
// C(m, n) = sum_k a(m, k) b(k, n), column-major operands:
//   transA: a(m,k) = A[k + m*lda]   else a(m,k) = A[m + k*lda];   b(k,n) = B[k + n*ldb]
// Split-K: blockIdx.z handles k in [z*kchunk, min(K,(z+1)*kchunk)); the partial goes to
// Cp + z*M*N (column-major, ld M).  Tile 4 TPX x 4 TPX, TPX^2 threads, 4 x 4 per thread;
// the next GK-deep slab of both operands is loaded into registers while the current one
// is multiplied.  With `sym` (M == N, A == B) blockIdx.x enumerates only the tiles with
// bm <= bn; each C(m, n) sums the same products in the same k order as C(n, m) would, so
// the mirrored lower triangle equals a full computation bit for bit.
constexpr int GT = 64, GK = 16;

template <typename T, int TPX>
__global__ void __launch_bounds__(TPX * TPX) gemm_tile_kernel(const T* __restrict__ A, int64_t lda, bool transA,
                                                              const T* __restrict__ B, int64_t ldb, int M, int N,
                                                              int64_t K, int64_t kchunk, int sym, T* __restrict__ Cp) {
  constexpr int TT = 4 * TPX, NT = TPX * TPX;
  constexpr int LD = (GK * TT + NT - 1) / NT;
  __shared__ T As[GK][TT + 1];
  __shared__ T Bs[GK][TT + 1];
  const int tx = threadIdx.x % TPX, ty = threadIdx.x / TPX;
  int bm = blockIdx.x, bn = blockIdx.y;
  if (sym) {
    int t = blockIdx.x;
    bn = 0;
    while (t > bn) {
      t -= bn + 1;
      ++bn;
    }
    bm = t;
  }
  const int m0 = bm * TT, n0 = bn * TT;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(K, kb + kchunk);
  T ra[LD], rb[LD];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int l = 0; l < LD; ++l) {
      const int idx = threadIdx.x + l * NT;
      ra[l] = T(0);
      rb[l] = T(0);
      if (idx < GK * TT) {
        int kk, mm;
        if (transA) {
          kk = idx % GK;
          mm = idx / GK;
        } else {
          mm = idx % TT;
          kk = idx / TT;
        }
        const int64_t k = k0 + kk;
        const int m = m0 + mm;
        if (k < ke && m < M) ra[l] = transA ? A[k + (int64_t)m * lda] : A[m + k * lda];
        const int nn = idx / GK, kk2 = idx % GK;
        const int64_t k2 = k0 + kk2;
        const int n = n0 + nn;
        if (k2 < ke && n < N) rb[l] = B[k2 + (int64_t)n * ldb];
      }
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int l = 0; l < LD; ++l) {
      const int idx = threadIdx.x + l * NT;
      if (idx < GK * TT) {
        if (transA) As[idx % GK][idx / GK] = ra[l];
        else As[idx / TT][idx % TT] = ra[l];
        Bs[idx % GK][idx / GK] = rb[l];
      }
    }
  };
  T acc[4][4] = {};
  if (kb < ke) load(kb);
  for (int64_t k0 = kb; k0 < ke; k0 += GK) {
    stage();
    __syncthreads();
    if (k0 + GK < ke) load(k0 + GK);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + TPX * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + TPX * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* C = Cp + (int64_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tx + TPX * i, n = n0 + ty + TPX * j;
      if (m < M && n < N) C[m + (int64_t)n * M] = acc[i][j];
    }
}
// C (M x N) = sum_z Cp[z] in a fixed order, compute type T
template <typename T>
__global__ void sum_partials_t_kernel(const T* __restrict__ Cp, int nz, int64_t len, T* __restrict__ C) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int z = 0; z < nz; ++z) s += Cp[z * len + i];
    C[i] = s;
  }
}

// C (M x N) = X^T Y with X (K x M), Y (K x N) column-major (ld K); split over K, fixed-order sum.
template <typename T>
cudaError_t gemm_tn(const T* X, const T* Y, int64_t K, int M, int N, T* C, T* work, cudaStream_t st) {
  const int64_t kc = std::max<int64_t>(256, ((K + 63) / 64 + GK - 1) / GK * GK);
  const int nz = (int)((K + kc - 1) / kc);
  dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT, nz);
  count_launch();
  gemm_tile_kernel<T, 16><<<grid, 256, 0, st>>>(X, K, true, Y, K, M, N, K, kc, 0, work);
  NYS_CUDA_TRY(cudaGetLastError());
  count_launch();
  sum_partials_t_kernel<T><<<(unsigned)std::min<int64_t>(1024, ((int64_t)M * N + 255) / 256), 256, 0, st>>>(
      work, nz, (int64_t)M * N, C);
  return cudaGetLastError();
}
template <typename T>
size_t gemm_tn_work_elems(int64_t K, int M, int N) {
  const int64_t kc = std::max<int64_t>(256, ((K + 63) / 64 + GK - 1) / GK * GK);
  return (size_t)((K + kc - 1) / kc) * M * N;
}
// C (M x N) = B (M x K) V (K x N), column-major
template <typename T>
cudaError_t gemm_nn_t(const T* B, int64_t M, int K, const T* V, int N, T* C, cudaStream_t st) {
  dim3 grid((unsigned)((M + GT - 1) / GT), (N + GT - 1) / GT, 1);
  count_launch();
  gemm_tile_kernel<T, 16><<<grid, 256, 0, st>>>(B, M, false, V, K, (int)M, N, K, K, 0, C);
  return cudaGetLastError();
}
template cudaError_t gemm_tn<float>(const float*, const float*, int64_t, int, int, float*, float*, cudaStream_t);
template cudaError_t gemm_tn<double>(const double*, const double*, int64_t, int, int, double*, double*, cudaStream_t);
template size_t gemm_tn_work_elems<float>(int64_t, int, int);
template size_t gemm_tn_work_elems<double>(int64_t, int, int);
template cudaError_t gemm_nn_t<float>(const float*, int64_t, int, const float*, int, float*, cudaStream_t);
template cudaError_t gemm_nn_t<double>(const double*, int64_t, int, const double*, int, double*, cudaStream_t);

// Gram-type products X^T Y (d x s operands, s x s result) on 40 x 40 tiles (s = 200 and
// 400 tile exactly; the FP64 pipe, not memory, bounds these products, so padded tiles are
// wasted time).  The split over d is sized for about kGramCtas CTAs -- a constant, so
// the summation order, and the result, do not depend on the device -- with chunks of at
// least 128 rows.
constexpr int kGramTpx = 10;
constexpr int kGramTile = 4 * kGramTpx;
constexpr int kGramCtas = 1216;
static int gram_tiles(int s, bool sym) {
  const int tb = (s + kGramTile - 1) / kGramTile;
  return sym ? tb * (tb + 1) / 2 : tb * tb;
}
static int64_t gram_kchunk(int64_t K, int tiles) {
  const int64_t nz0 = std::max<int64_t>(1, kGramCtas / tiles);
  const int64_t kc = ((K + nz0 - 1) / nz0 + GK - 1) / GK * GK;
  return std::max<int64_t>(128, kc);
}

size_t gram_work_bytes(int64_t d, int s) {
  int64_t nz = 1;
  for (int sym = 0; sym < 2; ++sym) {
    const int64_t kc = gram_kchunk(d, gram_tiles(s, sym != 0));
    nz = std::max<int64_t>(nz, (d + kc - 1) / kc);
  }
  return (size_t)nz * s * s * sizeof(double);
}

// C = sum_z Cp[z] (fixed order); with `sym` the entries below the diagonal tiles are read
// from their mirror (the tiles there were not computed).
__global__ void sum_partials_gram_kernel(const double* __restrict__ Cp, int nz, int s, int sym,
                                         double* __restrict__ C) {
  const int64_t len = (int64_t)s * s;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < len;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % s), j = (int)(idx / s);
    const int64_t src = (sym && i / kGramTile > j / kGramTile) ? j + (int64_t)i * s : idx;
    double acc = 0.0;
    for (int z = 0; z < nz; ++z) acc += Cp[z * len + src];
    C[idx] = acc;
  }
}

// C (s x s) = X^T Y, X and Y d x s column-major (ld d); symmetric form when X == Y
cudaError_t gram_xty(const double* X, const double* Y, int64_t d, int s, double* C, double* work,
                     cudaStream_t st) {
  const bool sym = X == Y;
  const int tiles = gram_tiles(s, sym);
  const int64_t kc = gram_kchunk(d, tiles);
  const int nz = (int)((d + kc - 1) / kc);
  const int tb = (s + kGramTile - 1) / kGramTile;
  const dim3 grid(sym ? tiles : tb, sym ? 1 : tb, nz);
  count_launch();
  gemm_tile_kernel<double, kGramTpx><<<grid, kGramTpx * kGramTpx, 0, st>>>(X, d, true, Y, d, s, s, d, kc, sym ? 1 : 0,
                                                                          work);
  NYS_CUDA_TRY(cudaGetLastError());
  count_launch();
  sum_partials_gram_kernel<<<std::min<int64_t>(1024, ((int64_t)s * s + 255) / 256), 256, 0, st>>>(work, nz, s,
                                                                                                   sym ? 1 : 0, C);
  return cudaGetLastError();
}

// C (d x s) = B (d x s) * V (s x s), all column-major
static cudaError_t gemm_nn(const double* B, int64_t d, int s, const double* V, double* C, cudaStream_t st) {
  dim3 grid((unsigned)((d + kGramTile - 1) / kGramTile), (s + kGramTile - 1) / kGramTile, 1);
  count_launch();
  gemm_tile_kernel<double, kGramTpx><<<grid, kGramTpx * kGramTpx, 0, st>>>(B, d, false, V, s, (int)d, s, s, s, 0, C);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Cholesky (upper, in place)
// Single CTA.  M (s x s, column-major) is symmetrised, then overwritten by the upper
// factor C (C^T C = M); the strict lower triangle is zeroed.  info = 0 or k+1 when
// the k-th pivot is not positive / not finite.
__global__ void __launch_bounds__(1024) chol_upper_kernel(double* M, int s, int* info, double rel_tol) {
  const int tid = threadIdx.x, T = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = T >> 5;
  __shared__ int bad;
  __shared__ double thresh;
  for (int j = warp; j < s; j += nwarp)
    for (int i = lane; i < j; i += 32) M[i + (int64_t)j * s] = 0.5 * (M[i + (int64_t)j * s] + M[j + (int64_t)i * s]);
  if (tid == 0) {
    bad = 0;
    double mx = 0.0;
    for (int j = 0; j < s; ++j) mx = fmax(mx, fabs(M[j + (int64_t)j * s]));
    thresh = rel_tol * mx;
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (tid == 0) {
      const double dj = M[j + (int64_t)j * s];
      if (!(dj > 0.0) || !(dj > thresh) || !isfinite(dj)) {
        bad = j + 1;
      } else {
        M[j + (int64_t)j * s] = sqrt(dj);
      }
    }
    __syncthreads();
    if (bad) break;
    const double piv = M[j + (int64_t)j * s];
    for (int c = j + 1 + tid; c < s; c += T) M[j + (int64_t)c * s] /= piv;
    __syncthreads();
    // trailing update of the upper triangle: M[i][c] -= C[j][i] C[j][c], j < i <= c
    // (warps over columns c, lanes over rows i: no index division in the inner loop)
    for (int c = j + 1 + warp; c < s; c += nwarp) {
      const double rc = M[j + (int64_t)c * s];
      double* col = M + (int64_t)c * s;
      for (int i = j + 1 + lane; i <= c; i += 32) col[i] -= M[j + (int64_t)i * s] * rc;
    }
    __syncthreads();
  }
  if (tid == 0) *info = bad;
  // zero the strict lower triangle
  for (int j = warp; j < s; j += nwarp)
    for (int i = j + 1 + lane; i < s; i += 32) M[i + (int64_t)j * s] = 0.0;
}

// Same algorithm and operation order with the upper triangle held in shared memory
// (packed by columns: (i, c), i <= c, at c (c + 1) / 2 + i), so that every step's
// pivot, row scaling and trailing update touch on-chip data instead of L2.
__global__ void __launch_bounds__(1024) chol_upper_smem_kernel(double* M, int s, int* info, double rel_tol) {
  extern __shared__ double up[];
  const int tid = threadIdx.x, T = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = T >> 5;
  __shared__ int bad;
  __shared__ double thresh;
  auto at = [](int i, int c) { return c * (c + 1) / 2 + i; };
  for (int j = warp; j < s; j += nwarp)
    for (int i = lane; i <= j; i += 32)
      up[at(i, j)] = i < j ? 0.5 * (M[i + (int64_t)j * s] + M[j + (int64_t)i * s]) : M[i + (int64_t)i * s];
  if (tid == 0) {
    bad = 0;
    double mx = 0.0;
    for (int j = 0; j < s; ++j) mx = fmax(mx, fabs(up[at(j, j)]));
    thresh = rel_tol * mx;
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (tid == 0) {
      const double dj = up[at(j, j)];
      if (!(dj > 0.0) || !(dj > thresh) || !isfinite(dj)) {
        bad = j + 1;
      } else {
        up[at(j, j)] = sqrt(dj);
      }
    }
    __syncthreads();
    if (bad) break;
    const double piv = up[at(j, j)];
    for (int c = j + 1 + tid; c < s; c += T) up[at(j, c)] /= piv;
    __syncthreads();
    // trailing update of the upper triangle: M[i][c] -= C[j][i] C[j][c], j < i <= c
    // (warps over columns c, lanes over rows i: no index division in the inner loop)
    for (int c = j + 1 + warp; c < s; c += nwarp) {
      const double rc = up[at(j, c)];
      double* col = up + at(0, c);
      for (int i = j + 1 + lane; i <= c; i += 32) col[i] -= up[at(j, i)] * rc;
    }
    __syncthreads();
  }
  if (tid == 0) *info = bad;
  for (int j = warp; j < s; j += nwarp)
    for (int i = lane; i < s; i += 32) M[i + (int64_t)j * s] = i <= j ? up[at(i, j)] : 0.0;
}

cudaError_t chol_upper(double* M, int s, int* info, cudaStream_t st, double rel_tol) {
  const size_t smem = (size_t)s * (s + 1) / 2 * sizeof(double);
  if (smem <= 200 * 1024) {
    NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)chol_upper_smem_kernel, 200 * 1024));
    count_launch();
    chol_upper_smem_kernel<<<1, 1024, smem, st>>>(M, s, info, rel_tol);
    return cudaGetLastError();
  }
  count_launch();
  chol_upper_kernel<<<1, 1024, 0, st>>>(M, s, info, rel_tol);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ triangular solve B C = Y
// One thread per row j of Y (d x s, column-major): b_c = (y_c - sum_{k<c} b_k C[k][c]) / C[c][c].
__global__ void trsm_ru_kernel(const double* __restrict__ Cm, int s, double* Y, int64_t d) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= d) return;
  for (int c = 0; c < s; ++c) {
    double acc = Y[j + (int64_t)c * d];
    const double* col = Cm + (int64_t)c * s;
    for (int k = 0; k < c; ++k) acc = fma(-Y[j + (int64_t)k * d], col[k], acc);
    Y[j + (int64_t)c * d] = acc / col[c];
  }
}

// Same recurrence and order, 64 rows per block (d = 10,000 rows spread over ~160 SMs
// instead of 79) with each row's solved prefix b_0 .. b_{c-1} kept in shared memory
// ([k][64], conflict-free) instead of re-read from global memory.
constexpr int kTrsmRows = 64;
__global__ void __launch_bounds__(kTrsmRows) trsm_ru_smem_kernel(const double* __restrict__ Cm, int s, double* Y,
                                                                 int64_t d) {
  extern __shared__ double bs[];  // [s][kTrsmRows]
  const int t = threadIdx.x;
  const int64_t j = blockIdx.x * (int64_t)kTrsmRows + t;
  const bool act = j < d;
  for (int c = 0; c < s; ++c) {
    double acc = act ? Y[j + (int64_t)c * d] : 0.0;
    const double* col = Cm + (int64_t)c * s;
    for (int k = 0; k < c; ++k) acc = fma(-bs[k * kTrsmRows + t], col[k], acc);
    const double b = acc / col[c];
    bs[c * kTrsmRows + t] = b;
    if (act) Y[j + (int64_t)c * d] = b;
  }
}

// Same recurrence and order again, blocked by columns so that most of the work runs on
// every thread: a CTA holds R rows of Y in shared memory ([c][R]) and, per block of 32
// columns, those columns of C.  For each block it first subtracts sum_{k < j0} b_k C[k][c]
// from all R x 32 entries (4 R threads, each row's k in ascending order), then one thread
// per row finishes the block (k from j0 to c - 1, then the division).  Every entry sees the same fma sequence as in
// trsm_ru_kernel, so the result is bitwise the same.  R = ceil(d / #SMs): one wave.
constexpr int kTrsmBlk = 32;
__global__ void __launch_bounds__(1024) trsm_ru_blocked_kernel(const double* __restrict__ Cm, int s, double* Y,
                                                               int64_t d, int R) {
  extern __shared__ double bs[];  // [s][R], then the block's columns of C: cs[k][32], k < j1
  double* cs = bs + (size_t)s * R;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int nr = (int)min((int64_t)R, d - r0);
  for (int idx = threadIdx.x; idx < s * R; idx += blockDim.x) {
    const int c = idx / R, r = idx % R;
    bs[idx] = r < nr ? Y[r0 + r + (int64_t)c * d] : 0.0;
  }
  const int r = threadIdx.x % R, cg = threadIdx.x / R;
  for (int j0 = 0; j0 < s; j0 += kTrsmBlk) {
    const int j1 = min(s, j0 + kTrsmBlk);
    const int w = j1 - j0;
    // C[k][c] for k < j1, c in [j0, j1): read by every row of the CTA, staged once
    for (int idx = threadIdx.x; idx < j1 * w; idx += blockDim.x) {
      const int k = idx % j1, cc = idx / j1;
      cs[k * kTrsmBlk + cc] = Cm[k + (int64_t)(j0 + cc) * s];
    }
    __syncthreads();
    if (cg < 4 && j0 > 0) {
      double acc[kTrsmBlk / 4];
#pragma unroll
      for (int q = 0; q < kTrsmBlk / 4; ++q) {
        const int c = j0 + cg + 4 * q;
        acc[q] = c < j1 ? bs[c * R + r] : 0.0;
      }
      for (int k = 0; k < j0; ++k) {
        const double bk = bs[k * R + r];
#pragma unroll
        for (int q = 0; q < kTrsmBlk / 4; ++q) {
          const int c = j0 + cg + 4 * q;
          if (c < j1) acc[q] = fma(-bk, cs[k * kTrsmBlk + cg + 4 * q], acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < kTrsmBlk / 4; ++q) {
        const int c = j0 + cg + 4 * q;
        if (c < j1) bs[c * R + r] = acc[q];
      }
    }
    __syncthreads();
    if (threadIdx.x < R) {
      for (int c = j0; c < j1; ++c) {
        const double* col = cs + (c - j0);
        double acc = bs[c * R + r];
        for (int k = j0; k < c; ++k) acc = fma(-bs[k * R + r], col[k * kTrsmBlk], acc);
        bs[c * R + r] = acc / col[c * kTrsmBlk];
      }
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < s * R; idx += blockDim.x) {
    const int c = idx / R, rr = idx % R;
    if (rr < nr) Y[r0 + rr + (int64_t)c * d] = bs[idx];
  }
}

cudaError_t trsm_right_upper(const double* C, int s, double* Y, int64_t d, cudaStream_t st) {
  {
    int R = (int)std::min<int64_t>(128, (d + sm_count() - 1) / sm_count());
    R = std::max(R, 1);
    const size_t cblk = (size_t)s * kTrsmBlk * sizeof(double);   // staged columns of C
    while (R > 8 && (size_t)s * R * sizeof(double) + cblk > 200 * 1024) R /= 2;
    const size_t smem_b = (size_t)s * R * sizeof(double) + cblk;
    if (R >= 8 && smem_b <= 200 * 1024) {
      NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)trsm_ru_blocked_kernel, 200 * 1024));
      const int threads = (4 * R + 31) / 32 * 32;
      count_launch();
      trsm_ru_blocked_kernel<<<(unsigned)((d + R - 1) / R), threads, smem_b, st>>>(C, s, Y, d, R);
      return cudaGetLastError();
    }
  }
  const size_t smem = (size_t)s * kTrsmRows * sizeof(double);
  if (smem <= 200 * 1024) {
    NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)trsm_ru_smem_kernel, 200 * 1024));
    count_launch();
    trsm_ru_smem_kernel<<<(unsigned)((d + kTrsmRows - 1) / kTrsmRows), kTrsmRows, smem, st>>>(C, s, Y, d);
    return cudaGetLastError();
  }
  count_launch();
  trsm_ru_kernel<<<(unsigned)((d + 127) / 128), 128, 0, st>>>(C, s, Y, d);
  return cudaGetLastError();
}

__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

cudaError_t axpy_panel(double nu, const double* X, double* Y, int64_t n, cudaStream_t st) {
  count_launch();
  axpy_kernel<<<(unsigned)std::min<int64_t>(4096, (n + 255) / 256), 256, 0, st>>>(nu, X, Y, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ power iteration (lambda_max)
// 30 power iterations on the symmetric s x s Gram matrix G (column-major; row i is column
// i).  One SM's FP64 pipe (about 2 FMA per clock) would need ~10 us per s = 200 matvec, so
// the rows are spread over kPowBlocks co-resident blocks (cooperative launch): block b
// forms w_i for its rows (one warp per row, lanes over k, then a warp sum), writes them,
// and after a grid barrier every block reads all of w through L2 and takes the same
// fixed-order norms, so every block holds the same v.  lam = the Rayleigh quotient
// v^T G v / v^T v of the last iterate.
constexpr int kPowThreads = 256;
__global__ void __launch_bounds__(kPowThreads) power_kernel(const double* __restrict__ G, int s, int iters,
                                                            double* out, double* wbuf, unsigned* bar) {
  __shared__ double sh[kPowThreads / 32];
  extern __shared__ double vs[];   // v (s)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kPowThreads / 32;
  const int rows_per = (s + gridDim.x - 1) / gridDim.x;
  const int i_lo = blockIdx.x * rows_per, i_hi = min(s, i_lo + rows_per);
  // a barrier that runs out leaves NaN here: the shift, and with it the factorisation, fails
  if (blockIdx.x == 0 && tid == 0) *out = __longlong_as_double(0x7ff8000000000000LL);
  for (int i = tid; i < s; i += kPowThreads) vs[i] = 1.0 + 1e-3 * (double)(i % 7);  // deterministic start
  __syncthreads();
  double lam = 0.0;
  unsigned target = 0;
  for (int it = 0; it < iters; ++it) {
    double* w = wbuf + (size_t)(it & 1) * s;   // alternate buffers: no block overwrites a w still being read
    for (int i = i_lo + warp; i < i_hi; i += NW) {
      const double* col = G + (int64_t)i * s;
      double acc = 0.0;
      for (int k = lane; k < s; k += 32) acc = fma(__ldg(col + k), vs[k], acc);
      acc = warp_sum(acc);
      if (lane == 0) w[i] = acc;
    }
    target += gridDim.x;
    if (!grid_barrier_mono(bar, target)) {
      if (tid == 0) atomicExch(bar + 1, 1u);
      return;
    }
    double num = 0.0, l2 = 0.0, vv = 0.0;
    for (int i = tid; i < s; i += kPowThreads) {
      const double wi = __ldcg(w + i);
      num += vs[i] * wi;
      l2 += wi * wi;
      vv += vs[i] * vs[i];
    }
    num = block_sum<kPowThreads>(num, sh);
    const double nw2 = block_sum<kPowThreads>(l2, sh);
    const double nv2 = block_sum<kPowThreads>(vv, sh);
    lam = num / nv2;
    const double inv = nw2 > 0 ? 1.0 / sqrt(nw2) : 0.0;
    for (int i = tid; i < s; i += kPowThreads) vs[i] = __ldcg(w + i) * inv;
    __syncthreads();
  }
  if (blockIdx.x == 0 && tid == 0) *out = lam;
}

// work: 2 s doubles + 2 words (barrier counter, timeout flag)
cudaError_t power_lambda_max(const double* G, int s, double* out, double* work, cudaStream_t st) {
  if (s > 4096) return cudaErrorInvalidValue;
  unsigned* bar = reinterpret_cast<unsigned*>(work + 2 * (size_t)s);
  NYS_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  int per_sm = 0;
  NYS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, power_kernel, kPowThreads,
                                                             (size_t)s * sizeof(double)));
  const int nb = std::max(1, std::min({(s + 7) / 8, 64, per_sm * sm_count()}));
  int iters = 30;
  const double* g = G;
  double* w = work;
  void* args[] = {(void*)&g, (void*)&s, (void*)&iters, (void*)&out, (void*)&w, (void*)&bar};
  count_launch();
  NYS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)power_kernel, dim3(nb), dim3(kPowThreads), args,
                                           (size_t)s * sizeof(double), st));
  return cudaGetLastError();
}

// ------------------------------------------------------------------ parallel cyclic Jacobi
// Round-robin ("circle") pairing of N = even size: round r in [0, N-1):
//   pair 0 = (N-1, r);  pair m >= 1 = ((r+m) mod (N-1), (r-m+N-1) mod (N-1)).
__device__ __forceinline__ void rr_pair(int N, int r, int m, int& p, int& q) {
  if (m == 0) {
    p = N - 1;
    q = r;
  } else {
    // (r + m) mod (N - 1) and (r - m) mod (N - 1) for 0 <= r < N - 1, 0 < m < N / 2: both
    // sums lie in [0, 2 (N - 1)), so one conditional subtraction replaces the division
    p = r + m;
    if (p >= N - 1) p -= N - 1;
    q = r - m + (N - 1);
    if (q >= N - 1) q -= N - 1;
  }
}

// Rotation (c, sn) that zeroes a_pq of the 2x2 block [[app, apq], [apq, aqq]] under
// J^T A J with J_pp = J_qq = c, J_pq = sn, J_qp = -sn (Golub & Van Loan, Alg. 8.4.1: the
// smaller root t of t^2 + 2 tau t - 1 = 0, tau = (aqq - app) / (2 apq), c = 1/sqrt(1 + t^2),
// sn = t c).  With h = aqq - app, g = 2 apq and r = sqrt(h^2 + g^2) that root is
// t = sign(tau) |g| / (|h| + r), and 1 + t^2 = 2 r (r + |h|) / (|h| + r)^2, so
//   c = (|h| + r) / sqrt(2 r (r + |h|)),   sn = sign(tau) |g| / sqrt(2 r (r + |h|)):
// one square root and one reciprocal square root instead of two of each and three
// divisions (the FP64 divide / square-root chain bounded each Jacobi round).
__device__ __forceinline__ void jacobi_rot(double app, double aqq, double apq, double& c, double& sn) {
  if (apq == 0.0 || fabs(apq) <= 1e-300 || apq * apq < 1e-34 * fabs(app * aqq)) {
    c = 1.0;
    sn = 0.0;
    return;
  }
  const double h = aqq - app, g = 2.0 * apq;
  const double ah = fabs(h);
  const double r = sqrt(fma(h, h, g * g));
  const double inv = rsqrt(2.0 * r * (r + ah));
  // sign(tau) = sign(h) sign(g), and +1 for h = 0
  const double gs = h > 0.0 ? g : (h < 0.0 ? -g : fabs(g));
  c = (ah + r) * inv;
  sn = gs * inv;
}

// One round: Aout = J^T Ain J and V <- V J for the round's N/2 disjoint rotations.
// Block (bx, by) owns a 16 x 16 tile of 2x2 pair-blocks of A (pairs ma = bx*16 + tx,
// mb = by*16 + ty); the 32 rotations it needs are computed once into shared memory.
// Every block also applies its 16 column rotations to one row slice of V (slice by of gy).
// The pair indices of a round depend only on (N, r), so every load of the round -- the
// three entries behind each rotation, the tile's four entries, the V entries -- is issued
// before any rotation is formed: one memory latency per round instead of three.
// In the persistent form Ain and V were written by other blocks earlier in the same launch:
// their loads go through L2 (__ldcg), never through this SM's L1, which may hold the lines
// from an earlier round.
// 8 x 8 pair-blocks per tile: s = 200 gives 13 x 13 = 169 tiles, so a round's FP64
// rotations (the pipe runs about 2 FMA per clock per SM) spread over every SM.
constexpr int JT = 8;
constexpr int kJacVMax = 4;   // V (row, pair) elements per thread: rows <= kJacVMax * 256 / 16
struct JacobiRoundSmem {
  double rc[2][JT], rs[2][JT];
  int rp[2][JT], rq[2][JT];
};
// `tid` is the thread's index among the tile's JT * JT threads and `sync` their barrier.
template <int VMAX, typename Sync>
__device__ __forceinline__ void jacobi_round_t(const double* Ain, double* Aout, double* V, int N, int r, int bx, int by,
                                               int gy, JacobiRoundSmem& sh, const int tid, Sync sync) {
  const int H = N / 2;
  const int tx = tid % JT, ty = tid / JT;
  // rotation inputs (threads < 32)
  int rp_ = 0, rq_ = 1;
  double app = 0.0, aqq = 0.0, apq = 0.0;
  bool have_rot = false;
  if (tid < 2 * JT) {
    const int side = tid / JT, t = tid % JT;
    const int m = (side == 0 ? bx : by) * JT + t;
    if (m < H) {
      rr_pair(N, r, m, rp_, rq_);
      app = __ldcg(Ain + rp_ + (int64_t)rp_ * N);
      aqq = __ldcg(Ain + rq_ + (int64_t)rq_ * N);
      apq = __ldcg(Ain + rp_ + (int64_t)rq_ * N);
      have_rot = true;
    }
  }
  // tile entries
  const int ma = bx * JT + tx, mb = by * JT + ty;
  const bool in_tile = ma < H && mb < H;
  int pa = 0, qa = 1, pb = 0, qb = 1;
  double x_pp = 0.0, x_pq = 0.0, x_qp = 0.0, x_qq = 0.0;
  if (in_tile) {
    rr_pair(N, r, ma, pa, qa);
    rr_pair(N, r, mb, pb, qb);
    x_pp = __ldcg(Ain + pa + (int64_t)pb * N);
    x_pq = __ldcg(Ain + pa + (int64_t)qb * N);
    x_qp = __ldcg(Ain + qa + (int64_t)pb * N);
    x_qq = __ldcg(Ain + qa + (int64_t)qb * N);
  }
  // V entries: this block's 16 pairs (those of bx) over rows [lo, hi)
  const int npair = min(JT, H - bx * JT);
  const int lo = (int)((int64_t)N * by / gy), hi = (int)((int64_t)N * (by + 1) / gy);
  const int rows = hi - lo;
  const int nel = npair > 0 ? npair * rows : 0;
  double vp[VMAX], vq[VMAX];
  int vrow[VMAX], vpi[VMAX], vqi[VMAX], vt[VMAX];
#pragma unroll
  for (int c = 0; c < VMAX; ++c) {
    const int e = tid + c * JT * JT;
    vt[c] = -1;
    if (e < nel) {
      const int t = e / rows, row = lo + e % rows;
      int p, q;
      rr_pair(N, r, bx * JT + t, p, q);
      vt[c] = t;
      vrow[c] = row;
      vpi[c] = p;
      vqi[c] = q;
      vp[c] = __ldcg(V + row + (int64_t)p * N);
      vq[c] = __ldcg(V + row + (int64_t)q * N);
    }
  }
  if (tid < 2 * JT) {
    const int side = tid / JT, t = tid % JT;
    double c = 1.0, sn = 0.0;
    if (have_rot) jacobi_rot(app, aqq, apq, c, sn);
    sh.rc[side][t] = c;
    sh.rs[side][t] = sn;
    sh.rp[side][t] = rp_;
    sh.rq[side][t] = rq_;
  }
  sync();
  if (in_tile) {
    const double ca = sh.rc[0][tx], sa = sh.rs[0][tx], cb = sh.rc[1][ty], sb = sh.rs[1][ty];
    // columns: p' = c p - s q, q' = s p + c q
    const double y_pp = cb * x_pp - sb * x_pq, y_pq = sb * x_pp + cb * x_pq;
    const double y_qp = cb * x_qp - sb * x_qq, y_qq = sb * x_qp + cb * x_qq;
    // rows
    double z_pp = ca * y_pp - sa * y_qp, z_pq = ca * y_pq - sa * y_qq;
    double z_qp = sa * y_pp + ca * y_qp, z_qq = sa * y_pq + ca * y_qq;
    if (ma == mb) {  // the rotated pair itself: off-diagonal is zero by construction
      z_pq = 0.0;
      z_qp = 0.0;
    }
    Aout[pa + (int64_t)pb * N] = z_pp;
    Aout[pa + (int64_t)qb * N] = z_pq;
    Aout[qa + (int64_t)pb * N] = z_qp;
    Aout[qa + (int64_t)qb * N] = z_qq;
  }
  // V <- V J (the pairs of a round are disjoint: every (row, pair) element is independent)
#pragma unroll
  for (int c = 0; c < VMAX; ++c) {
    if (vt[c] >= 0) {
      const double cc = sh.rc[0][vt[c]], sn = sh.rs[0][vt[c]];
      V[vrow[c] + (int64_t)vpi[c] * N] = cc * vp[c] - sn * vq[c];
      V[vrow[c] + (int64_t)vqi[c] * N] = sn * vp[c] + cc * vq[c];
    }
  }
  // elements beyond VMAX per thread (only for very tall slices): the plain loop
  for (int e = tid + VMAX * JT * JT; e < nel; e += JT * JT) {
    const int t = e / rows, row = lo + e % rows;
    const int p = sh.rp[0][t], q = sh.rq[0][t];
    const double c = sh.rc[0][t], sn = sh.rs[0][t];
    const double a = __ldcg(V + row + (int64_t)p * N), bq = __ldcg(V + row + (int64_t)q * N);
    V[row + (int64_t)p * N] = c * a - sn * bq;
    V[row + (int64_t)q * N] = sn * a + c * bq;
  }
}

__device__ __forceinline__ void jacobi_round(const double* Ain, double* Aout, double* V, int N, int r, int bx, int by,
                                             int gy, JacobiRoundSmem& sh) {
  jacobi_round_t<kJacVMax>(Ain, Aout, V, N, r, bx, by, gy, sh, (int)threadIdx.x, [] { __syncthreads(); });
}

__global__ void __launch_bounds__(JT * JT) jacobi_round_kernel(const double* __restrict__ Ain, double* __restrict__ Aout,
                                                               double* V, int N, int r, const int* __restrict__ done) {
  if (*done) return;
  __shared__ JacobiRoundSmem sh;
  jacobi_round(Ain, Aout, V, N, r, blockIdx.x, blockIdx.y, gridDim.y, sh);
}

// The whole eigensolve in one launch: the grid (co-resident, cooperative launch) runs the
// rounds of every sweep separated by grid barriers, then takes off(A)^2 / ||A||_F^2 from
// per-block partials summed by every block in the same fixed order, so all blocks take
// the same stop decision.  The rotations and their order are those of jacobi_round_kernel,
// so the result is bitwise that of the round-per-launch form.  ctl[0] = barrier count,
// ctl[1] = barrier generation, ctl[2] = sweeps done, ctl[3] = 1 if a barrier wait ran out.
__global__ void __launch_bounds__(JT * JT) jacobi_persistent_kernel(double* A0, double* A1, double* V, int N,
                                                                    int max_sweeps, double tol2, double* part,
                                                                    unsigned* ctl) {
  __shared__ JacobiRoundSmem sh;
  __shared__ double red[2][JT * JT / 32];
  const int nblk = gridDim.x * gridDim.y;
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  const int H = N / 2;
  double* cur = A0;
  double* nxt = A1;
  int sweeps = 0;
  unsigned target = 0;
  for (; sweeps < max_sweeps; ++sweeps) {
    for (int r = 0; r < N - 1; ++r) {
      jacobi_round(cur, nxt, V, N, r, blockIdx.x, blockIdx.y, gridDim.y, sh);
      target += (unsigned)nblk;
      if (!grid_barrier_mono(&ctl[0], target)) {
        if (threadIdx.x == 0) atomicExch(&ctl[3], 1u);
        return;
      }
      double* t = cur;
      cur = nxt;
      nxt = t;
    }
    // off-diagonal and total squares of this block's tile of the current matrix
    double off = 0.0, tot = 0.0;
    {
      const int tx = threadIdx.x % JT, ty = threadIdx.x / JT;
      const int ma = blockIdx.x * JT + tx, mb = blockIdx.y * JT + ty;
      if (ma < H && mb < H) {
        const int ia[2] = {2 * ma, 2 * ma + 1}, ib[2] = {2 * mb, 2 * mb + 1};
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const double x = __ldcg(cur + ia[u] + (int64_t)ib[v] * N);
            tot += x * x;
            if (ia[u] != ib[v]) off += x * x;
          }
      }
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = off;
      red[1][threadIdx.x >> 5] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double o = 0.0, t = 0.0;
      for (int w = 0; w < JT * JT / 32; ++w) {
        o += red[0][w];
        t += red[1][w];
      }
      part[2 * bid] = o;
      part[2 * bid + 1] = t;
    }
    target += (unsigned)nblk;
    if (!grid_barrier_mono(&ctl[0], target)) {
      if (threadIdx.x == 0) atomicExch(&ctl[3], 1u);
      return;
    }
    double o = 0.0, t = 0.0;
    for (int b = 0; b < nblk; ++b) {
      o += __ldcg(part + 2 * b);
      t += __ldcg(part + 2 * b + 1);
    }
    // every block has read the partials before any block overwrites them next sweep
    target += (unsigned)nblk;
    if (!grid_barrier_mono(&ctl[0], target)) {
      if (threadIdx.x == 0) atomicExch(&ctl[3], 1u);
      return;
    }
    if (o <= tol2 * t) {
      ++sweeps;
      break;
    }
  }
  if (bid == 0 && threadIdx.x == 0) ctl[2] = (unsigned)sweeps;
  // leave the diagonalised matrix in A0
  if (cur != A0) {
    for (int64_t idx = (int64_t)bid * blockDim.x + threadIdx.x; idx < (int64_t)N * N; idx += (int64_t)nblk * blockDim.x)
      A0[idx] = __ldcg(cur + idx);
  }
}

// off(A)^2 and ||A||_F^2; sets *done when off <= tol^2 * ||A||_F^2.
__global__ void __launch_bounds__(256) jacobi_offnorm_kernel(const double* __restrict__ A, int N, double tol2,
                                                             int* done, double* offout) {
  __shared__ double sh[8];
  double off = 0.0, tot = 0.0;
  for (int64_t idx = threadIdx.x; idx < (int64_t)N * N; idx += 256) {
    const double v = A[idx];
    tot += v * v;
    if (idx % N != idx / N) off += v * v;
  }
  off = block_sum<256>(off, sh);
  tot = block_sum<256>(tot, sh);
  if (threadIdx.x == 0) {
    *offout = off;
    if (off <= tol2 * tot) *done = 1;
  }
}

// Pad G (s x s) into N x N (N = s rounded up to even) and set V = I.
__global__ void jacobi_setup_kernel(const double* __restrict__ G, int s, double* A, double* V, int N, int* done) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)N * N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % N), j = (int)(idx / N);
    double g = 0.0;
    if (i < s && j < s) g = 0.5 * (G[i + (int64_t)j * s] + G[j + (int64_t)i * s]);
    A[idx] = g;
    V[idx] = (i == j) ? 1.0 : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *done = 0;
}

// max_ij |G_ij - delta_ij| of an m x m matrix (one block, fixed-order max: exact)
__global__ void __launch_bounds__(256) identity_gap_kernel(const double* __restrict__ G, int m, double* out) {
  __shared__ double sh[8];
  double g = 0.0;
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * m; idx += 256) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    g = fmax(g, fabs(G[idx] - (i == j ? 1.0 : 0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < 8; ++w) r = fmax(r, sh[w]);
    *out = r;
  }
}

cudaError_t identity_gap(const double* G, int m, double* out, cudaStream_t st) {
  count_launch();
  identity_gap_kernel<<<1, 256, 0, st>>>(G, m, out);
  return cudaGetLastError();
}

size_t jacobi_work_bytes(int s) {
  const int N = s + (s & 1);
  const int HT = (N / 2 + JT - 1) / JT;
  // A0, A1, spare N x N, flags, per-block partials of the persistent form, its barrier words
  return (size_t)3 * N * N * sizeof(double) + 64 + (size_t)2 * HT * HT * sizeof(double) + 64;
}

// Eigendecomposition of the symmetric s x s matrix G.  Results: eigenvalues on the
// diagonal of `evals_mat` (N x N, in work), eigenvectors in the columns of Vout (N x N).
// work layout: A0 (N*N), A1 (N*N), V (N*N), flags.  Sweeps stop once the off-diagonal
// Frobenius norm is at most tol times the whole matrix's.
cudaError_t jacobi_eig(double* G, double* Vout, int s, double* work, int* sweeps_out, cudaStream_t st, double tol) {
  const int N = s + (s & 1);
  const double tol_sq = tol * tol;
  double* A0 = work;
  double* A1 = work + (size_t)N * N;
  int* done = reinterpret_cast<int*>(work + (size_t)3 * N * N);
  double* offv = work + (size_t)3 * N * N + 1;
  count_launch();
  jacobi_setup_kernel<<<std::max(1, std::min(1024, (N * N + 255) / 256)), 256, 0, st>>>(G, s, A0, Vout, N, done);
  NYS_CUDA_TRY(cudaGetLastError());
  const int HT = (N / 2 + JT - 1) / JT;
  const dim3 blocks(HT, HT);
  const int kMaxSweeps = 30;
  // one cooperative launch for all sweeps when the grid can be co-resident
  // (NYS_JACOBI_PERSISTENT=0 selects the round-per-launch form)
  const char* jp = std::getenv("NYS_JACOBI_PERSISTENT");
  if (N > 2 && (jp == nullptr || std::atoi(jp) != 0)) {
    int dev = 0, coop = 0, per_sm = 0;
    NYS_CUDA_TRY(cudaGetDevice(&dev));
    NYS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    NYS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_persistent_kernel, JT * JT, 0));
    if (N > 2 && coop && (int64_t)per_sm * sm_count() >= (int64_t)HT * HT) {
      double* part = work + (size_t)3 * N * N + 8;                       // 2 doubles per block
      unsigned* ctl = reinterpret_cast<unsigned*>(part + 2 * (size_t)HT * HT);
      NYS_CUDA_TRY(cudaMemsetAsync(ctl, 0, 4 * sizeof(unsigned), st));
      double* a0 = A0;
      double* a1 = A1;
      double* vv = Vout;
      int n = N, ms = kMaxSweeps;
      double tol2 = tol_sq;
      void* args[] = {&a0, &a1, &vv, &n, &ms, &tol2, &part, &ctl};
      count_launch();
      NYS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_persistent_kernel, blocks, dim3(JT * JT), args, 0, st));
      unsigned h[4] = {0, 0, 0, 0};
      NYS_CUDA_TRY(cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
      NYS_CUDA_TRY(cudaStreamSynchronize(st));
      if (h[3]) return cudaErrorLaunchTimeout;   // a barrier wait ran out (reported as NYS_ECUDA)
      if (sweeps_out) *sweeps_out = (int)h[2];
      return cudaSuccess;
    }
  }
  int sweeps = 0;
  int done_h = 0;
  // One sweep = N - 1 round launches (ping-pong between A0 and A1; N - 1 is odd for even
  // N, so after a sweep the roles of A0 and A1 swap).  Sweeps are captured once as two CUDA
  // graphs (A0 -> A1 and A1 -> A0 starting buffers) and replayed, which removes the
  // per-launch host overhead of ~N launches per sweep.
  double* cur = A0;
  double* nxt = A1;
  cudaGraphExec_t sweep_exec[2] = {nullptr, nullptr};
  const bool trace = std::getenv("NYS_TRACE") != nullptr;
  auto t_cap = std::chrono::steady_clock::now();
  bool graphs_ok = N > 2;
  if (graphs_ok) {
    cudaStream_t cap = nullptr;
    graphs_ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int gi = 0; gi < 2 && graphs_ok; ++gi) {
      double* c = gi == 0 ? A0 : A1;
      double* x = gi == 0 ? A1 : A0;
      cudaGraph_t gr = nullptr;
      count_launch_suspend(true);
      graphs_ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) == cudaSuccess;
      for (int r = 0; r < N - 1 && graphs_ok; ++r) {
        jacobi_round_kernel<<<blocks, JT * JT, 0, cap>>>(c, x, Vout, N, r, done);
        std::swap(c, x);
      }
      graphs_ok = cudaStreamEndCapture(cap, &gr) == cudaSuccess && graphs_ok;
      count_launch_suspend(false);
      if (graphs_ok) graphs_ok = cudaGraphInstantiate(&sweep_exec[gi], gr, 0) == cudaSuccess;
      if (gr) cudaGraphDestroy(gr);
    }
    if (cap) cudaStreamDestroy(cap);
    cudaGetLastError();
  }
  if (trace) {
    cudaStreamSynchronize(st);
    std::fprintf(stderr, "[nys] jacobi capture+inst   %9.3f ms\n",
                 std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_cap).count());
  }
  for (; sweeps < kMaxSweeps; ++sweeps) {
    auto t_sw = std::chrono::steady_clock::now();
    if (N <= 2 && sweeps > 0) break;
    if (graphs_ok) {
      NYS_CUDA_TRY(cudaGraphLaunch(sweep_exec[cur == A0 ? 0 : 1], st));
      count_launch_add(N - 1);
      if ((N - 1) % 2 == 1) std::swap(cur, nxt);
    } else {
      for (int r = 0; r < N - 1; ++r) {
        count_launch();
        jacobi_round_kernel<<<blocks, JT * JT, 0, st>>>(cur, nxt, Vout, N, r, done);
        std::swap(cur, nxt);
      }
    }
    NYS_CUDA_TRY(cudaGetLastError());
    count_launch();
    jacobi_offnorm_kernel<<<1, 256, 0, st>>>(cur, N, tol_sq, done, offv);
    NYS_CUDA_TRY(cudaMemcpyAsync(&done_h, done, sizeof(int), cudaMemcpyDeviceToHost, st));
    NYS_CUDA_TRY(cudaStreamSynchronize(st));
    if (trace)
      std::fprintf(stderr, "[nys] jacobi sweep %2d       %9.3f ms\n", sweeps,
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_sw).count());
    if (done_h) {
      ++sweeps;
      break;
    }
  }
  for (auto& e : sweep_exec)
    if (e) cudaGraphExecDestroy(e);
  // copy the diagonalised matrix back into G's storage layout (N x N in A0 slot)
  if (cur != A0) NYS_CUDA_TRY(cudaMemcpyAsync(A0, cur, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (sweeps_out) *sweeps_out = sweeps;
  return cudaGetLastError();
}

// Sort eigenpairs (diagonal of Ad, N x N) descending over the first s, build
// Vs (s x s) = selected eigenvector columns (rows < s), sig2 (s).
__global__ void __launch_bounds__(512) eig_sort_kernel(const double* __restrict__ Ad, const double* __restrict__ V,
                                                       int N, int s, double* Vs, double* sig2) {
  // rank-based ordering over the N eigenvalues (padding row/col, if any, has eigenvalue ~0
  // and is excluded by keeping the s largest after dropping the pad index's contribution)
  extern __shared__ double ev[];
  int* rank = reinterpret_cast<int*>(ev + N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) ev[i] = Ad[i + (int64_t)i * N];
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    int r = 0;
    for (int j = 0; j < N; ++j) r += (ev[j] > ev[i]) || (ev[j] == ev[i] && j < i);
    rank[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int r = rank[i];
    if (r < s) {
      sig2[r] = ev[i];
      for (int row = 0; row < s; ++row) Vs[row + (int64_t)r * s] = V[row + (int64_t)i * N];
    }
  }
}

// U[:, c] = BV[:, c] / sigma_c  (sigma_c = sqrt(sig2_c) if sig2_c > 0 else column set to 0),
// lam_c = max(0, sig2_c - nu)
__global__ void finish_scale_kernel(double* U, int64_t d, int s, const double* __restrict__ sig2, double nu,
                                    double* lam) {
  const int64_t total = d * s;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / d);
    const double g = sig2[c];
    U[idx] = g > 0.0 ? U[idx] / sqrt(g) : 0.0;
  }
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < s; c += blockDim.x) lam[c] = fmax(0.0, sig2[c] - nu);
}

cudaError_t nystrom_finish(const double* B, int64_t d, int s, const double* Ad, const double* V, double nu,
                           double* U, double* lam, double* work, cudaStream_t st) {
  const int N = s + (s & 1);
  double* Vs = work;
  double* sig2 = work + (size_t)s * s;
  const size_t sm = (size_t)N * sizeof(double) + (size_t)N * sizeof(int);
  count_launch();
  eig_sort_kernel<<<1, 512, sm, st>>>(Ad, V, N, s, Vs, sig2);
  NYS_CUDA_TRY(cudaGetLastError());
  NYS_CUDA_TRY(gemm_nn(B, d, s, Vs, U, st));
  count_launch();
  finish_scale_kernel<<<(unsigned)std::min<int64_t>(4096, (d * s + 255) / 256), 256, 0, st>>>(U, d, s, sig2, nu,
                                                                                              lam);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ sketch GEMMs
// ------------------------------------------------------------------ fast float-compute sketch GEMM
// C (M x N, column-major, ld ldc) = op(A) B for FP32 / BF16 storage of A, FP32 B:
//   AW  (transA = 0): M = n rows of A, K = d:  op(A)[m][k] = A[m*ld + k]   (W = A Omega)
//   ATW (transA = 1): M = d cols of A, K = n:  op(A)[m][k] = A[k*ld + m]   (Y_z = A^T W, rows kb..ke)
// B is K x N column-major (ld ldb).  128 x 64 block tile, 256 threads, each thread an
// 8 x 4 sub-tile with packed FP32 FMAs; the next K tile is prefetched into registers
// while the current one is in shared memory (k-slow layout As[16][128], Bs[16][64]).
constexpr int FBM = 128, FBN = 64, FBK = 16;

template <int DT, bool TRANS>
__global__ void __launch_bounds__(256) fgemm_kernel(const unsigned char* __restrict__ Araw, int64_t lda, int64_t M,
                                                    int N, int64_t K, int64_t kchunk, const float* __restrict__ B,
                                                    int64_t ldb, const double* __restrict__ Drow,
                                                    float* __restrict__ Cout_base, int64_t ldc,
                                                    int64_t slice_stride) {
  __shared__ __align__(16) float As[2][FBK][FBM];
  __shared__ __align__(16) float Bs[2][FBK][FBN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * FBM;
  const int n0 = blockIdx.y * FBN;
  // split-K: slice z covers k in [z * kchunk, min(K, (z + 1) * kchunk)) and writes its own partial
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(K, kb + kchunk);
  float* Cout = Cout_base + (int64_t)blockIdx.z * slice_stride;
  // --- global -> register staging of one K tile
  // A tile: 128 (m) x 16 (k) values; 8 values per thread.
  // B tile: 16 (k) x 64 (n) values; 4 values per thread.
  float ra[8], rb[4];
  auto load_tile = [&](int64_t k0) {
    if (!TRANS) {
      // thread -> row m = tid >> 1, k half = (tid & 1) * 8: 8 consecutive k of one row
      const int64_t m = m0 + (tid >> 1);
      const int64_t k = k0 + (tid & 1) * 8;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        ra[e] = (m < M && k + e < ke) ? load_elem<DT>(Araw, m * lda + k + e) : 0.f;
    } else {
      // thread -> k row = tid >> 4, 8 consecutive m at (tid & 15) * 8
      const int64_t k = k0 + (tid >> 4);
      const int64_t m = m0 + (tid & 15) * 8;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        ra[e] = (k < ke && m + e < M) ? load_elem<DT>(Araw, k * lda + m + e) : 0.f;
    }
    // B: column n = tid >> 2, 4 consecutive k at (tid & 3) * 4
    const int n = n0 + (tid >> 2);
    const int64_t k = k0 + (tid & 3) * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) rb[e] = (n < N && k + e < ke) ? B[(int64_t)n * ldb + k + e] : 0.f;
  };
  auto store_tile = [&](int buf) {
    if (!TRANS) {
      const int m = tid >> 1, kk = (tid & 1) * 8;
#pragma unroll
      for (int e = 0; e < 8; ++e) As[buf][kk + e][m] = ra[e];
    } else {
      const int kk = tid >> 4, m = (tid & 15) * 8;
      *reinterpret_cast<float4*>(&As[buf][kk][m]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
      *reinterpret_cast<float4*>(&As[buf][kk][m + 4]) = make_float4(ra[4], ra[5], ra[6], ra[7]);
    }
    const int n = tid >> 2, kk = (tid & 3) * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) Bs[buf][kk + e][n] = rb[e];
  };
  float2 acc[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
  int buf = 0;
  load_tile(kb);
  store_tile(0);
  __syncthreads();
  for (int64_t k0 = kb; k0 < ke; k0 += FBK) {
    const bool more = k0 + FBK < ke;
    if (more) load_tile(k0 + FBK);
#pragma unroll
    for (int kk = 0; kk < FBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float2 b01 = make_float2(bv.x, bv.y), b23 = make_float2(bv.z, bv.w);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 ai = make_float2(av[i], av[i]);
        acc[i][0] = __ffma2_rn(ai, b01, acc[i][0]);
        acc[i][1] = __ffma2_rn(ai, b23, acc[i][1]);
      }
    }
    if (more) {
      store_tile(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + ty * 8 + i;
    if (m >= M) continue;
    const float dm = Drow ? (float)Drow[m] : 1.f;
    const float v[4] = {acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n < N) Cout[m + (int64_t)n * ldc] = dm * v[j];
    }
  }
}

// W (n x s, column-major, ld n, compute type C) = diag(D) A Om, Om d x s column-major (ld d).
template <int DT>
__global__ void __launch_bounds__(256) sketch_aw_kernel(const unsigned char* __restrict__ Araw, int64_t n,
                                                        int64_t d, int64_t ld,
                                                        const typename Stor<DT>::C* __restrict__ Om, int s,
                                                        const double* __restrict__ D,
                                                        typename Stor<DT>::C* __restrict__ W) {
  using C = typename Stor<DT>::C;
  __shared__ C As[GK][GT + 1];
  __shared__ C Bs[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t m0 = (int64_t)blockIdx.x * GT;
  const int n0 = blockIdx.y * GT;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = C(0);
  for (int64_t k0 = 0; k0 < d; k0 += GK) {
    for (int idx = threadIdx.x; idx < GK * GT; idx += 256) {
      const int kk = idx % GK, mm = idx / GK;  // A row-major: consecutive k
      const int64_t k = k0 + kk, m = m0 + mm;
      As[kk][mm] = (k < d && m < n) ? load_elem<DT>(Araw, m * ld + k) : C(0);
      const int nn = idx / GK;
      const int c = n0 + nn;
      Bs[kk][nn] = (k < d && c < s) ? Om[k + (int64_t)c * d] : C(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + tx + 16 * i;
    if (m >= n) continue;
    const double dm = D ? D[m] : 1.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + ty + 16 * j;
      if (c < s) W[m + (int64_t)c * n] = (C)(dm * (double)acc[i][j]);
    }
  }
}

// Partial Y_z (d x s) = A[rows z]^T W[rows z]
template <int DT>
__global__ void __launch_bounds__(256) sketch_atw_kernel(const unsigned char* __restrict__ Araw, int64_t n,
                                                         int64_t d, int64_t ld,
                                                         const typename Stor<DT>::C* __restrict__ W, int s,
                                                         int64_t kchunk, typename Stor<DT>::C* __restrict__ Yp) {
  using C = typename Stor<DT>::C;
  __shared__ C As[GK][GT + 1];
  __shared__ C Bs[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t j0 = (int64_t)blockIdx.x * GT;
  const int c0 = blockIdx.y * GT;
  const int64_t kb = (int64_t)blockIdx.z * kchunk, ke = min(n, kb + kchunk);
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = C(0);
  for (int64_t k0 = kb; k0 < ke; k0 += GK) {
    for (int idx = threadIdx.x; idx < GK * GT; idx += 256) {
      const int jj = idx % GT, kk = idx / GT;  // A row-major: consecutive j
      const int64_t k = k0 + kk, j = j0 + jj;
      As[kk][jj] = (k < ke && j < d) ? load_elem<DT>(Araw, k * ld + j) : C(0);
      const int kk2 = idx % GK, cc = idx / GK;  // W column-major: consecutive k
      const int64_t k2 = k0 + kk2;
      const int c = c0 + cc;
      Bs[kk2][cc] = (k2 < ke && c < s) ? W[k2 + (int64_t)c * n] : C(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  C* Y = Yp + (int64_t)blockIdx.z * d * s;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t j = j0 + tx + 16 * i;
    if (j >= d) continue;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int c = c0 + ty + 16 * jj;
      if (c < s) Y[j + (int64_t)c * d] = acc[i][jj];
    }
  }
}

template <typename C>
__global__ void sum_partials_to_f64_kernel(const C* __restrict__ Yp, int nz, int64_t len, double* __restrict__ Y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += (double)Yp[z * len + i];
    Y[i] = s;
  }
}

static int64_t atw_kchunk(int64_t n, int64_t d, int s) {
  // enough z-splits to give ~4 CTAs per SM worth of tiles, chunks of >= 1024 rows
  const int64_t tiles = ((d + GT - 1) / GT) * ((s + GT - 1) / GT);
  int64_t nz = std::max<int64_t>(1, (152 * 4 + tiles - 1) / tiles);
  nz = std::min<int64_t>(nz, std::max<int64_t>(1, n / 1024));
  int64_t kc = (n + nz - 1) / nz;
  kc = (kc + GK - 1) / GK * GK;
  return kc;
}

size_t sketch_atw_work_bytes(const nys_matrix* A, int s) {
  const int64_t kc = atw_kchunk(A->n, A->d, s);
  const int64_t nz = (A->n + kc - 1) / kc;
  const size_t csz = compute_is_f64(A->dtype) ? 8 : 4;
  return (size_t)nz * A->d * s * csz;
}

cudaError_t sketch_aw(const nys_matrix* A, const void* Omega, int s, const double* D, void* W, cudaStream_t st) {
  dim3 grid((unsigned)((A->n + GT - 1) / GT), (s + GT - 1) / GT, 1);
  const unsigned char* Ar = reinterpret_cast<const unsigned char*>(A->data);
  switch (A->dtype) {
    case NYS_F64:
      count_launch();
      sketch_aw_kernel<NYS_F64><<<grid, 256, 0, st>>>(Ar, A->n, A->d, A->ld, (const double*)Omega, s, D, (double*)W);
      break;
    case NYS_F32:
      count_launch();
      sketch_aw_kernel<NYS_F32><<<grid, 256, 0, st>>>(Ar, A->n, A->d, A->ld, (const float*)Omega, s, D, (float*)W);
      break;
    case NYS_BF16:
      count_launch();
      sketch_aw_kernel<NYS_BF16><<<grid, 256, 0, st>>>(Ar, A->n, A->d, A->ld, (const float*)Omega, s, D, (float*)W);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t sketch_atw(const nys_matrix* A, const void* W, int s, double* Y, void* work, size_t work_bytes,
                       cudaStream_t st) {
  const int64_t kc = atw_kchunk(A->n, A->d, s);
  const int nz = (int)((A->n + kc - 1) / kc);
  if (work_bytes < sketch_atw_work_bytes(A, s)) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((A->d + GT - 1) / GT), (s + GT - 1) / GT, nz);
  const unsigned char* Ar = reinterpret_cast<const unsigned char*>(A->data);
  const int64_t len = A->d * s;
  const unsigned rb = (unsigned)std::min<int64_t>(4096, (len + 255) / 256);
  switch (A->dtype) {
    case NYS_F64:
      count_launch();
      sketch_atw_kernel<NYS_F64><<<grid, 256, 0, st>>>(Ar, A->n, A->d, A->ld, (const double*)W, s, kc, (double*)work);
      NYS_CUDA_TRY(cudaGetLastError());
      count_launch();
      sum_partials_to_f64_kernel<double><<<rb, 256, 0, st>>>((const double*)work, nz, len, Y);
      break;
    case NYS_F32:
      count_launch();
      fgemm_kernel<NYS_F32, true><<<dim3((unsigned)((A->d + FBM - 1) / FBM), (s + FBN - 1) / FBN, nz), 256, 0, st>>>(
          Ar, A->ld, A->d, s, A->n, kc, (const float*)W, A->n, nullptr, (float*)work, A->d, A->d * s);
      NYS_CUDA_TRY(cudaGetLastError());
      count_launch();
      sum_partials_to_f64_kernel<float><<<rb, 256, 0, st>>>((const float*)work, nz, len, Y);
      break;
    case NYS_BF16:
      count_launch();
      fgemm_kernel<NYS_BF16, true><<<dim3((unsigned)((A->d + FBM - 1) / FBM), (s + FBN - 1) / FBN, nz), 256, 0, st>>>(
          Ar, A->ld, A->d, s, A->n, kc, (const float*)W, A->n, nullptr, (float*)work, A->d, A->d * s);
      NYS_CUDA_TRY(cudaGetLastError());
      count_launch();
      sum_partials_to_f64_kernel<float><<<rb, 256, 0, st>>>((const float*)work, nz, len, Y);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Partials of A^T W only (nz slices of d x s in compute type); returns nz.
cudaError_t sketch_atw_partials(const nys_matrix* A, const void* W, int s, void* work, size_t work_bytes, int* nz_out,
                                cudaStream_t st) {
  const int64_t kc = atw_kchunk(A->n, A->d, s);
  const int nz = (int)((A->n + kc - 1) / kc);
  if (work_bytes < sketch_atw_work_bytes(A, s)) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((A->d + GT - 1) / GT), (s + GT - 1) / GT, nz);
  const unsigned char* Ar = reinterpret_cast<const unsigned char*>(A->data);
  count_launch();
  switch (A->dtype) {
    case NYS_F64:
      sketch_atw_kernel<NYS_F64><<<grid, 256, 0, st>>>(Ar, A->n, A->d, A->ld, (const double*)W, s, kc, (double*)work);
      break;
    case NYS_F32:
      fgemm_kernel<NYS_F32, true><<<dim3((unsigned)((A->d + FBM - 1) / FBM), (s + FBN - 1) / FBN, nz), 256, 0, st>>>(
          Ar, A->ld, A->d, s, A->n, kc, (const float*)W, A->n, nullptr, (float*)work, A->d, A->d * s);
      break;
    case NYS_BF16:
      fgemm_kernel<NYS_BF16, true><<<dim3((unsigned)((A->d + FBM - 1) / FBM), (s + FBN - 1) / FBN, nz), 256, 0, st>>>(
          Ar, A->ld, A->d, s, A->n, kc, (const float*)W, A->n, nullptr, (float*)work, A->d, A->d * s);
      break;
    default: return cudaErrorInvalidValue;
  }
  *nz_out = nz;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ input checks
// *flag |= 1 when any of the n values (FP64, or FP32 when f32) is NaN or infinite.
__global__ void nonfinite_kernel(const void* __restrict__ x, int64_t n, int f32, int* flag) {
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = f32 ? (double)reinterpret_cast<const float*>(x)[i] : reinterpret_cast<const double*>(x)[i];
    bad |= !isfinite(v);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t any_nonfinite(const void* x, int64_t n, bool f32, int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  nonfinite_kernel<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, st>>>(x, n, f32 ? 1 : 0, flag);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ conversions
__global__ void f64_to_f32_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void f32_to_f64_kernel(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
// FP8 E4M3 with per-column scales -> FP32 (same row-major layout and ld).
__global__ void dequantize_fp8_kernel(const unsigned char* __restrict__ q, int64_t n, int64_t d, int64_t ld,
                                      const float* __restrict__ scale, float* __restrict__ out) {
  const int64_t total = n * ld;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx % ld;
    float v = 0.f;
    if (j < d) {
      const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q[idx], __NV_E4M3);
      v = __half2float(*reinterpret_cast<const __half*>(&h)) * scale[j];
    }
    out[idx] = v;
  }
}

cudaError_t dequantize_fp8(const nys_matrix* A, float* out, cudaStream_t st) {
  if (A->dtype != NYS_FP8E4M3 || !A->col_scale) return cudaErrorInvalidValue;
  count_launch();
  dequantize_fp8_kernel<<<(unsigned)std::min<int64_t>(8192, (A->n * A->ld + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const unsigned char*>(A->data), A->n, A->d, A->ld, A->col_scale, out);
  return cudaGetLastError();
}

cudaError_t convert_f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  f64_to_f32_kernel<<<(unsigned)std::min<int64_t>(4096, (n + 255) / 256), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}
cudaError_t convert_f32_to_f64(const float* x, double* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  f32_to_f64_kernel<<<(unsigned)std::min<int64_t>(4096, (n + 255) / 256), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

}  // namespace nys
