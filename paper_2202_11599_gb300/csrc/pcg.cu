// Nystrom PCG (App. B, Alg. Nystrom PCG) on the device, plus the ADMM vector
// steps of Alg. NysADMM (z-prox by soft-thresholding, scaled dual update,
// primal/dual residuals of Sec. 2.1).
//
// One PCG iteration is six stream-ordered launches; every scalar (alpha, beta,
// ||w||, the stop test) lives in a device PcgState, so the host only reads the
// state once per chunk of iterations.  Kernels launched past convergence see
// `done` and return at once, which keeps the iterate sequence identical to a
// host-checked loop.  All reductions are fixed-order (run-to-run identical).
#include "device_util.cuh"
#include "solver.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

namespace nys {

// Fixed-order sum of n doubles by one warp; all lanes get the result.
__device__ __forceinline__ double warp_fixed_sum(const double* a, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += a[i];
  return warp_sum(s);
}

// Block-wide broadcast of warp 0's fixed-order sum.
__device__ __forceinline__ double block_fixed_sum(const double* a, int n, double* slot) {
  if (threadIdx.x < 32) {
    const double s = warp_fixed_sum(a, n);
    if (threadIdx.x == 0) *slot = s;
  }
  __syncthreads();
  const double r = *slot;
  __syncthreads();
  return r;
}

// Same sums reading through L2 (__ldcg): for partials written by other blocks of the
// running kernel, which this block's L1 may not see.
__device__ __forceinline__ double warp_fixed_sum_cg(const double* a, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += __ldcg(a + i);
  return warp_sum(s);
}
__device__ __forceinline__ double block_fixed_sum_cg(const double* a, int n, double* slot) {
  if (threadIdx.x < 32) {
    const double s = warp_fixed_sum_cg(a, n);
    if (threadIdx.x == 0) *slot = s;
  }
  __syncthreads();
  const double r = *slot;
  __syncthreads();
  return r;
}

// Two fixed-order sums of the same kind as block_fixed_sum_cg in one pass (same values).
__device__ __forceinline__ void block_fixed_sum2_cg(const double* a, const double* b, int n, double* out_a,
                                                    double* out_b, double* slot2) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x & 31;
    double sa = 0.0, sb = 0.0;
    for (int i = lane; i < n; i += 32) {
      sa += __ldcg(a + i);
      sb += __ldcg(b + i);
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (threadIdx.x == 0) {
      slot2[0] = sa;
      slot2[1] = sb;
    }
  }
  __syncthreads();
  *out_a = slot2[0];
  *out_b = slot2[1];
  __syncthreads();
}

// Five block_sum<kVecThreads> reductions with one pair of barriers (same values as five calls),
// results in thread 0 only.
__device__ __forceinline__ void block_sum5(double (&v)[5]) {
  __shared__ double sh5[5][kVecThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 5; ++t) v[t] = warp_sum(v[t]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < 5; ++t) sh5[t][w] = v[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < kVecThreads / 32; ++i) s += sh5[t][i];
      v[t] = s;
    }
  }
  __syncthreads();
}

// Last-block election for a kernel that ends with a grid-wide scalar step: every block
// calls it after writing its partials; it returns true (to every thread) only in the block
// that arrived last, which then sees the other blocks' writes, and resets the ticket for
// the next launch.  This replaces a separate one-block kernel launch.
__device__ __forceinline__ bool last_block_done(unsigned int* ticket) {
  __shared__ unsigned int prev;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) prev = atomicAdd(ticket, 1u);
  __syncthreads();
  if (prev != gridDim.x - 1) return false;
  __threadfence();
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__global__ void pcg_reset_kernel(PcgState* st, double tol, int tol_abs, int maxit, int fixed,
                                 const double* dev_tol) {
  st->wy = 0.0;
  st->w2 = 0.0;
  st->r2 = 0.0;
  st->thresh2 = 0.0;
  st->tol = dev_tol ? *dev_tol : tol;
  st->tol_abs = dev_tol ? 1 : tol_abs;
  st->iters = 0;
  st->done = 0;
  st->status = 0;
  st->maxit = maxit;
  st->fixed = fixed;
  st->ticket[0] = 0u;
  st->ticket[1] = 0u;
}

// K4 body (run by the last block of K3): ||w||^2, stop test, iteration count,
// Partials of U^T w over one block's chunk of w (in shared memory, len elements from j0):
// out[i] = sum over the chunk of U[i, j] w_j, each lane adding its lane-strided elements in
// increasing j, then a warp sum.  Eight rows of U per warp pass keep 64 loads in flight.
template <typename C>
__device__ __forceinline__ void utw_partials(const C* wch, int len, const C* __restrict__ U, int64_t d, int64_t j0,
                                             int s, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int RW = 8;
  for (int i0 = warp * RW; i0 < s; i0 += (kVecThreads / 32) * RW) {
    C acc[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) acc[q] = C(0);
#pragma unroll 8
    for (int jj = lane; jj < len; jj += 32) {
      const C wv = wch[jj];
#pragma unroll
      for (int q = 0; q < RW; ++q)
        if (i0 + q < s) acc[q] = fma(U[(int64_t)(i0 + q) * d + j0 + jj], wv, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) acc[q] = warp_sum(acc[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < RW; ++q)
        if (i0 + q < s) out[i0 + q] = (double)acc[q];
    }
  }
}

// g_i = c_i (U^T w)_i.
template <typename C>
__device__ void pcg_scalar_body(int init, int nb3, const double* part_w2, const double* part_r2,
                                const double* part_g, int s, const C* __restrict__ cvec, C* __restrict__ gs,
                                const double* pv_part, int npv, const double* wy_part, int nwy, PcgState* st,
                                cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double slot;
  const double w2 = block_fixed_sum_cg(part_w2, nb3, &slot);
  double r2 = 0.0, pv = 1.0, wy = 0.0;
  if (init) {
    r2 = block_fixed_sum_cg(part_r2, nb3, &slot);
  } else {
    pv = block_fixed_sum(pv_part, npv, &slot);
    wy = block_fixed_sum(wy_part, nwy, &slot);
  }
  if (threadIdx.x == 0) {
    if (init) {
      st->r2 = r2;
      st->thresh2 = st->tol_abs ? st->tol * st->tol : st->tol * st->tol * r2;
      st->iters = 0;
    } else {
      if (!(pv > 0.0) || !isfinite(pv) || !isfinite(w2)) {
        // First iteration: H + rho I is not positive definite on p (a bad input).
        // Later: the recursion has reached the rounding floor of the compute type;
        // the current x (from the previous iteration) is kept and reported unconverged.
        st->status = st->iters == 0 ? NYS_EBREAKDOWN : NYS_ENOCONV;
        st->done = 1;
      } else {
        st->wy = wy;
        st->iters += 1;
      }
    }
    if (!st->done) {
      st->w2 = w2;
      if (st->fixed >= 0) {
        if (st->iters >= st->fixed) st->done = 1;
      } else if (!(w2 > st->thresh2)) {
        st->done = 1;
      } else if (st->iters >= st->maxit) {
        st->done = 1;
        st->status = NYS_ENOCONV;
      }
    }
  }
  for (int i = threadIdx.x; i < s; i += kVecThreads) {
    const double g = sum_strided_fixed<true>(part_g, nb3, s, i, 0.0);
    gs[i] = (C)((double)cvec[i] * g);
  }
  __syncthreads();
  if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// K3: init  -> w = r - v (v = (H + rho I) x0, or x0 = 0), partial ||r||^2;
//     step  -> alpha = w^T y / p^T v, x += alpha p, w -= alpha v.
// Both: partial ||w||^2 and partial U^T w over this block's chunk of w; the last block
// to finish then runs the scalar step K4 (pcg_scalar_body) and sets the loop condition.
template <typename C>
__global__ void __launch_bounds__(kVecThreads) pcg_update_kernel(int init, int64_t d, int chunk, C* __restrict__ x,
                                                                 C* __restrict__ w, const C* __restrict__ r,
                                                                 const C* __restrict__ v, const C* __restrict__ p,
                                                                 const C* __restrict__ U, int s,
                                                                 const double* __restrict__ pv_part, int npv,
                                                                 const double* __restrict__ wy_part, int nwy,
                                                                 double* part_w2, double* part_r2, double* part_g,
                                                                 PcgState* st, C* __restrict__ hx,
                                                                 const C* __restrict__ cvec, C* __restrict__ gs,
                                                                 cudaGraphConditionalHandle cond, int use_cond,
                                                                 const double* __restrict__ rq,
                                                                 const double* __restrict__ rz,
                                                                 const double* __restrict__ ru, double rrho,
                                                                 C* __restrict__ r_out) {
  if (st->done) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* wch = reinterpret_cast<C*>(sm_raw);
  __shared__ double sh[kVecThreads / 32];
  __shared__ double slot;
  const int64_t j0 = (int64_t)blockIdx.x * chunk;
  const int64_t j1 = min(d, j0 + chunk);
  double alpha = 0.0;
  bool bad = false;
  if (!init) {
    const double pv = block_fixed_sum(pv_part, npv, &slot);
    const double wy = block_fixed_sum(wy_part, nwy, &slot);
    bad = !(pv > 0.0) || !isfinite(pv);  // breakdown: flagged by the scalar step
    if (!bad) alpha = wy / pv;
  }
  if (!bad) {
    const C a = (C)alpha;
    double lw2 = 0.0, lr2 = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += kVecThreads) {
      C wj;
      if (init) {
        // with rq: the ADMM right-hand side r = q + rho (z - u) is formed here (and stored)
        C rj;
        if (rq) {
          rj = (C)fma(rrho, rz[j] - ru[j], rq[j]);
          r_out[j] = rj;
        } else {
          rj = r[j];
        }
        wj = v ? rj - v[j] : rj;
        lr2 += (double)rj * (double)rj;
      } else {
        const C vj = v[j];
        x[j] = fma(a, p[j], x[j]);
        wj = fma(-a, vj, w[j]);
        if (hx) hx[j] = fma(a, vj, hx[j]);  // (H + rho I) x follows x: x += a p  =>  += a v
      }
      w[j] = wj;
      wch[j - j0] = wj;
      lw2 += (double)wj * (double)wj;
    }
    const double tw2 = block_sum_t0<kVecThreads>(lw2, sh);
    const double tr2 = block_sum_t0<kVecThreads>(lr2, sh);
    if (threadIdx.x == 0) {
      part_w2[blockIdx.x] = tw2;
      if (init) part_r2[blockIdx.x] = tr2;
    }
    __syncthreads();
    utw_partials<C>(wch, (int)(j1 - j0), U, d, j0, s, part_g + (int64_t)blockIdx.x * s);
  }
  if (!last_block_done(&st->ticket[0])) return;
  pcg_scalar_body<C>(init, (int)gridDim.x, part_w2, part_r2, part_g, s, cvec, gs, pv_part, npv, wy_part, nwy, st,
                     cond, use_cond);
}

// K5: y = w + U gs (= P^{-1} w), partial w^T y; when p is given, the last block to finish
// runs K6 over the whole vector: beta = (w^T y)_new / (w^T y)_old, p = y + beta p
// (init: p = y).
template <typename C>
__global__ void __launch_bounds__(kVecThreads) pcg_tail_kernel(int64_t d, const C* __restrict__ w, C* __restrict__ y,
                                                               const C* __restrict__ U, int s,
                                                               const C* __restrict__ gs, double* part_wy,
                                                               PcgState* st, int init, C* __restrict__ p) {
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* g = reinterpret_cast<C*>(sm_raw);
  __shared__ double sh[kVecThreads / 32];
  __shared__ double slot;
  for (int i = threadIdx.x; i < s; i += kVecThreads) g[i] = gs[i];
  __syncthreads();
  double lwy = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)gridDim.x * kVecThreads) {
    const C wj = w[j];
    const C acc = urow_dot(U, d, j, s, g, wj);
    y[j] = acc;
    lwy += (double)wj * (double)acc;
  }
  const double t = block_sum_t0<kVecThreads>(lwy, sh);
  if (threadIdx.x == 0) part_wy[blockIdx.x] = t;
  if (!p) return;
  if (!last_block_done(&st->ticket[1])) return;
  double beta = 0.0;
  if (!init) beta = block_fixed_sum_cg(part_wy, (int)gridDim.x, &slot) / st->wy;
  const C b = (C)beta;
  for (int64_t j = threadIdx.x; j < d; j += kVecThreads) {
    const C yj = __ldcg(y + j);
    p[j] = init ? yj : fma(b, p[j], yj);
  }
}

// Row-sharded matvec, after the sum over ranks of the local A_g^T D_g A_g p (in v):
// v = rho p + v and the per-block partials of p^T v, with the loop and order of
// apass_reduce_kernel (so an unsharded run and a one-rank sharded run agree bitwise).
template <typename C>
__global__ void __launch_bounds__(kVecThreads) shard_finish_kernel(int64_t d, C rho, const C* __restrict__ p,
                                                                   C* __restrict__ v, double* dot_part, const int* skip) {
  if (skip && *skip) return;
  __shared__ double sh[kVecThreads / 32];
  double dacc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    const C pj = p ? p[j] : C(0);
    const C yj = fma(rho, pj, v[j]);
    v[j] = yj;
    dacc += (double)pj * (double)yj;
  }
  if (dot_part) {
    const double t = block_sum_t0<kVecThreads>(dacc, sh);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = t;
  }
}

// v = (A^T D A + rho I) p with the row sum completed over the ranks of a sharded solve.
template <typename C>
static cudaError_t sharded_reduce(const ApassArgs& aa, const ApassPlan& plan, const void* apart, double rho, C* v,
                                  double* dot_part, int nblk, cudaStream_t stream, nys_status* comm_status) {
  NYS_CUDA_TRY(apass_reduce(aa, plan, apart, 0.0, v, nullptr, 0, stream));  // local sum, no shift
  const nys_status cs = shard_sum(v, aa.d, sizeof(C) == 8 ? NYS_F64 : NYS_F32, stream);
  if (cs != NYS_OK) {
    *comm_status = cs;
    return cudaErrorUnknown;
  }
  count_launch();
  shard_finish_kernel<C><<<nblk, kVecThreads, 0, stream>>>(aa.d, (C)rho, reinterpret_cast<const C*>(aa.p), v, dot_part,
                                                             aa.skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ host driver

static int upd_chunk(int64_t d) {
  // ~2 blocks per SM at large d, >= 256 elements per block
  int64_t ch = std::max<int64_t>(256, (d + 303) / 304);
  ch = (ch + 31) / 32 * 32;
  return (int)ch;
}

int pcg_nb3(int64_t d) { return (int)((d + upd_chunk(d) - 1) / upd_chunk(d)); }

template <typename C>
nys_status pcg_run(const PcgProblem& pb, const PrecondView& P, const C* r, C* x, const PcgParams& prm,
                   cudaStream_t stream, int* iters_out, double* resnorm_out) {
  Pool pool(stream);
  const int64_t d = pb.A->d;
  const int s = P.s;
  const C* U = reinterpret_cast<const C*>(P.U);
  const C* cvec = reinterpret_cast<const C*>(P.c);
  const int chunk = upd_chunk(d);
  const int nb3 = (int)((d + chunk - 1) / chunk);
  const int nbr = reduce_blocks(d);
  const int nb5 = nbr;

  C* w = pool.alloc<C>(d);
  C* y = pool.alloc<C>(d);
  C* p = pool.alloc<C>(d);
  C* v = pool.alloc<C>(d);
  C* gs = pool.alloc<C>(std::max(1, s));
  double* part_w2 = pool.alloc<double>(nb3);
  double* part_r2 = pool.alloc<double>(nb3);
  double* part_g = pool.alloc<double>((size_t)nb3 * std::max(1, s));
  double* pv_part = pool.alloc<double>(nbr);
  double* wy_part = pool.alloc<double>(nb5);
  void* apart = pool.alloc<unsigned char>(apass_partial_bytes(pb.A, pb.plan));
  PcgState* st = pool.alloc<PcgState>(1);
  int* dstat = pool.alloc<int>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  if (cudaMemsetAsync(dstat, 0, sizeof(int), stream) != cudaSuccess) return NYS_ECUDA;

  ApassArgs aa;
  aa.A = pb.A->data;
  aa.n = pb.A->n;
  aa.d = d;
  aa.ld = pb.A->ld;
  aa.dtype = pb.A->dtype;
  aa.col_scale = pb.A->col_scale;
  aa.D = pb.D;
  aa.b = nullptr;
  aa.D_out = nullptr;
  aa.t_out = nullptr;
  aa.mode = pb.D ? MODE_DIAG : MODE_ID;
  aa.skip = &st->done;

  const size_t sm_upd = (size_t)chunk * sizeof(C);
  const size_t sm_tail = (size_t)std::max(1, s) * sizeof(C);
  cudaError_t e = cudaSuccess;
#define LAUNCH_OK(x)                \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return NYS_ECUDA; \
  } while (0)

  count_launch();
  pcg_reset_kernel<<<1, 1, 0, stream>>>(st, prm.tol, prm.tol_abs, prm.maxit, prm.fixed, prm.dev_tol);
  LAUNCH_OK(cudaGetLastError());
  const bool sharded = shard_comm().fn != nullptr;
  nys_status comm_status = NYS_OK;
#define MATVEC_REDUCE(rho_, dots_, nd_)                                                                  \
  do {                                                                                                  \
    if (sharded) {                                                                                      \
      e = sharded_reduce<C>(aa, pb.plan, apart, (rho_), v, (dots_), nbr, stream, &comm_status);          \
      if (comm_status != NYS_OK) return comm_status;                                                    \
      if (e != cudaSuccess) return NYS_ECUDA;                                                           \
    } else {                                                                                            \
      LAUNCH_OK(apass_reduce(aa, pb.plan, apart, (rho_), v, (dots_), (nd_), stream));                  \
    }                                                                                                   \
  } while (0)
  const C* v0 = nullptr;
  if (!prm.x0_zero) {
    aa.p = x;
    const int* skip0 = aa.skip;
    aa.skip = nullptr;
    LAUNCH_OK(apass_run(aa, pb.plan, apart, nullptr, dstat, stream));
    MATVEC_REDUCE(pb.rho, nullptr, 0);
    aa.skip = skip0;
    v0 = v;
  }
  count_launch();
  pcg_update_kernel<C><<<nb3, kVecThreads, sm_upd, stream>>>(1, d, chunk, x, w, r, v0, p, U, s, pv_part, nbr,
                                                             wy_part, nb5, part_w2, part_r2, part_g, st, (C*)nullptr,
                                                             cvec, gs, 0ull, 0, nullptr, nullptr, nullptr, 0.0,
                                                             (C*)nullptr);
  LAUNCH_OK(cudaGetLastError());
  count_launch();
  pcg_tail_kernel<C><<<nb5, kVecThreads, sm_tail, stream>>>(d, w, y, U, s, gs, wy_part, st, 1, p);
  LAUNCH_OK(cudaGetLastError());

  PcgState* hs = host_state();
  int launched = 0;
  const int cap = prm.fixed >= 0 ? prm.fixed : prm.maxit;
  int chunk_it = std::max(1, std::min(4, cap));
  for (;;) {
    for (int c = 0; c < chunk_it && launched < cap; ++c, ++launched) {
      aa.p = p;
      LAUNCH_OK(apass_run(aa, pb.plan, apart, nullptr, dstat, stream));
      MATVEC_REDUCE(pb.rho, pv_part, nbr);
      count_launch();
      pcg_update_kernel<C><<<nb3, kVecThreads, sm_upd, stream>>>(0, d, chunk, x, w, r, v, p, U, s, pv_part, nbr,
                                                                 wy_part, nb5, part_w2, part_r2, part_g, st, (C*)nullptr,
                                                                 cvec, gs, 0ull, 0, nullptr, nullptr, nullptr, 0.0,
                                                                 (C*)nullptr);
      LAUNCH_OK(cudaGetLastError());
      count_launch();
      pcg_tail_kernel<C><<<nb5, kVecThreads, sm_tail, stream>>>(d, w, y, U, s, gs, wy_part, st, 0, p);
      LAUNCH_OK(cudaGetLastError());
    }
    LAUNCH_OK(cudaMemcpyAsync(hs, st, sizeof(PcgState), cudaMemcpyDeviceToHost, stream));
    LAUNCH_OK(cudaStreamSynchronize(stream));
    if (hs->done || launched >= cap) break;
    chunk_it = std::min(32, chunk_it * 2);
  }
  int dstat_h = 0;
  LAUNCH_OK(cudaMemcpyAsync(&dstat_h, dstat, sizeof(int), cudaMemcpyDeviceToHost, stream));
  LAUNCH_OK(cudaStreamSynchronize(stream));
#undef LAUNCH_OK
#undef MATVEC_REDUCE
  if (iters_out) *iters_out = hs->iters;
  if (resnorm_out) *resnorm_out = std::sqrt(hs->w2);
  if (dstat_h) return (nys_status)dstat_h;
  if (!hs->done && prm.fixed < 0) return NYS_ENOCONV;
  return (nys_status)hs->status;
}

template nys_status pcg_run<double>(const PcgProblem&, const PrecondView&, const double*, double*, const PcgParams&,
                                    cudaStream_t, int*, double*);
template nys_status pcg_run<float>(const PcgProblem&, const PrecondView&, const float*, float*, const PcgParams&,
                                   cudaStream_t, int*, double*);

// ------------------------------------------------------------------ P^{-1} on k vectors (standalone apply)
template <typename C>
nys_status precond_apply_run(const PrecondView& P, int64_t d, const C* V, C* Y, int64_t k, cudaStream_t stream) {
  Pool pool(stream);
  const int s = P.s;
  const int chunk = upd_chunk(d);
  const int nb3 = (int)((d + chunk - 1) / chunk);
  const int nb5 = reduce_blocks(d);
  C* w = pool.alloc<C>(d);
  C* gs = pool.alloc<C>(std::max(1, s));
  double* part_w2 = pool.alloc<double>(nb3);
  double* part_r2 = pool.alloc<double>(nb3);
  double* part_g = pool.alloc<double>((size_t)nb3 * std::max(1, s));
  double* wy_part = pool.alloc<double>(nb5);
  PcgState* st = pool.alloc<PcgState>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  for (int64_t c = 0; c < k; ++c) {
    count_launch();
    pcg_reset_kernel<<<1, 1, 0, stream>>>(st, 0.0, 1, 1, -1, nullptr);
    // init-mode update copies V[:, c] into w and forms the partials of U^T w
    count_launch();
    pcg_update_kernel<C><<<nb3, kVecThreads, (size_t)chunk * sizeof(C), stream>>>(
        1, d, chunk, nullptr, w, V + c * d, nullptr, nullptr, reinterpret_cast<const C*>(P.U), s, nullptr, 0,
        nullptr, 0, part_w2, part_r2, part_g, st, (C*)nullptr, reinterpret_cast<const C*>(P.c), gs, 0ull, 0, nullptr,
        nullptr, nullptr, 0.0, (C*)nullptr);
    // the scalar step may mark the state done (||w|| <= 0 threshold); force the tail to run
    count_launch();
    pcg_reset_kernel<<<1, 1, 0, stream>>>(st, 0.0, 1, 1, -1, nullptr);
    count_launch();
    pcg_tail_kernel<C><<<nb5, kVecThreads, (size_t)std::max(1, s) * sizeof(C), stream>>>(
        d, w, Y + c * d, reinterpret_cast<const C*>(P.U), s, gs, wy_part, st, 1, (C*)nullptr);
    if (cudaGetLastError() != cudaSuccess) return NYS_ECUDA;
  }
  if (cudaStreamSynchronize(stream) != cudaSuccess) return NYS_ECUDA;
  return NYS_OK;
}

template nys_status precond_apply_run<double>(const PrecondView&, int64_t, const double*, double*, int64_t,
                                              cudaStream_t);
template nys_status precond_apply_run<float>(const PrecondView&, int64_t, const float*, float*, int64_t, cudaStream_t);

// ------------------------------------------------------------------ ADMM vector kernels (FP64 state)

// r = q + rho (z - u)   or, for the refined x-step, the residual of Eq. ADMMSubProb at x:
// r = rho (z - u - x) - mu x - yres  (yres = A^T (A x - b); mu = 0 except for H^g = mu I)
template <typename C>
__global__ void admm_rhs_kernel(int64_t d, const double* __restrict__ q, const double* __restrict__ z,
                                const double* __restrict__ u, double rho, const double* __restrict__ x,
                                const double* __restrict__ yres, C* __restrict__ r, double mu) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    const double zu = z[j] - u[j];
    const double rj = yres ? rho * (zu - x[j]) - mu * x[j] - yres[j] : fma(rho, zu, q[j]);
    r[j] = (C)rj;
  }
}

// x <- xc (or x += xc), z_old = z, z = S_kappa(x + u), u += x - z, residual partials.
template <typename C>
__global__ void __launch_bounds__(kVecThreads) admm_zu_kernel(int64_t d, const C* __restrict__ xc, int accumulate,
                                                              double* __restrict__ x, double* __restrict__ z,
                                                              double* __restrict__ u, double kappa,
                                                              double* __restrict__ ztrace, double* part5) {
  __shared__ double sh[kVecThreads / 32];
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
  for (int64_t j = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)gridDim.x * kVecThreads) {
    const double xj = accumulate ? x[j] + (double)xc[j] : (double)xc[j];
    const double zo = z[j];
    const double vj = xj + u[j];
    const double mag = fabs(vj) - kappa;
    const double zj = mag > 0.0 ? copysign(mag, vj) : 0.0;
    const double uj = u[j] + xj - zj;
    x[j] = xj;
    z[j] = zj;
    u[j] = uj;
    if (ztrace) ztrace[j] = zj;
    a0 += (xj - zj) * (xj - zj);
    a1 += (zj - zo) * (zj - zo);
    a2 += xj * xj;
    a3 += zj * zj;
    a4 += uj * uj;
  }
  a0 = block_sum_t0<kVecThreads>(a0, sh);
  a1 = block_sum_t0<kVecThreads>(a1, sh);
  a2 = block_sum_t0<kVecThreads>(a2, sh);
  a3 = block_sum_t0<kVecThreads>(a3, sh);
  a4 = block_sum_t0<kVecThreads>(a4, sh);
  if (threadIdx.x == 0) {
    double* o = part5 + (int64_t)blockIdx.x * 5;
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
    o[3] = a3;
    o[4] = a4;
  }
}

// Sum of the per-block partials part5[b * 5 + t] over b = 0 .. nb-1 in a fixed order, called
// by one full warp; every lane gets the five sums.  Lane l adds the partials b = l, l + 32,
// ... in increasing b, then a warp tree adds the lanes: a dependent chain of about
// nb / 32 + 5 FP64 adds instead of nb (dependent FP64 adds are slow on this GPU).  Every
// caller -- the host-driven loop, both graph bodies and the cooperative kernels -- uses this
// function, so they agree bit for bit.
constexpr int kPart5Max = 256;
__device__ __forceinline__ void sum_part5(int nb, const double* part5, double (&a)[5]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 5; ++t) a[t] = 0.0;
  for (int b = lane; b < nb; b += 32) {
    const double* o = part5 + (int64_t)b * 5;
#pragma unroll
    for (int t = 0; t < 5; ++t) a[t] += __ldcg(o + t);
  }
#pragma unroll
  for (int t = 0; t < 5; ++t) a[t] = warp_sum(a[t]);
}

// r_p, r_d (Sec. 2.1), the next PCG tolerance sqrt(r_p r_d) (Sec. 5) and the
// residual stopping test.
__global__ void admm_scalar_kernel(int nb, const double* part5, double rho, int k, double* rp_trace,
                                   double* rd_trace, double* eps_next, double eps_abs, double eps_rel, int* stop) {
  double a[5];
  sum_part5(nb, part5, a);
  if (threadIdx.x != 0) return;
  const double rp = sqrt(a[0]);
  const double rd = rho * sqrt(a[1]);
  rp_trace[k] = rp;
  rd_trace[k] = rd;
  *eps_next = sqrt(rp * rd);
  if (eps_rel > 0.0) {
    const double tp = eps_abs + eps_rel * fmax(sqrt(a[2]), sqrt(a[3]));
    const double td = eps_abs + eps_rel * rho * sqrt(a[4]);
    if (rp <= tp && rd <= td) *stop = 1;
  }
}

int admm_blocks(int64_t d) { return reduce_blocks(d); }

template <typename C>
cudaError_t admm_rhs(int64_t d, const double* q, const double* z, const double* u, double rho, const double* x,
                     const double* yres, C* r, cudaStream_t st, double mu) {
  count_launch();
  admm_rhs_kernel<C><<<admm_blocks(d), kVecThreads, 0, st>>>(d, q, z, u, rho, x, yres, r, mu);
  return cudaGetLastError();
}
template cudaError_t admm_rhs<double>(int64_t, const double*, const double*, const double*, double, const double*,
                                      const double*, double*, cudaStream_t, double);
template cudaError_t admm_rhs<float>(int64_t, const double*, const double*, const double*, double, const double*,
                                     const double*, float*, cudaStream_t, double);

template <typename C>
cudaError_t admm_zu(int64_t d, const C* xc, int accumulate, double* x, double* z, double* u, double kappa,
                    double* ztrace, double* part5, cudaStream_t st) {
  count_launch();
  admm_zu_kernel<C><<<admm_blocks(d), kVecThreads, 0, st>>>(d, xc, accumulate, x, z, u, kappa, ztrace, part5);
  return cudaGetLastError();
}
template cudaError_t admm_zu<double>(int64_t, const double*, int, double*, double*, double*, double, double*,
                                     double*, cudaStream_t);
template cudaError_t admm_zu<float>(int64_t, const float*, int, double*, double*, double*, double, double*, double*,
                                    cudaStream_t);

cudaError_t admm_scalar(int64_t d, const double* part5, double rho, int k, double* rp, double* rd, double* eps_next,
                        double eps_abs, double eps_rel, int* stop, cudaStream_t st) {
  count_launch();
  admm_scalar_kernel<<<1, 32, 0, st>>>(admm_blocks(d), part5, rho, k, rp, rd, eps_next, eps_abs, eps_rel, stop);
  return cudaGetLastError();
}

void keep_mempool_cached() {
  static std::atomic<unsigned long long> done_mask{0};   // one bit per device ordinal
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return;
  const unsigned long long bit = 1ull << dev;
  if (done_mask.load(std::memory_order_relaxed) & bit) return;
  cudaMemPool_t mp;
  if (cudaDeviceGetDefaultMemPool(&mp, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done_mask.fetch_or(bit);
}

// Pinned host slot the host-driven PCG loop reads its convergence flags through: one per
// host thread, so threads driving different GPUs (or streams) never share it.
PcgState* host_state() {
  static thread_local PcgState* hs = nullptr;
  if (!hs) {
    if (cudaMallocHost((void**)&hs, sizeof(PcgState)) != cudaSuccess) {
      static thread_local PcgState fallback;
      hs = &fallback;
    }
  }
  return hs;
}

}  // namespace nys

namespace nys {
// =========================================================================== device-side ADMM loop
// The lasso NysADMM loop as ONE CUDA graph: an outer conditional WHILE node runs
// ADMM iterations and an inner one runs PCG iterations; the scalar kernels set the
// loop conditions on the device, so a whole solve needs no host synchronisation.
// The kernels and their order are those of the host-driven loop.
struct AdmmCtl {
  int k;            // ADMM iteration counter
  int stop;         // residual stop reached
  int hx_skip;      // 1: reuse the tracked (H + rho I) x; 0: recompute it this iteration
  unsigned int ticket;  // last-block election of the fused zu / scalar kernel
  long long nodes;  // kernel launches executed (instrumentation)
  double eps_next;  // sqrt(r_p r_d) of the last iteration
  unsigned int bar_count, bar_gen;  // grid barrier of admm_head_kernel
  int hx_pending;   // admm_head_kernel asked for the (H + rho I) x recompute of iteration k
};

namespace {


// PCG tolerance of ADMM iteration k: SQRT_RPRD uses sqrt(r_p r_d) of the previous
// iteration (absolute), ABS the fixed tol, REL the fixed relative tol, and the decaying
// schedule ||r^k|| / k^beta (beta = tol, k counted from 1) a relative tol.
__device__ __forceinline__ void iter_tol(int tol_mode, double tol, double tol_floor, int k, double eps_next,
                                         double* tol_out, int* abs_out) {
  if (tol_mode == NYS_TOL_SQRT_RPRD && k > 0) {
    *tol_out = eps_next;
    *abs_out = 1;
  } else if (tol_mode == NYS_TOL_ABS) {
    *tol_out = tol;
    *abs_out = 1;
  } else {
    const double t = tol_mode == NYS_TOL_RNORM_POW ? pow((double)(k + 1), -tol) : tol;
    *tol_out = fmax(t, tol_floor);
    *abs_out = 0;
  }
}

// The schedule (k + 1)^(-beta) of NYS_TOL_RNORM_POW for k < K, filled once per solve by the
// same device pow that iter_tol calls (so a table entry equals the value iter_tol forms).
__global__ void tolpow_kernel(double* tab, int K, double beta) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) tab[k] = pow((double)(k + 1), -beta);
}

// iter_tol with the power schedule read from tolpow_kernel's table (one load instead of a
// pow on the FP64 pipe in the loop's critical path).
__device__ __forceinline__ void iter_tol_tab(int tol_mode, double tol, double tol_floor, int k, double eps_next,
                                             const double* tab, double* tol_out, int* abs_out) {
  if (tol_mode == NYS_TOL_RNORM_POW && tab) {
    *tol_out = fmax(tab[k], tol_floor);
    *abs_out = 0;
  } else {
    iter_tol(tol_mode, tol, tol_floor, k, eps_next, tol_out, abs_out);
  }
}

// k = 0 and refined steps start from x = 0 (hx = 0); otherwise (H + rho I) x is recomputed
// when hx_refresh == 0 (as printed) or every hx_refresh iterations.  1 = reuse the tracked hx.
__device__ __forceinline__ int iter_hx_skip(int refine, int k, int hx_refresh) {
  if (refine || k == 0) return 1;
  return (hx_refresh == 0 || k % hx_refresh == 0) ? 0 : 1;
}

__global__ void admm_begin_kernel(AdmmCtl* ctl, PcgState* st, double tol, double tol_floor, int tol_mode, int maxit,
                                  const int* __restrict__ fixed_dev, int hx_refresh, int refine,
                                  cudaGraphConditionalHandle hx_cond, long long hx_nodes) {
  const int k = ctl->k;
  st->wy = 0.0;
  st->w2 = 0.0;
  st->r2 = 0.0;
  st->thresh2 = 0.0;
  st->iters = 0;
  st->done = 0;
  st->status = 0;
  st->maxit = maxit;
  st->fixed = fixed_dev ? fixed_dev[k] : -1;
  st->ticket[0] = 0u;
  st->ticket[1] = 0u;
  iter_tol(tol_mode, tol, tol_floor, k, ctl->eps_next, &st->tol, &st->tol_abs);
  ctl->hx_skip = iter_hx_skip(refine, k, hx_refresh);
  // the recompute pass sits in a conditional IF node: skipped iterations launch nothing
  if (!ctl->hx_skip) ctl->nodes += hx_nodes;
  cudaGraphSetConditional(hx_cond, ctl->hx_skip ? 0u : 1u);
}

// r = q + rho (z - u); refined step: r = rho (z - u - x) - mu x - yres, and the PCG starts at 0.
template <typename C>
__global__ void admm_rhs_g_kernel(int64_t d, const double* __restrict__ q, const double* __restrict__ z,
                                  const double* __restrict__ u, double rho, double mu, const double* __restrict__ x,
                                  const double* __restrict__ yres, int refine, C* __restrict__ r, C* __restrict__ xc,
                                  C* __restrict__ hx) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    const double zu = z[j] - u[j];
    if (refine) {
      r[j] = (C)(rho * (zu - x[j]) - mu * x[j] - yres[j]);
      xc[j] = C(0);
      hx[j] = C(0);
    } else {
      r[j] = (C)fma(rho, zu, q[j]);
    }
  }
}

// Scalar step of an ADMM iteration in the graph (one warp of the last zu block): r_p, r_d,
// the next PCG tolerance, the stop test and the WHILE condition.
__device__ void admm_scalar_g_body(int nb, const double* part5, double rho, int K, double eps_abs,
                                     double eps_rel, double* rp_trace, double* rd_trace, int* pcg_it_trace,
                                     const PcgState* st, AdmmCtl* ctl, long long nodes_per_iter,
                                     long long nodes_per_pcg_iter, cudaGraphConditionalHandle cond) {
  double a[5];
  sum_part5(nb, part5, a);  // partials of the running kernel: read through L2
  if (threadIdx.x != 0) return;
  const int k = ctl->k;
  const double rp = sqrt(a[0]);
  const double rd = rho * sqrt(a[1]);
  rp_trace[k] = rp;
  rd_trace[k] = rd;
  pcg_it_trace[k] = st->iters;
  ctl->eps_next = sqrt(rp * rd);
  if (eps_rel > 0.0) {
    const double tp = eps_abs + eps_rel * fmax(sqrt(a[2]), sqrt(a[3]));
    const double td = eps_abs + eps_rel * rho * sqrt(a[4]);
    if (rp <= tp && rd <= td) ctl->stop = 1;
  }
  if (st->status == NYS_EBREAKDOWN) ctl->stop = 2;
  ctl->nodes += nodes_per_iter + nodes_per_pcg_iter * (long long)st->iters;
  ctl->k = k + 1;
  cudaGraphSetConditional(cond, (k + 1 < K && !ctl->stop) ? 1u : 0u);
}

template <typename C>
__global__ void __launch_bounds__(kVecThreads) admm_zu_g_kernel(int64_t d, const C* __restrict__ xc, int accumulate,
                                                                double* __restrict__ x, double* __restrict__ z,
                                                                double* __restrict__ u, double kappa,
                                                                double* __restrict__ ztrace, AdmmCtl* ctl,
                                                                double* part5, double rho, int K, double eps_abs,
                                                                double eps_rel, double* rp_trace, double* rd_trace,
                                                                int* pcg_it_trace, const PcgState* st,
                                                                long long nodes_per_iter, long long nodes_per_pcg_iter,
                                                                cudaGraphConditionalHandle cond) {
  double* zt = ztrace ? ztrace + (int64_t)ctl->k * d : nullptr;
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
  for (int64_t j = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)gridDim.x * kVecThreads) {
    const double xj = accumulate ? x[j] + (double)xc[j] : (double)xc[j];
    const double zo = z[j];
    const double vj = xj + u[j];
    const double mag = fabs(vj) - kappa;
    const double zj = mag > 0.0 ? copysign(mag, vj) : 0.0;
    const double uj = u[j] + xj - zj;
    x[j] = xj;
    z[j] = zj;
    u[j] = uj;
    if (zt) zt[j] = zj;
    a0 += (xj - zj) * (xj - zj);
    a1 += (zj - zo) * (zj - zo);
    a2 += xj * xj;
    a3 += zj * zj;
    a4 += uj * uj;
  }
  double a5[5] = {a0, a1, a2, a3, a4};
  block_sum5(a5);
  if (threadIdx.x == 0) {
    double* o = part5 + (int64_t)blockIdx.x * 5;
#pragma unroll
    for (int t = 0; t < 5; ++t) o[t] = a5[t];
  }
  // the last block to finish runs the scalar step of the iteration
  if (!last_block_done(&ctl->ticket)) return;
  if (threadIdx.x < 32)
    admm_scalar_g_body((int)gridDim.x, part5, rho, K, eps_abs, eps_rel, rp_trace, rd_trace, pcg_it_trace, st, ctl,
                       nodes_per_iter, nodes_per_pcg_iter, cond);
}


// Head of the device loop's ADMM iteration, one cooperative launch (tracked warm start,
// no refined step or warm-start model).  It replaces the begin / right-hand side / PCG-init
// (P^{-1} w) launches of the general body, and it runs the iterations whose x-subproblem
// needs no PCG step -- the common case under the decaying schedules of Sec. 5, where the
// tracked warm start often already meets the iteration's tolerance -- back to back:
//   1. r = q + rho (z - u), w = r - (H + rho I) x (tracked), partial ||w||^2, ||r||^2 and
//      U^T w (blocks, thread mapping and order of pcg_update_kernel's init step);
//   2. every block sums the partials in the order of pcg_scalar_body and takes the same stop
//      decision;
//   3a. no step: x stays; z = S_kappa(x + u), u += x - z and the residual partials (blocks of
//      admm_zu_g_kernel); every block forms r_p, r_d, the stop test and the next tolerance as
//      admm_scalar_g_body does (block 0 records them) and goes on with iteration k + 1;
//   3b. a step: g = c o U^T w (order of pcg_scalar_body), y = w + U g, p = y and the partials
//      of w^T y (blocks and order of pcg_tail_kernel), the PCG state as the begin and init
//      kernels leave it; the PCG WHILE node and the prox/dual kernel finish iteration k.
// When (H + rho I) x is due for a recompute at iteration k the kernel requests it (IF node
// before it) and returns; the next launch continues at k.  The arithmetic and its order are
// those of the general body, so the iterates are bitwise those of a solve without this
// kernel.  Grid barriers are bounded (NYS_ETIMEOUT).
// One PCG iteration after its A-pass as ONE cooperative launch (Alg. Nystrom PCG): the
// reduction of the per-CTA A-pass partials (apass_reduce_kernel), the update of x, w and the
// tracked (H + rho I) x with the partials of ||w||^2 and U^T w (pcg_update_kernel), the
// scalar step (pcg_scalar_body), y = P^{-1} w (pcg_tail_kernel) and the next direction
// p = y + beta p, separated by grid barriers instead of kernel boundaries.  Every element and
// every partial is formed by the same code, block mapping and order as in those kernels, so
// the result is bitwise theirs; data written by other blocks in the same launch is read
// through L2.  With zu set, the iteration that ends the PCG loop also runs the prox / dual
// step and the scalars of the ADMM iteration (admm_zu_g_kernel, admm_scalar_g_body).
template <typename C>
struct PostArgs {
  int64_t d;
  int chunk, nbr, nb3, nb5, nbz;
  const C* partial;      // [G][dpad] A-pass partials
  int G;
  int64_t dpad;
  C rho;                 // rho + mu of the H-matvec
  const float* cscale;   // FP8 column scales, or null
  C *p, *v, *x, *w, *hx, *y;
  const C* U;
  int s;
  const C* cvec;
  C* gs;
  double *pv_part, *wy_part, *part_w2, *part_g;
  PcgState* st;
  cudaGraphConditionalHandle cond;   // the PCG WHILE
  // prox / dual step (zu != 0)
  int zu;
  double *xd, *z, *u, *ztrace, *part5, *rp, *rd;
  int* pcg_it;
  double kappa, rho_admm, eps_abs, eps_rel;
  int K;
  AdmmCtl* ctl;
  cudaGraphConditionalHandle h_admm;
  int* dstat;            // NYS_ETIMEOUT when a grid barrier wait runs out
};

template <typename C>
__global__ void __launch_bounds__(kVecThreads) pcg_post_kernel(const PostArgs<C> a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* wch = reinterpret_cast<C*>(sm_raw);   // chunk of w (U^T w), then g (y = w + U g)
  __shared__ double sh[kVecThreads / 32];
  __shared__ double slot;
  PcgState* st = a.st;
  const int b = blockIdx.x;
  const unsigned nblk = gridDim.x;
  const int64_t d = a.d;
  const int s = a.s;
  // every block reads the state before block 0 changes it below (after two barriers)
  const int done0 = st->done;
  const int iters0 = st->iters, fixed = st->fixed, maxit = st->maxit;
  const double thresh2 = st->thresh2;
  if (done0) {
    if (b == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
    return;
  }
  auto fail = [&]() {
    if (b == 0 && threadIdx.x == 0) {
      atomicExch(a.dstat, (int)NYS_ETIMEOUT);
      st->done = 1;
      cudaGraphSetConditional(a.cond, 0u);
      if (a.zu) cudaGraphSetConditional(a.h_admm, 0u);
    }
  };
  // ---- R: v = sum_g partial[g] + rho p, partials of p^T v (apass_reduce_kernel)
  if (b < a.nbr) {
    double dacc = 0.0;
    for (int64_t j = b * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)a.nbr * kVecThreads) {
      C sj = sum_strided_fixed<false>(a.partial, a.G, a.dpad, j, C(0));
      if (a.cscale) sj *= (C)a.cscale[j];
      const C pj = a.p[j];
      const C yj = fma(a.rho, pj, sj);
      a.v[j] = yj;
      dacc += (double)pj * (double)yj;
    }
    const double t = block_sum_t0<kVecThreads>(dacc, sh);
    if (threadIdx.x == 0) a.pv_part[b] = t;
  }
  if (!grid_barrier(&st->bar_count, &st->bar_gen, nblk)) return fail();
  // ---- U: alpha = w^T y / p^T v, x += alpha p, w -= alpha v, hx += alpha v (pcg_update_kernel)
  const double pv = block_fixed_sum_cg(a.pv_part, a.nbr, &slot);
  const double wy = block_fixed_sum_cg(a.wy_part, a.nb5, &slot);
  const bool bad = !(pv > 0.0) || !isfinite(pv);
  if (threadIdx.x == 0) slot = wy / pv;   // one division (the FP64 pipe is narrow), shared
  __syncthreads();
  const double alpha = slot;
  if (!bad && b < a.nb3) {
    const C al = (C)alpha;
    const int64_t j0 = (int64_t)b * a.chunk;
    const int64_t j1 = min(d, j0 + a.chunk);
    double lw2 = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += kVecThreads) {
      const C vj = __ldcg(a.v + j);
      a.x[j] = fma(al, a.p[j], a.x[j]);
      const C wj = fma(-al, vj, a.w[j]);
      if (a.hx) a.hx[j] = fma(al, vj, a.hx[j]);
      a.w[j] = wj;
      wch[j - j0] = wj;
      lw2 += (double)wj * (double)wj;
    }
    const double tw2 = block_sum_t0<kVecThreads>(lw2, sh);
    if (threadIdx.x == 0) a.part_w2[b] = tw2;
  }
  if (!grid_barrier(&st->bar_count, &st->bar_gen, nblk)) return fail();
  // ---- S: ||w||^2, stop test, iteration count (pcg_scalar_body; every block takes the same
  // decision, block 0 records it).  U^T w and g = c o U^T w follow only if PCG goes on: the
  // iteration that ends the loop needs no P^{-1} w (the separate kernels form it regardless;
  // the values they use are the same).
  const double w2 = block_fixed_sum_cg(a.part_w2, a.nb3, &slot);
  const bool stepped = !bad && isfinite(w2);
  int iters = iters0, done = 0, status = 0;
  if (!stepped) {
    // first iteration: H + rho I not positive definite on p; later: the rounding floor
    status = iters0 == 0 ? NYS_EBREAKDOWN : NYS_ENOCONV;
    done = 1;
  } else {
    iters += 1;
    if (fixed >= 0) {
      if (iters >= fixed) done = 1;
    } else if (!(w2 > thresh2)) {
      done = 1;
    } else if (iters >= maxit) {
      done = 1;
      status = NYS_ENOCONV;
    }
  }
  if (b == 0 && threadIdx.x == 0) {
    if (stepped) {
      st->wy = wy;
      st->iters = iters;
      st->w2 = w2;
    }
    if (status) st->status = status;
    st->done = done;
    cudaGraphSetConditional(a.cond, done ? 0u : 1u);
  }
  if (!done) {
    // U^T w partials over this block's chunk of the new w, still in shared memory (every
    // block that stepped has !bad here)
    if (b < a.nb3) {
      const int64_t j0 = (int64_t)b * a.chunk;
      const int64_t j1 = min(d, j0 + a.chunk);
      utw_partials<C>(wch, (int)(j1 - j0), a.U, d, j0, s, a.part_g + (int64_t)b * s);
    }
    if (!grid_barrier(&st->bar_count, &st->bar_gen, nblk)) return fail();
    for (int i = threadIdx.x; i < s; i += kVecThreads) {
      const double g = sum_strided_fixed<true>(a.part_g, a.nb3, s, i, 0.0);
      const C gi = (C)((double)a.cvec[i] * g);
      wch[i] = gi;
      if (b == 0) a.gs[i] = gi;
    }
    __syncthreads();
    // ---- T: y = w + U g, partials of w^T y (pcg_tail_kernel)
    if (b < a.nb5) {
      double lwy = 0.0;
      for (int64_t j = b * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)a.nb5 * kVecThreads) {
        const C wj = __ldcg(a.w + j);
        const C acc = urow_dot(a.U, d, j, s, wch, wj);
        a.y[j] = acc;
        lwy += (double)wj * (double)acc;
      }
      const double t = block_sum_t0<kVecThreads>(lwy, sh);
      if (threadIdx.x == 0) a.wy_part[b] = t;
    }
    if (!grid_barrier(&st->bar_count, &st->bar_gen, nblk)) return fail();
    // ---- B: beta = (w^T y)_new / (w^T y)_old, p = y + beta p
    const double wy_new = block_fixed_sum_cg(a.wy_part, a.nb5, &slot);
    if (threadIdx.x == 0) slot = wy_new / wy;
    __syncthreads();
    const C bc = (C)slot;
    for (int64_t j = b * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)nblk * kVecThreads)
      a.p[j] = fma(bc, a.p[j], __ldcg(a.y + j));
    return;
  }
  if (!a.zu) return;
  // ---- Z: prox / dual step with the final x and the scalars of the ADMM iteration
  // (admm_zu_g_kernel; x was written by other blocks above: read through L2)
  if (b < a.nbz) {
    double* zt = a.ztrace ? a.ztrace + (int64_t)a.ctl->k * d : nullptr;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    for (int64_t j = b * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)a.nbz * kVecThreads) {
      const double xj = (double)__ldcg(a.x + j);
      const double zo = a.z[j];
      const double vj = xj + a.u[j];
      const double mag = fabs(vj) - a.kappa;
      const double zj = mag > 0.0 ? copysign(mag, vj) : 0.0;
      const double uj = a.u[j] + xj - zj;
      a.xd[j] = xj;
      a.z[j] = zj;
      a.u[j] = uj;
      if (zt) zt[j] = zj;
      a0 += (xj - zj) * (xj - zj);
      a1 += (zj - zo) * (zj - zo);
      a2 += xj * xj;
      a3 += zj * zj;
      a4 += uj * uj;
    }
    double a5[5] = {a0, a1, a2, a3, a4};
    block_sum5(a5);
    if (threadIdx.x == 0) {
      double* o = a.part5 + (int64_t)b * 5;
#pragma unroll
      for (int t = 0; t < 5; ++t) o[t] = a5[t];
    }
  }
  if (!grid_barrier(&st->bar_count, &st->bar_gen, nblk)) return fail();
  if (b == 0 && threadIdx.x < 32)
    admm_scalar_g_body(a.nbz, a.part5, a.rho_admm, a.K, a.eps_abs, a.eps_rel, a.rp, a.rd, a.pcg_it, st, a.ctl, 0, 2,
                       a.h_admm);
}

struct HeadArgs {
  int64_t d;
  int chunk, nb3, nbz, nb5, s;
  const double* q;
  double *x, *z, *u;
  double rho, kappa;
  double *part_w2, *part_r2, *part_g, *wy_part, *part5;
  AdmmCtl* ctl;
  PcgState* st;
  double tol, tol_floor;
  int tol_mode, maxit, hx_refresh, K;
  const int* fixed_dev;
  const double* tolpow;   // (k + 1)^(-tol) for k < K (NYS_TOL_RNORM_POW), else null
  double eps_abs, eps_rel;
  double *ztrace, *rp_trace, *rd_trace;
  int* pcg_it_trace;
  int* dstat;
  cudaGraphConditionalHandle h_admm, h_pcg, h_zu, h_hx;
  int has_zu;   // 0: the PCG post kernel runs the prox / dual step, there is no IF (h_zu) node
};

template <typename C>
__global__ void __launch_bounds__(kVecThreads) admm_head_kernel(HeadArgs a, const C* __restrict__ xc,
                                                                const C* __restrict__ hx, C* __restrict__ w,
                                                                C* __restrict__ rc, C* __restrict__ y,
                                                                C* __restrict__ p, const C* __restrict__ U,
                                                                const C* __restrict__ cvec, C* __restrict__ gs) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* wch = reinterpret_cast<C*>(sm_raw);   // chunk of w (U^T w), then g (y = w + U g)
  __shared__ double sh[kVecThreads / 32];
  __shared__ double slot;
  __shared__ double slot2[2];
  __shared__ int s_go;
  __shared__ double s_tolk;
  __shared__ int s_tabs;
  const int b = blockIdx.x;
  const unsigned nblk = gridDim.x;
  const int64_t d = a.d;
  const int s = a.s;
  AdmmCtl* ctl = a.ctl;
  int k = ctl->k;
  double eps_next = ctl->eps_next;
  const int refreshed = ctl->hx_pending;   // the recompute of iteration k ran just before this launch
  auto fail = [&]() {
    if (b == 0 && threadIdx.x == 0) {
      atomicExch(a.dstat, (int)NYS_ETIMEOUT);
      cudaGraphSetConditional(a.h_admm, 0u);
      cudaGraphSetConditional(a.h_pcg, 0u);
      if (a.has_zu) cudaGraphSetConditional(a.h_zu, 0u);
      cudaGraphSetConditional(a.h_hx, 0u);
    }
  };
  bool first = true;
  for (;;) {
    // ---- (H + rho I) x due for a recompute at iteration k: request it and return
    if (!iter_hx_skip(0, k, a.hx_refresh) && !(first && refreshed)) {
      if (b == 0 && threadIdx.x == 0) {
        ctl->hx_pending = 1;
        ctl->nodes += 1;
        cudaGraphSetConditional(a.h_hx, 1u);
        cudaGraphSetConditional(a.h_pcg, 0u);
        if (a.has_zu) cudaGraphSetConditional(a.h_zu, 0u);
      }
      return;
    }
    // one thread evaluates the schedule (a pow on the narrow FP64 pipe), the block shares it
    if (threadIdx.x == 0) {
      double t;
      int ab;
      iter_tol_tab(a.tol_mode, a.tol, a.tol_floor, k, eps_next, a.tolpow, &t, &ab);
      s_tolk = t;
      s_tabs = ab;
    }
    __syncthreads();
    const double tolk = s_tolk;
    const int tol_abs = s_tabs;
    // ---- 1. right-hand side, warm-start residual, ||w||^2, ||r||^2, U^T w partials
    if (b < a.nb3) {
      const int64_t j0 = (int64_t)b * a.chunk;
      const int64_t j1 = min(d, j0 + a.chunk);
      double lw2 = 0.0, lr2 = 0.0;
      for (int64_t j = j0 + threadIdx.x; j < j1; j += kVecThreads) {
        const C rj = (C)fma(a.rho, __ldcg(a.z + j) - __ldcg(a.u + j), a.q[j]);
        rc[j] = rj;
        const C wj = rj - hx[j];
        lr2 += (double)rj * (double)rj;
        w[j] = wj;
        wch[j - j0] = wj;
        lw2 += (double)wj * (double)wj;
      }
      const double tw2 = block_sum_t0<kVecThreads>(lw2, sh);
      const double tr2 = block_sum_t0<kVecThreads>(lr2, sh);
      if (threadIdx.x == 0) {
        a.part_w2[b] = tw2;
        a.part_r2[b] = tr2;
      }
    }
    if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, nblk)) return fail();
    if (first && refreshed && b == 0 && threadIdx.x == 0) ctl->hx_pending = 0;
    first = false;
    // ---- 2. stop decision of the warm start (every block, the order of pcg_scalar_body)
    double w2, r2;
    block_fixed_sum2_cg(a.part_w2, a.part_r2, a.nb3, &w2, &r2, slot2);
    const double thresh2 = tol_abs ? tolk * tolk : tolk * tolk * r2;
    const int fixed = a.fixed_dev ? a.fixed_dev[k] : -1;
    const bool nostep = fixed >= 0 ? fixed == 0 : !(w2 > thresh2);
    if (!nostep) {
      // ---- 3b. P^{-1} w and the PCG state; the PCG WHILE node takes over.  U^T w partials
      // over the blocks' chunks of w (the mapping and order of pcg_update_kernel's init step)
      if (b < a.nb3) {
        const int64_t j0 = (int64_t)b * a.chunk;
        const int64_t j1 = min(d, j0 + a.chunk);
        for (int64_t j = j0 + threadIdx.x; j < j1; j += kVecThreads) wch[j - j0] = __ldcg(w + j);
        __syncthreads();
        utw_partials<C>(wch, (int)(j1 - j0), U, d, j0, s, a.part_g + (int64_t)b * s);
      }
      if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, nblk)) return fail();
      for (int i = threadIdx.x; i < s; i += kVecThreads) {
        const double gsum = sum_strided_fixed<true>(a.part_g, a.nb3, s, i, 0.0);
        const C gi = (C)((double)cvec[i] * gsum);
        wch[i] = gi;
        if (b == 0) gs[i] = gi;
      }
      __syncthreads();
      if (b < a.nb5) {
        double lwy = 0.0;
        for (int64_t j = b * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)a.nb5 * kVecThreads) {
          const C wj = __ldcg(w + j);
          const C acc = urow_dot(U, d, j, s, wch, wj);
          y[j] = acc;
          p[j] = acc;
          lwy += (double)wj * (double)acc;
        }
        const double t = block_sum_t0<kVecThreads>(lwy, sh);
        if (threadIdx.x == 0) a.wy_part[b] = t;
      }
      if (b == 0 && threadIdx.x == 0) {
        PcgState* st = a.st;
        st->wy = 0.0;
        st->w2 = w2;
        st->r2 = r2;
        st->thresh2 = thresh2;
        st->tol = tolk;
        st->tol_abs = tol_abs;
        st->iters = 0;
        st->done = 0;
        st->status = 0;
        st->maxit = a.maxit;
        st->fixed = fixed;
        st->ticket[0] = 0u;
        st->ticket[1] = 0u;
        ctl->nodes += 1;
        cudaGraphSetConditional(a.h_hx, 0u);
        cudaGraphSetConditional(a.h_pcg, 1u);
        if (a.has_zu) cudaGraphSetConditional(a.h_zu, 1u);
      }
      return;
    }
    // ---- 3a. prox / dual step with x unchanged, residual partials
    if (b < a.nbz) {
      double* zt = a.ztrace ? a.ztrace + (int64_t)k * d : nullptr;
      double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
      for (int64_t j = b * (int64_t)kVecThreads + threadIdx.x; j < d; j += (int64_t)a.nbz * kVecThreads) {
        const double xj = (double)xc[j];
        const double zo = __ldcg(a.z + j);
        const double uo = __ldcg(a.u + j);
        const double vj = xj + uo;
        const double mag = fabs(vj) - a.kappa;
        const double zj = mag > 0.0 ? copysign(mag, vj) : 0.0;
        const double uj = uo + xj - zj;
        a.x[j] = xj;
        a.z[j] = zj;
        a.u[j] = uj;
        if (zt) zt[j] = zj;
        a0 += (xj - zj) * (xj - zj);
        a1 += (zj - zo) * (zj - zo);
        a2 += xj * xj;
        a3 += zj * zj;
        a4 += uj * uj;
      }
      double a5[5] = {a0, a1, a2, a3, a4};
      block_sum5(a5);
      if (threadIdx.x == 0) {
        double* o = a.part5 + (int64_t)b * 5;
#pragma unroll
        for (int t = 0; t < 5; ++t) o[t] = a5[t];
      }
    }
    if (!grid_barrier(&ctl->bar_count, &ctl->bar_gen, nblk)) return fail();
    // ---- 4. scalars of the iteration (every block; block 0 records them)
    if (threadIdx.x < 32) {
      double sums[5];
      sum_part5(a.nbz, a.part5, sums);
      if (threadIdx.x == 0) {
        const double rp = sqrt(sums[0]);
        const double rd = a.rho * sqrt(sums[1]);
        eps_next = sqrt(rp * rd);
        int stop = 0;
        if (a.eps_rel > 0.0) {
          const double tp = a.eps_abs + a.eps_rel * fmax(sqrt(sums[2]), sqrt(sums[3]));
          const double td = a.eps_abs + a.eps_rel * a.rho * sqrt(sums[4]);
          if (rp <= tp && rd <= td) stop = 1;
        }
        if (b == 0) {
          a.rp_trace[k] = rp;
          a.rd_trace[k] = rd;
          a.pcg_it_trace[k] = 0;
          ctl->eps_next = eps_next;
          ctl->stop = stop;
          ctl->k = k + 1;
        }
        s_go = (k + 1 < a.K && !stop) ? 1 : 0;
        slot = eps_next;
      }
    }
    __syncthreads();
    eps_next = slot;
    const int go = s_go;
    __syncthreads();
    k += 1;
    if (!go) {
      if (b == 0 && threadIdx.x == 0) {
        ctl->nodes += 1;
        cudaGraphSetConditional(a.h_admm, 0u);
        cudaGraphSetConditional(a.h_hx, 0u);
        cudaGraphSetConditional(a.h_pcg, 0u);
        if (a.has_zu) cudaGraphSetConditional(a.h_zu, 0u);
      }
      return;
    }
    // the partials of steps 1 and 3a are rewritten only after the next barrier, which every
    // block reaches after its reads above
  }
}

}  // namespace

namespace {
// Learned warm start: features f = [U^T r / ||r||, log10 rho, k / 100, ln ||r||].
// Block i < s: (U^T r)_i; block s: ||r||^2 (double accumulation, fixed order).
template <typename C>
__global__ void __launch_bounds__(kVecThreads) ws_proj_kernel(int64_t d, int s, const C* __restrict__ U,
                                                              const C* __restrict__ v, const C* __restrict__ vsub,
                                                              double* out) {
  __shared__ double sh[kVecThreads / 32];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < d; j += kVecThreads) {
    const double vj = vsub ? (double)v[j] - (double)vsub[j] : (double)v[j];
    acc += (i < s ? (double)U[(int64_t)i * d + j] : vj) * vj;
  }
  acc = block_sum_t0<kVecThreads>(acc, sh);
  if (threadIdx.x == 0) out[i] = acc;
}

__global__ void ws_features_kernel(int s, const double* proj, double rho, const AdmmCtl* ctl, float* feat,
                                   double* rnorm) {
  const double rn = sqrt(proj[s]);
  const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) feat[i] = (float)(proj[i] * inv);
  if (threadIdx.x == 0) {
    feat[s] = (float)log10(rho);
    feat[s + 1] = (float)(ctl->k / 100.0);
    feat[s + 2] = (float)(rn > 0.0 ? log(rn) : 0.0);
    *rnorm = rn;
  }
}

// The model predicts the subspace coordinates of the solution, U^T x ~ m(f) ||r|| / rho;
// x0 = x_prev + U c with c = m(f) ||r|| / rho - U^T x_prev (uxp).  The warm start
// changed, so (H + rho I) x0 is recomputed.
template <typename C>
__global__ void ws_apply_kernel(int64_t d, int s, const C* __restrict__ U, const float* __restrict__ c,
                                const double* __restrict__ uxp, const double* rnorm, double rho, C* __restrict__ xc,
                                C* __restrict__ xprev, AdmmCtl* ctl, cudaGraphConditionalHandle hx_cond,
                                long long hx_nodes) {
  const double scale = *rnorm / rho;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < s; ++i) acc += (double)U[(int64_t)i * d + j] * ((double)c[i] * scale - uxp[i]);
    const C x0 = xc[j];
    if (xprev) xprev[j] = x0;
    xc[j] = (C)((double)x0 + acc);
  }
  // x moved off x_prev: the tracked (H + rho I) x is stale, open the recompute node
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (ctl->hx_skip) ctl->nodes += hx_nodes;
    ctl->hx_skip = 0;
    cudaGraphSetConditional(hx_cond, 1u);
  }
}

template <typename C>
__global__ void ws_copy_kernel(int64_t d, const C* __restrict__ x, C* __restrict__ y) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x)
    y[j] = x[j];
}

// record row k = [f (s + 3), U^T x_new * rho / ||r|| (s)]
__global__ void ws_record_kernel(int s, const float* feat, const double* proj, const double* rnorm, double rho,
                                 const AdmmCtl* ctl, float* rec) {
  float* row = rec + (int64_t)ctl->k * (2 * s + 3);
  const double sc = *rnorm > 0.0 ? rho / *rnorm : 0.0;
  for (int i = threadIdx.x; i < s + 3; i += blockDim.x) row[i] = feat[i];
  for (int i = threadIdx.x; i < s; i += blockDim.x) row[s + 3 + i] = (float)(proj[i] * sc);
}
}  // namespace

// Adds one instance's device-side loop (an outer conditional WHILE over ADMM iterations
// containing the PCG WHILE) to `graph` as an independent branch.  Buffers come from
// `pool`, which must outlive the graph's execution; state is initialised on `stream`.
template <typename C>
nys_status admm_graph_add(cudaGraph_t graph, const GraphLoopArgs& g, cudaStream_t stream, Pool& pool,
                          GraphInstance* inst) {
  const int64_t d = g.pb.A->d;
  const int s = g.P.s;
  const C* U = reinterpret_cast<const C*>(g.P.U);
  const C* cvec = reinterpret_cast<const C*>(g.P.c);
  const int chunk = upd_chunk(d);
  const int nb3 = (int)((d + chunk - 1) / chunk);
  const int nbr = reduce_blocks(d);
  const int nb5 = nbr;
  const int nbz = admm_blocks(d);
  const int K = g.K;
  C* w = pool.alloc<C>(d);
  C* y = pool.alloc<C>(d);
  C* p = pool.alloc<C>(d);
  C* v = pool.alloc<C>(d);
  C* gs = pool.alloc<C>(std::max(1, s));
  double* part_w2 = pool.alloc<double>(nb3);
  double* part_r2 = pool.alloc<double>(nb3);
  double* part_g = pool.alloc<double>((size_t)nb3 * std::max(1, s));
  double* pv_part = pool.alloc<double>(nbr);
  double* wy_part = pool.alloc<double>(nb5);
  void* apart = pool.alloc<unsigned char>(apass_partial_bytes(g.pb.A, g.pb.plan));
  void* apart_ref = g.Aref ? pool.alloc<unsigned char>(apass_partial_bytes(g.Aref, g.plan_ref)) : nullptr;
  PcgState* st = pool.alloc<PcgState>(1);
  AdmmCtl* ctl = pool.alloc<AdmmCtl>(1);
  int* dstat = pool.alloc<int>(1);
  double* part5 = pool.alloc<double>((size_t)nbz * 5);
  int* fixed_dev = g.fixed_host ? pool.alloc<int>(K) : nullptr;
  double* tolpow = g.tol_mode == NYS_TOL_RNORM_POW && K > 0 ? pool.alloc<double>(K) : nullptr;
  if (!pool.ok()) return NYS_ENOMEM;
  C* xc = reinterpret_cast<C*>(g.xc);
  C* rc = reinterpret_cast<C*>(g.rc);
  C* hx = reinterpret_cast<C*>(g.hx);
  cudaError_t e = cudaSuccess;
#define G_OK(x)                                                                              \
  do {                                                                                       \
    e = (x);                                                                                 \
    if (e != cudaSuccess) {                                                                  \
      if (std::getenv("NYS_TRACE"))                                                          \
        std::fprintf(stderr, "[nys] graph build: %s at pcg.cu:%d\n", cudaGetErrorString(e), __LINE__); \
      (void)cudaGetLastError(); /* a failed build leaves no error behind for later launches */ \
      return NYS_ECUDA;                                                                      \
    }                                                                                        \
  } while (0)
  G_OK(cudaMemsetAsync(ctl, 0, sizeof(AdmmCtl), stream));
  G_OK(cudaMemsetAsync(st, 0, sizeof(PcgState), stream));   // the post kernel's barrier words start at 0
  G_OK(cudaMemsetAsync(dstat, 0, sizeof(int), stream));
  G_OK(cudaMemsetAsync(hx, 0, d * sizeof(C), stream));
  if (fixed_dev) G_OK(cudaMemcpyAsync(fixed_dev, g.fixed_host, K * sizeof(int), cudaMemcpyHostToDevice, stream));
  if (tolpow) {
    count_launch();
    tolpow_kernel<<<(K + 255) / 256, 256, 0, stream>>>(tolpow, K, g.tol);
    G_OK(cudaGetLastError());
  }
  G_OK(apass_prepare(g.pb.A, g.pb.plan));
  if (g.Aref) G_OK(apass_prepare(g.Aref, g.plan_ref));

  // a private stream to capture on (a legacy default stream cannot be captured)
  cudaStream_t cap = capture_stream();
  if (!cap) return NYS_ECUDA;
  cudaGraphConditionalHandle h_admm, h_pcg;
  G_OK(cudaGraphConditionalHandleCreate(&h_admm, graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h_admm;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t n_admm;
  G_OK(cudaGraphAddNode(&n_admm, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];

  ApassArgs aa;
  aa.A = g.pb.A->data;
  aa.n = g.pb.A->n;
  aa.d = d;
  aa.ld = g.pb.A->ld;
  aa.dtype = g.pb.A->dtype;
  aa.col_scale = g.pb.A->col_scale;
  aa.D = g.pb.D;
  aa.b = nullptr;
  aa.D_out = nullptr;
  aa.t_out = nullptr;
  aa.mode = g.pb.D ? MODE_DIAG : MODE_ID;

  // One PCG iteration after its A-pass as one cooperative launch (pcg_post_kernel) instead of
  // the reduce, update and tail kernels, for a single instance (its grid barriers want the
  // grid co-resident; concurrent graph branches keep the separate kernels).  NYS_PCG_POST=0
  // selects the separate kernels.
  const int nbp = std::max(std::max(nbr, nb3), std::max(nb5, nbz));
  const size_t sm_post = (size_t)std::max(chunk, std::max(1, s)) * sizeof(C);
  bool use_post = g.allow_nostep && nbz <= kPart5Max;
  {
    const char* pe = std::getenv("NYS_PCG_POST");
    if (pe && std::atoi(pe) == 0) use_post = false;
    if (use_post) {
      int per_sm = 0, coop = 0;
      G_OK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, current_device()));
      G_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_post_kernel<C>, kVecThreads, sm_post));
      use_post = coop && (int64_t)per_sm * sm_count() >= nbp;
    }
  }
  PostArgs<C> pa = {};
  pa.d = d;
  pa.chunk = chunk;
  pa.nbr = nbr;
  pa.nb3 = nb3;
  pa.nb5 = nb5;
  pa.nbz = nbz;
  pa.partial = reinterpret_cast<const C*>(apart);
  pa.G = g.pb.plan.grid;
  pa.dpad = g.pb.plan.dpad;
  pa.rho = (C)(g.rho + g.mu);
  pa.cscale = g.pb.A->dtype == NYS_FP8E4M3 ? g.pb.A->col_scale : nullptr;
  pa.p = p;
  pa.v = v;
  pa.x = xc;
  pa.w = w;
  pa.hx = hx;
  pa.y = y;
  pa.U = U;
  pa.s = s;
  pa.cvec = cvec;
  pa.gs = gs;
  pa.pv_part = pv_part;
  pa.wy_part = wy_part;
  pa.part_w2 = part_w2;
  pa.part_g = part_g;
  pa.st = st;
  pa.xd = g.x;
  pa.z = g.z;
  pa.u = g.u;
  pa.ztrace = g.ztrace;
  pa.part5 = part5;
  pa.rp = g.rp;
  pa.rd = g.rd;
  pa.pcg_it = g.pcg_it;
  pa.kappa = g.gamma / g.rho;
  pa.rho_admm = g.rho;
  pa.eps_abs = g.eps_abs;
  pa.eps_rel = g.eps_rel;
  pa.K = K;
  pa.ctl = ctl;
  pa.dstat = dstat;
  auto launch_post = [&](cudaGraphConditionalHandle hc, int zu, cudaGraphConditionalHandle ha) {
    PostArgs<C> q = pa;
    q.cond = hc;
    q.zu = zu;
    q.h_admm = ha;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nbp);
    cfg.blockDim = dim3(kVecThreads);
    cfg.dynamicSmemBytes = sm_post;
    cfg.stream = cap;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pcg_post_kernel<C>, q);
  };

  // Fast body (tracked warm start, no refined step or warm-start model, a single instance):
  //   admm_head_kernel (cooperative) -> IF (h_hx) [ (H + rho I) x recompute ] ->
  //   WHILE (h_pcg) [ A-pass, reduce, update, P^{-1} tail ] -> IF (h_zu) [ prox / dual + scalars ]
  // The head kernel runs the iterations that need no PCG step itself and prepares the PCG
  // state of the others; when the recompute is due it sets only h_hx and returns, and the
  // next pass of the body continues that iteration.  It sets all three conditionals on every
  // exit (their handles have no default value).  NYS_ADMM_NOSTEP=0 selects the general body.
  {
    const bool use_model = (g.warm || g.warm_record) && s > 0;
    const char* env = std::getenv("NYS_ADMM_NOSTEP");
    bool fast = !g.Aref && !use_model && g.hx_refresh > 0 && g.allow_nostep && !(env && std::atoi(env) == 0);
    const int nbf = std::max(std::max(nb3, nbz), nbr);
    const size_t sm_head = (size_t)std::max(chunk, std::max(1, s)) * sizeof(C);
    if (fast) {
      int per_sm = 0, coop = 0;
      G_OK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, current_device()));
      G_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, admm_head_kernel<C>, kVecThreads, sm_head));
      fast = coop && (int64_t)per_sm * sm_count() >= nbf && nbz <= kPart5Max;
    }
    if (fast) {
      cudaGraphConditionalHandle h_hx, h_zu = 0;
      G_OK(cudaGraphConditionalHandleCreate(&h_hx, body, 0u, 0u));
      G_OK(cudaGraphConditionalHandleCreate(&h_pcg, body, 0u, 0u));
      // a handle must belong to a conditional node: h_zu only with the IF (h_zu) node
      if (!use_post) G_OK(cudaGraphConditionalHandleCreate(&h_zu, body, 0u, 0u));
      auto add_cond = [&](cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                          const std::vector<cudaGraphNode_t>& deps, cudaGraphNode_t* node, cudaGraph_t* child) {
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = type;
        np.conditional.size = 1;
        const cudaError_t ce = cudaGraphAddNode(node, body, deps.data(), nullptr, deps.size(), &np);
        *child = np.conditional.phGraph_out[0];
        return ce;
      };
      // head kernel first: it sets every conditional of the body (the handles carry no
      // default, so no conditional node may be evaluated before the kernel has run)
      count_launch_suspend(true);
      G_OK(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      HeadArgs ha;
      ha.d = d;
      ha.chunk = chunk;
      ha.nb3 = nb3;
      ha.nbz = nbz;
      ha.nb5 = nb5;
      ha.s = s;
      ha.q = g.q;
      ha.x = g.x;
      ha.z = g.z;
      ha.u = g.u;
      ha.rho = g.rho;
      ha.kappa = g.gamma / g.rho;
      ha.part_w2 = part_w2;
      ha.part_r2 = part_r2;
      ha.part_g = part_g;
      ha.wy_part = wy_part;
      ha.part5 = part5;
      ha.ctl = ctl;
      ha.st = st;
      ha.tol = g.tol;
      ha.tol_floor = g.tol_floor;
      ha.tol_mode = g.tol_mode;
      ha.maxit = g.maxit;
      ha.hx_refresh = g.hx_refresh;
      ha.K = K;
      ha.fixed_dev = fixed_dev;
      ha.tolpow = tolpow;
      ha.eps_abs = g.eps_abs;
      ha.eps_rel = g.eps_rel;
      ha.ztrace = g.ztrace;
      ha.rp_trace = g.rp;
      ha.rd_trace = g.rd;
      ha.pcg_it_trace = g.pcg_it;
      ha.dstat = dstat;
      ha.h_admm = h_admm;
      ha.h_pcg = h_pcg;
      ha.h_zu = h_zu;
      ha.has_zu = use_post ? 0 : 1;
      ha.h_hx = h_hx;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)nbf);
      cfg.blockDim = dim3(kVecThreads);
      cfg.dynamicSmemBytes = sm_head;
      cfg.stream = cap;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      G_OK(cudaLaunchKernelEx(&cfg, admm_head_kernel<C>, ha, (const C*)xc, (const C*)hx, w, rc, y, p, U, cvec, gs));
      cudaStreamCaptureStatus cst0;
      const cudaGraphNode_t* deps0 = nullptr;
      size_t ndeps0 = 0;
      G_OK(cudaStreamGetCaptureInfo(cap, &cst0, nullptr, nullptr, &deps0, nullptr, &ndeps0));
      std::vector<cudaGraphNode_t> leaf0(deps0, deps0 + ndeps0);
      G_OK(cudaStreamEndCapture(cap, &body));
      // IF (h_hx): (H + rho I) x with one pass over A, when the head kernel asked for it
      cudaGraphNode_t n_hx;
      cudaGraph_t hbody;
      G_OK(add_cond(h_hx, cudaGraphCondTypeIf, leaf0, &n_hx, &hbody));
      G_OK(cudaStreamBeginCaptureToGraph(cap, hbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      aa.p = xc;
      aa.skip = nullptr;
      G_OK(apass_run(aa, g.pb.plan, apart, nullptr, dstat, cap, true));
      G_OK(apass_reduce(aa, g.pb.plan, apart, g.rho + g.mu, hx, nullptr, 0, cap));
      G_OK(cudaStreamEndCapture(cap, &hbody));
      // WHILE (h_pcg): PCG iterations
      cudaGraphNode_t n_pcg;
      cudaGraph_t pbody;
      G_OK(add_cond(h_pcg, cudaGraphCondTypeWhile, {n_hx}, &n_pcg, &pbody));
      G_OK(cudaStreamBeginCaptureToGraph(cap, pbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      aa.p = p;
      aa.skip = &st->done;
      G_OK(apass_run(aa, g.pb.plan, apart, nullptr, dstat, cap, true));
      if (use_post) {
        // the iteration that ends the PCG loop runs the prox / dual step itself: no IF (h_zu)
        G_OK(launch_post(h_pcg, 1, h_admm));
        G_OK(cudaStreamEndCapture(cap, &pbody));
      } else {
        G_OK(apass_reduce(aa, g.pb.plan, apart, g.rho + g.mu, v, pv_part, nbr, cap));
        pcg_update_kernel<C><<<nb3, kVecThreads, (size_t)chunk * sizeof(C), cap>>>(
            0, d, chunk, xc, w, rc, v, p, U, s, pv_part, nbr, wy_part, nb5, part_w2, part_r2, part_g, st, hx, cvec, gs,
            h_pcg, 1, nullptr, nullptr, nullptr, 0.0, (C*)nullptr);
        pcg_tail_kernel<C><<<nb5, kVecThreads, (size_t)std::max(1, s) * sizeof(C), cap>>>(d, w, y, U, s, gs, wy_part,
                                                                                         st, 0, p);
        G_OK(cudaStreamEndCapture(cap, &pbody));
        // IF (h_zu): prox / dual step of an iteration that took PCG steps
        cudaGraphNode_t n_zu;
        cudaGraph_t zbody;
        G_OK(add_cond(h_zu, cudaGraphCondTypeIf, {n_pcg}, &n_zu, &zbody));
        G_OK(cudaStreamBeginCaptureToGraph(cap, zbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        admm_zu_g_kernel<C><<<nbz, kVecThreads, 0, cap>>>(d, xc, 0, g.x, g.z, g.u, g.gamma / g.rho, g.ztrace, ctl,
                                                          part5, g.rho, K, g.eps_abs, g.eps_rel, g.rp, g.rd, g.pcg_it,
                                                          st, 1, 4, h_admm);
        G_OK(cudaStreamEndCapture(cap, &zbody));
      }
      count_launch_suspend(false);
      G_OK(cudaGetLastError());
      inst->ctl = ctl;
      inst->dstat = dstat;
      return NYS_OK;
    }
  }
  G_OK(cudaGraphConditionalHandleCreate(&h_pcg, body, 0u, 0u));
  cudaGraphConditionalHandle h_hx;
  G_OK(cudaGraphConditionalHandleCreate(&h_hx, body, 0u, 0u));

  const size_t sm_upd = (size_t)chunk * sizeof(C);
  const size_t sm_tail = (size_t)std::max(1, s) * sizeof(C);
  const int refine = g.Aref ? 1 : 0;
  long long seg_nodes = 0, body_nodes = 0;

  // ---- segment 1: begin, (exact residual pass), right-hand side, PCG init
  count_launch_suspend(true);
  G_OK(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  admm_begin_kernel<<<1, 1, 0, cap>>>(ctl, st, g.tol, g.tol_floor, g.tol_mode, g.maxit, fixed_dev, g.hx_refresh, refine, h_hx,
                                      2);
  ++seg_nodes;
  if (refine) {
    ApassArgs ar;
    ar.A = g.Aref->data;
    ar.n = g.Aref->n;
    ar.d = d;
    ar.ld = g.Aref->ld;
    ar.dtype = g.Aref->dtype;
    ar.col_scale = g.Aref->col_scale;
    ar.p = g.x;
    ar.D = nullptr;
    ar.b = g.b;
    ar.D_out = nullptr;
    ar.t_out = nullptr;
    ar.mode = MODE_RESID;
    G_OK(apass_run(ar, g.plan_ref, apart_ref, nullptr, dstat, cap, true));
    ApassArgs ar2 = ar;
    ar2.p = nullptr;
    G_OK(apass_reduce(ar2, g.plan_ref, apart_ref, 0.0, g.yres, nullptr, 0, cap));
    seg_nodes += 2;
  }
  const bool use_ws = (g.warm || g.warm_record) && s > 0;
  // without a refined step or a warm-start model the right-hand side is formed by the
  // PCG-init update kernel itself (one launch fewer per iteration)
  const bool fuse_rhs = !refine && !use_ws;
  if (!fuse_rhs) {
    admm_rhs_g_kernel<C><<<nbz, kVecThreads, 0, cap>>>(d, g.q, g.z, g.u, g.rho, g.mu, g.x, g.yres, refine, rc, xc,
                                                        hx);
    ++seg_nodes;
  }
  float* feat = nullptr;
  double* proj = nullptr;
  double* rnorm = nullptr;
  C* xprev = nullptr;
  if (use_ws) {
    feat = pool.alloc<float>(s + 3);
    proj = pool.alloc<double>(s + 1);
    rnorm = pool.alloc<double>(1);
    xprev = pool.alloc<C>(d);
    float* mlp_buf = pool.alloc<float>(4 * 1024 + s);
    if (!pool.ok()) return NYS_ENOMEM;
    ws_proj_kernel<C><<<s + 1, kVecThreads, 0, cap>>>(d, s, U, rc, (const C*)nullptr, proj);
    ws_features_kernel<<<1, 128, 0, cap>>>(s, proj, g.rho, ctl, feat, rnorm);
    seg_nodes += 2;
    if (g.warm) {
      int ni, nh, no;
      mlp_dims(g.warm, &ni, &nh, &no);
      if (ni != s + 3 || no != s || nh > 1024) return NYS_EINVAL;
      float* cout = mlp_buf + 4 * 1024;
      double* uxp = pool.alloc<double>(s);
      if (!pool.ok()) return NYS_ENOMEM;
      ws_proj_kernel<C><<<s, kVecThreads, 0, cap>>>(d, s, U, xc, (const C*)nullptr, uxp);
      G_OK(mlp_forward_dev(g.warm, feat, 1, mlp_buf, mlp_buf + 1024, mlp_buf + 2048, mlp_buf + 3072, cout, cap));
      ws_apply_kernel<C><<<nbz, kVecThreads, 0, cap>>>(d, s, U, cout, uxp, rnorm, g.rho, xc, xprev, ctl, h_hx, 2);
      seg_nodes += 5;
    } else {
      ws_copy_kernel<C><<<nbz, kVecThreads, 0, cap>>>(d, xc, xprev);
      ++seg_nodes;
    }
  }
  // (H + rho I) x recompute: an IF node that admm_begin_kernel opens every hx_refresh
  // iterations (counted there when it runs)
  {
    cudaStreamCaptureStatus cst1;
    const cudaGraphNode_t* deps1 = nullptr;
    size_t ndeps1 = 0;
    G_OK(cudaStreamGetCaptureInfo(cap, &cst1, nullptr, nullptr, &deps1, nullptr, &ndeps1));
    std::vector<cudaGraphNode_t> leaf1(deps1, deps1 + ndeps1);
    G_OK(cudaStreamEndCapture(cap, &body));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_hx;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t n_hx;
    G_OK(cudaGraphAddNode(&n_hx, body, leaf1.data(), nullptr, leaf1.size(), &ip));
    cudaGraph_t hbody = ip.conditional.phGraph_out[0];
    G_OK(cudaStreamBeginCaptureToGraph(cap, hbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    aa.p = xc;
    aa.skip = nullptr;
    G_OK(apass_run(aa, g.pb.plan, apart, nullptr, dstat, cap, true));
    G_OK(apass_reduce(aa, g.pb.plan, apart, g.rho + g.mu, hx, nullptr, 0, cap));
    G_OK(cudaStreamEndCapture(cap, &hbody));
    G_OK(cudaStreamBeginCaptureToGraph(cap, body, &n_hx, nullptr, 1, cudaStreamCaptureModeRelaxed));
  }
  pcg_update_kernel<C><<<nb3, kVecThreads, sm_upd, cap>>>(1, d, chunk, xc, w, rc, hx, p, U, s, pv_part, nbr,
                                                          wy_part, nb5, part_w2, part_r2, part_g, st, (C*)nullptr,
                                                          cvec, gs, h_pcg, 1, fuse_rhs ? g.q : nullptr,
                                                          fuse_rhs ? g.z : nullptr, fuse_rhs ? g.u : nullptr, g.rho, rc);
  pcg_tail_kernel<C><<<nb5, kVecThreads, sm_tail, cap>>>(d, w, y, U, s, gs, wy_part, st, 1, p);
  seg_nodes += 2;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  G_OK(cudaStreamGetCaptureInfo(cap, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> leaf(deps, deps + ndeps);
  G_OK(cudaStreamEndCapture(cap, &body));

  // ---- PCG loop
  cudaGraphNodeParams pp = {};
  pp.type = cudaGraphNodeTypeConditional;
  pp.conditional.handle = h_pcg;
  pp.conditional.type = cudaGraphCondTypeWhile;
  pp.conditional.size = 1;
  cudaGraphNode_t n_pcg;
  G_OK(cudaGraphAddNode(&n_pcg, body, leaf.data(), nullptr, leaf.size(), &pp));
  cudaGraph_t pbody = pp.conditional.phGraph_out[0];
  G_OK(cudaStreamBeginCaptureToGraph(cap, pbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  aa.p = p;
  aa.skip = &st->done;
  G_OK(apass_run(aa, g.pb.plan, apart, nullptr, dstat, cap, true));
  if (use_post) {
    G_OK(launch_post(h_pcg, 0, h_admm));
    body_nodes = 2;
  } else {
    G_OK(apass_reduce(aa, g.pb.plan, apart, g.rho + g.mu, v, pv_part, nbr, cap));
    pcg_update_kernel<C><<<nb3, kVecThreads, sm_upd, cap>>>(0, d, chunk, xc, w, rc, v, p, U, s, pv_part, nbr, wy_part,
                                                            nb5, part_w2, part_r2, part_g, st, hx, cvec, gs, h_pcg, 1,
                                                            nullptr, nullptr, nullptr, 0.0, (C*)nullptr);
    pcg_tail_kernel<C><<<nb5, kVecThreads, sm_tail, cap>>>(d, w, y, U, s, gs, wy_part, st, 0, p);
    body_nodes = 4;
  }
  G_OK(cudaStreamEndCapture(cap, &pbody));

  // ---- segment 2: prox / dual step, residuals, loop condition
  G_OK(cudaStreamBeginCaptureToGraph(cap, body, &n_pcg, nullptr, 1, cudaStreamCaptureModeRelaxed));
  if (use_ws && g.warm_record) {
    ws_proj_kernel<C><<<s, kVecThreads, 0, cap>>>(d, s, U, xc, (const C*)nullptr, proj);
    ws_record_kernel<<<1, 128, 0, cap>>>(s, feat, proj, rnorm, g.rho, ctl, g.warm_record);
    seg_nodes += 2;
  }
  seg_nodes += 1;
  admm_zu_g_kernel<C><<<nbz, kVecThreads, 0, cap>>>(d, xc, refine, g.x, g.z, g.u, g.gamma / g.rho, g.ztrace, ctl,
                                                    part5, g.rho, K, g.eps_abs, g.eps_rel, g.rp, g.rd, g.pcg_it, st,
                                                    seg_nodes, body_nodes, h_admm);
  G_OK(cudaStreamEndCapture(cap, &body));
  count_launch_suspend(false);
  G_OK(cudaGetLastError());

  inst->ctl = ctl;
  inst->dstat = dstat;
  return NYS_OK;
#undef G_OK
}

// One instance: build, instantiate and launch its graph, then read its control block.
template <typename C>
nys_status admm_graph_run(const GraphLoopArgs& g, cudaStream_t stream, GraphLoopResult* res) {
  GraphInstance inst;
  return admm_graph_run_many<C>(&g, 1, stream, &inst, res);
}

template <typename C>
nys_status admm_graph_run_many(const GraphLoopArgs* gs, int count, cudaStream_t stream, GraphInstance* insts,
                               GraphLoopResult* res) {
  Pool pool(stream);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct Cleanup {
    cudaGraph_t* g;
    cudaGraphExec_t* x;
    ~Cleanup() {
      if (*x) cudaGraphExecDestroy(*x);
      if (*g) cudaGraphDestroy(*g);
    }
  } cleanup{&graph, &exec};
  const bool trace = std::getenv("NYS_TRACE") != nullptr;
  auto now = [&]() {
    if (trace) cudaStreamSynchronize(stream);
    return std::chrono::steady_clock::now();
  };
  auto t0 = now();
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return NYS_ECUDA;
  for (int i = 0; i < count; ++i) {
    GraphLoopArgs gi = gs[i];
    if (count > 1) gi.allow_nostep = false;   // branches run concurrently
    const nys_status s = admm_graph_add<C>(graph, gi, stream, pool, &insts[i]);
    if (s != NYS_OK) return s;
  }
  auto t1 = now();
  {
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    if (ie != cudaSuccess) {
      if (trace) std::fprintf(stderr, "[nys] graph instantiate: %s\n", cudaGetErrorString(ie));
      (void)cudaGetLastError();
      return NYS_ECUDA;
    }
  }
  auto t2 = now();
  {
    const cudaError_t le = cudaGraphLaunch(exec, stream);
    if (le != cudaSuccess) {
      if (trace) std::fprintf(stderr, "[nys] graph launch: %s\n", cudaGetErrorString(le));
      return NYS_ECUDA;
    }
  }
  if (trace) {
    auto t3 = now();
    auto ms = [](auto a, auto b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
    std::fprintf(stderr, "[nys] graph build %.3f ms, instantiate %.3f ms, run %.3f ms\n", ms(t0, t1), ms(t1, t2),
                 ms(t2, t3));
  }
  nys_status worst = NYS_OK;
  for (int i = 0; i < count; ++i) {
    AdmmCtl ctl_h;
    int dstat_h = 0;
    cudaError_t re = cudaMemcpyAsync(&ctl_h, insts[i].ctl, sizeof(AdmmCtl), cudaMemcpyDeviceToHost, stream);
    if (re == cudaSuccess) re = cudaMemcpyAsync(&dstat_h, insts[i].dstat, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (re == cudaSuccess) re = cudaStreamSynchronize(stream);
    if (re != cudaSuccess) {
      if (trace) std::fprintf(stderr, "[nys] graph run: %s\n", cudaGetErrorString(re));
      return NYS_ECUDA;
    }
    count_launch_add(ctl_h.nodes);
    res[i].admm_iters = ctl_h.k;
    res[i].breakdown = ctl_h.stop == 2;
    if (dstat_h) worst = (nys_status)dstat_h;
  }
  return worst;
}

template nys_status admm_graph_run<double>(const GraphLoopArgs&, cudaStream_t, GraphLoopResult*);
template nys_status admm_graph_run<float>(const GraphLoopArgs&, cudaStream_t, GraphLoopResult*);
template nys_status admm_graph_run_many<double>(const GraphLoopArgs*, int, cudaStream_t, GraphInstance*,
                                                GraphLoopResult*);
template nys_status admm_graph_run_many<float>(const GraphLoopArgs*, int, cudaStream_t, GraphInstance*,
                                               GraphLoopResult*);

}  // namespace nys
