// The whole device-side lasso / elastic-net NysADMM loop (Alg. 2 with the x-step of
// Eq. ADMMSubProb solved by Alg. Nystrom PCG) as ONE persistent cooperative kernel, for
// FP32-compute storage (FP32, BF16, FP8) whose A-pass takes the warp-specialised form.
//
// Every CTA sits on its own SM for the whole solve and plays two parts:
//   * the A-pass roles of apass_ws.cuh over its slab of rows of A (H-matvecs of the PCG
//     iterations and the periodic (H + rho I) x recompute): the stage ring and its
//     mbarriers carry on from pass to pass;
//   * the d-vector work on its slice of [0, d): right-hand side r = q + rho (z - u), the
//     warm-start residual w = r - (H + rho I) x, P^{-1} w = w + U diag(c) U^T w, the PCG
//     updates of x, w, (H + rho I) x and p, and the prox / dual step of Sec. 2.1.
// Grid-wide quantities (norms, dot products, U^T w, the per-CTA A-pass partials) are
// written per CTA and summed after a grid barrier by every CTA in the same fixed order,
// so all CTAs take the same decisions and the result is bitwise reproducible.
//
// Barriers per ADMM iteration: two when the warm start already meets the PCG tolerance,
// else two plus three per PCG iteration and one per further direction.  The next PCG
// direction p' = y + beta p is formed on the fly by the dot warps of the next pass (each
// CTA needs all of p'), so no barrier waits for p' to be stored.
//
// Arithmetic per element is that of the graph-driven loop (pcg.cu); the slices and hence
// the order of the grid-wide sums differ, so the two agree to rounding, not bit for bit.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "apass_ws.cuh"
#include "solver.cuh"

namespace nys {
namespace {

#define FUSED_CU(expr)                 \
  do {                                 \
    if ((expr) != cudaSuccess) {       \
      cudaGetLastError();              \
      return NYS_ECUDA;                \
    }                                  \
  } while (0)

constexpr int kFusedMaxS = 1024;     // U^T w and g held in shared memory
// Registers per thread: 18 warps x 32 x 112 = 64,512 of the SM's 65,536.  (A launch bound of
// 576 threads lets the compiler use only 96, and the pass's loops then spill once they sit
// inside the solve's loop; the stand-alone pass needs 83.)
constexpr int kFusedRegs = 112;
constexpr int kFusedMaxGrid = 1024;  // per-CTA partial arrays

struct FusedArgs {
  ApassKArgs pa;        // pass arguments (p unused: the pass takes p from its PSrc)
  int64_t d;
  int s;
  const float* U;       // s x d (row i = u_i)
  const float* cvec;    // (lam_s + rho) / (lam_i + rho) - 1
  const double* q;      // A^T b
  double *x, *z, *u;    // ADMM state (FP64)
  float *xc, *hx, *w, *y, *v, *pa_buf, *pb_buf;   // compute-type vectors (p double-buffered)
  float* partial;       // [grid][dpad] A-pass partials
  double* part;         // [grid][kPartW] per-CTA scalar partials
  float* part_g;        // [s][grid] U^T w partials
  unsigned* bar;        // grid barrier counter
  int* status;
  int* k_out;           // ADMM iterations done
  int* stop_out;        // 1 residual stop, 2 PCG breakdown
  double rho, mu, kappa;
  double tol, tol_floor;
  int tol_mode, maxit, hx_refresh, K;
  const int* fixed;     // replayed PCG counts, or null
  double eps_abs, eps_rel;
  double* ztrace;
  double *rp, *rd;
  int* pcg_it;
  long long* passes;    // A-passes run (instrumentation)
};

constexpr int kPartW = 16;  // doubles per CTA in `part`

// PCG tolerance of ADMM iteration k (same cases as the graph-driven loop).
__device__ __forceinline__ void fused_tol(const FusedArgs& a, int k, double eps_next, double* tol, int* tol_abs) {
  if (a.tol_mode == NYS_TOL_SQRT_RPRD && k > 0) {
    *tol = eps_next;
    *tol_abs = 1;
  } else if (a.tol_mode == NYS_TOL_ABS) {
    *tol = a.tol;
    *tol_abs = 1;
  } else {
    const double t = a.tol_mode == NYS_TOL_RNORM_POW ? pow((double)(k + 1), -a.tol) : a.tol;
    *tol = fmax(t, a.tol_floor);
    *tol_abs = 0;
  }
}

// Block-wide fixed-order sums of NV values over the first `nw` warps (the ones holding
// elements of the CTA's slice; the others hold zeros and skip the FP64 shuffles, which run
// on the slow FP64 pipe).  Every thread gets the sums.
template <int NV, int NT>
__device__ __forceinline__ void fused_block_sum(double (&v)[NV], double (*sh)[NT / 32], int nw) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < nw) {
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = warp_sum(v[t]);
  }
  __syncthreads();
  if (lane == 0 && w < nw) {
#pragma unroll
    for (int t = 0; t < NV; ++t) sh[t][w] = v[t];
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += sh[t][i];
    v[t] = s;
  }
  __syncthreads();
}

// Partial slots per CTA in FusedArgs::part.
enum : int { kSlotW2 = 0, kSlotR2 = 1, kSlotWy = 2, kSlotPv = 3, kSlotW2b = 4, kSlotWyb = 5, kSlotZu = 8 };

// Sums of N consecutive slots over the CTAs (CTA c at part[c * kPartW + first + t]) in a
// fixed order: lanes take every 32nd CTA, then a warp butterfly.  Every thread gets them.
template <int N>
__device__ __forceinline__ void grid_sums(const double* part, int nblk, int first, double (&out)[N], double* bc) {
  if (threadIdx.x < 32) {
    double acc[N];
#pragma unroll
    for (int t = 0; t < N; ++t) acc[t] = 0.0;
#pragma unroll 8
    for (int c = threadIdx.x; c < nblk; c += 32) {
#pragma unroll
      for (int t = 0; t < N; ++t) acc[t] += __ldcg(part + (int64_t)c * kPartW + first + t);
    }
#pragma unroll
    for (int t = 0; t < N; ++t) {
      acc[t] = warp_sum(acc[t]);
      if (threadIdx.x == 0) bc[t] = acc[t];
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < N; ++t) out[t] = bc[t];
  __syncthreads();
}

// Partials of U^T w over this CTA's slice: part_g[i * nblk + c] (CTA-contiguous, so that
// the sums over CTAs read coalesced rows).  w is this CTA's own slice.  Eight rows per warp
// at a time keep 8 x (slice / 32) loads of U in flight.
__device__ __forceinline__ void utw_partials(const FusedArgs& a, const float* w, int64_t j0, int64_t j1, int nblk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int len = (int)(j1 - j0);
  constexpr int RW = 8;
  for (int i0 = warp * RW; i0 < a.s; i0 += nw * RW) {
    float acc[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) acc[q] = 0.f;
#pragma unroll 4
    for (int jj = lane; jj < len; jj += 32) {
      const float wv = w[j0 + jj];
#pragma unroll
      for (int q = 0; q < RW; ++q)
        if (i0 + q < a.s) acc[q] = fmaf(__ldg(a.U + (int64_t)(i0 + q) * a.d + j0 + jj), wv, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      acc[q] = warp_sum(acc[q]);
      if (lane == 0 && i0 + q < a.s) a.part_g[(int64_t)(i0 + q) * nblk + blockIdx.x] = acc[q];
    }
  }
}

// g_i = c_i sum_c part_g[i][c] (fixed order: lanes over CTAs, then a warp butterfly) into
// shared memory, every CTA the same values.  FP32 sums (the graph-driven loop adds the
// same FP32 partials in FP64): each CTA forms all s values, and s x #CTA FP64 additions
// would cost the SM's slow FP64 pipe more than the whole vector step.
__device__ __forceinline__ void g_from_partials(const FusedArgs& a, int nblk, float* gsh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int RW = 8;
  for (int i0 = warp * RW; i0 < a.s; i0 += nw * RW) {
    float acc[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) acc[q] = 0.f;
#pragma unroll 4
    for (int c = lane; c < nblk; c += 32) {
#pragma unroll
      for (int q = 0; q < RW; ++q)
        if (i0 + q < a.s) acc[q] += __ldcg(a.part_g + (int64_t)(i0 + q) * nblk + c);
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      acc[q] = warp_sum(acc[q]);
      if (lane == 0 && i0 + q < a.s) gsh[i0 + q] = a.cvec[i0 + q] * acc[q];
    }
  }
  __syncthreads();
}

// out_j = fma(shift, pv_j, s_j) for j in [j0, j1), s_j = sum over CTAs of the A-pass
// partials (times the FP8 column scale): the CTAs are cut into NG groups, each group
// summed in order by its own threads, then the group sums in order.  Returns this
// thread's part of sum_j pv_j out_j.
__device__ __forceinline__ double reduce_partials(const FusedArgs& a, const float* pv, float shift, float* out,
                                                  int64_t j0, int64_t j1, int nblk, float* redv) {
  const int len = (int)(j1 - j0);
  const int64_t dpad = a.pa.dpad;
  const float* cs = a.pa.col_scale;
  int ng = len > 0 ? (int)blockDim.x / len : 1;
  ng = max(1, min(ng, 8));
  double dot = 0.0;
  if (ng == 1) {
    for (int jl = threadIdx.x; jl < len; jl += blockDim.x) {
      const int64_t j = j0 + jl;
      float s = 0.f;
#pragma unroll 8
      for (int c = 0; c < nblk; ++c) s += __ldcg(a.partial + (int64_t)c * dpad + j);
      if (cs) s *= cs[j];
      const float o = fmaf(shift, pv[j], s);
      out[j] = o;
      dot += (double)pv[j] * (double)o;
    }
    return dot;
  }
  if ((int)threadIdx.x < ng * len) {
    const int g = threadIdx.x / len, jl = threadIdx.x % len;
    const int c0 = (int)((int64_t)nblk * g / ng), c1 = (int)((int64_t)nblk * (g + 1) / ng);
    float s = 0.f;
#pragma unroll 8
    for (int c = c0; c < c1; ++c) s += __ldcg(a.partial + (int64_t)c * dpad + j0 + jl);
    redv[g * len + jl] = s;
  }
  __syncthreads();
  for (int jl = threadIdx.x; jl < len; jl += blockDim.x) {
    const int64_t j = j0 + jl;
    float s = 0.f;
    for (int g = 0; g < ng; ++g) s += redv[g * len + jl];
    if (cs) s *= cs[j];
    const float o = fmaf(shift, pv[j], s);
    out[j] = o;
    dot += (double)pv[j] * (double)o;
  }
  __syncthreads();
  return dot;
}

// y_j = w_j + sum_i U_ij g_i over this CTA's slice (P^{-1} w of Eq. Nystrom preconditioner
// rearranged); with few elements per CTA the sum over i is cut into NG groups summed by
// their own threads (one memory latency chain per group instead of one per element), then
// added to w_j in group order.  Optionally also p_j = y_j.  Returns this thread's part of
// sum_j w_j y_j.
__device__ __forceinline__ double pinv_slice(const FusedArgs& a, int64_t j0, int64_t j1, const float* gsh,
                                             float* redv, float* p_out) {
  const int len = (int)(j1 - j0);
  const int64_t d = a.d;
  int ng = len > 0 ? (int)blockDim.x / len : 1;
  ng = max(1, min(ng, 8));
  double dot = 0.0;
  if (ng > 1) {
    if ((int)threadIdx.x < ng * len) {
      const int g = threadIdx.x / len, jl = threadIdx.x % len;
      const int i0 = a.s * g / ng, i1 = a.s * (g + 1) / ng;
      float acc = 0.f;
#pragma unroll 8
      for (int i = i0; i < i1; ++i) acc = fmaf(__ldg(a.U + (int64_t)i * d + j0 + jl), gsh[i], acc);
      redv[g * len + jl] = acc;
    }
    __syncthreads();
  }
  for (int jl = threadIdx.x; jl < len; jl += blockDim.x) {
    const int64_t j = j0 + jl;
    const float wj = a.w[j];
    float acc = wj;
    if (ng > 1) {
      for (int g = 0; g < ng; ++g) acc += redv[g * len + jl];
    } else {
#pragma unroll 8
      for (int i = 0; i < a.s; ++i) acc = fmaf(__ldg(a.U + (int64_t)i * d + j), gsh[i], acc);
    }
    a.y[j] = acc;
    if (p_out) p_out[j] = acc;
    dot += (double)wj * (double)acc;
  }
  __syncthreads();
  return dot;
}

// Loop state that lives across the A-passes.  It is kept in shared memory (written by
// thread 0, read by all after a barrier), and the kernel has ONE call site of the pass
// (a small state machine picks what the next pass is for), so that during a pass the
// roles' loops have the register file to themselves.
struct FusedLoop {
  double eps_next, tolk, thresh2, wy;
  const float *py, *pold;   // next pass: p_j = fmaf(pb, pold_j, py_j)
  float *pcur, *pnext;
  float pb;
  int k, kbase, iters, pstat, fixedk, stop, tol_abs, step;
  int at_start;   // 1: iteration k has not run its right-hand side yet
  int hx_done;    // the (H + rho I) x recompute of iteration k has run
  int mode;       // what the pending pass is for: 0 the recompute, 1 a PCG direction
  unsigned target;
  long long passes;
  int64_t j0, j1;
  int nwa;       // warps holding elements of the slice
};

template <int DT, int VPT, int R, int G>
__global__ void __maxnreg__(kFusedRegs) admm_fused_kernel(const FusedArgs a) {
  constexpr int NT = (2 * G + 2) * 32;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) WsFloatSmem<R, G> sm;
  __shared__ float gsh[kFusedMaxS];
  __shared__ float redv[NT];
  __shared__ double shv[5][NT / 32];
  __shared__ double bc[8];
  __shared__ FusedLoop L;
  volatile FusedLoop& V = L;
  const int tid = threadIdx.x;
  const int nblk = gridDim.x;
  if (tid == 0) {
    ws_init(sm.bars, a.pa.S, G, G);
    sm.abort_flag = 0;
    sm.loss = 0.0;
    L.eps_next = 0.0;
    L.k = 0;
    L.kbase = 0;
    L.stop = 0;
    L.at_start = 1;
    L.hx_done = 0;
    L.target = 0;
    L.passes = 0;
    L.pcur = a.pa_buf;
    L.pnext = a.pb_buf;
    L.j0 = a.d * blockIdx.x / nblk;
    L.j1 = a.d * (blockIdx.x + 1) / nblk;
    L.nwa = (int)min((int64_t)(NT / 32), (L.j1 - L.j0 + 31) / 32);
  }
  __syncthreads();
  auto barrier = [&]() -> bool {
    unsigned t = 0;
    if (tid == 0) {
      L.target += (unsigned)nblk;
      t = L.target;
    }
    if (grid_barrier_mono(a.bar, t)) return true;
    if (tid == 0) atomicExch(a.status, (int)NYS_ETIMEOUT);
    return false;
  };
  // prox / dual step with the new x and the scalars of the iteration; false: stop
  auto finish_iter = [&]() -> bool {
    {
      double* zt = a.ztrace ? a.ztrace + (int64_t)V.k * a.d : nullptr;
      double v5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int64_t j = V.j0 + tid; j < V.j1; j += NT) {
        const double xj = (double)a.xc[j];
        const double zo = a.z[j];
        const double uo = a.u[j];
        const double vj = xj + uo;
        const double mag = fabs(vj) - a.kappa;
        const double zj = mag > 0.0 ? copysign(mag, vj) : 0.0;
        const double uj = uo + xj - zj;
        a.x[j] = xj;
        a.z[j] = zj;
        a.u[j] = uj;
        if (zt) zt[j] = zj;
        v5[0] += (xj - zj) * (xj - zj);
        v5[1] += (zj - zo) * (zj - zo);
        v5[2] += xj * xj;
        v5[3] += zj * zj;
        v5[4] += uj * uj;
      }
      fused_block_sum<5, NT>(v5, shv, V.nwa);
      if (tid == 0) {
#pragma unroll
        for (int t = 0; t < 5; ++t) a.part[(int64_t)blockIdx.x * kPartW + kSlotZu + t] = v5[t];
      }
    }
    if (!barrier()) return false;
    double s5[5];
    grid_sums<5>(a.part, nblk, kSlotZu, s5, bc);
    if (tid == 0) {
      const double rp = sqrt(s5[0]);
      const double rd = a.rho * sqrt(s5[1]);
      L.eps_next = sqrt(rp * rd);
      if (a.eps_rel > 0.0) {
        const double tp = a.eps_abs + a.eps_rel * fmax(sqrt(s5[2]), sqrt(s5[3]));
        const double td = a.eps_abs + a.eps_rel * a.rho * sqrt(s5[4]);
        if (rp <= tp && rd <= td) L.stop = 1;
      }
      if (L.pstat == NYS_EBREAKDOWN) L.stop = 2;
      if (blockIdx.x == 0) {
        a.rp[L.k] = rp;
        a.rd[L.k] = rd;
        a.pcg_it[L.k] = L.iters;
      }
      L.k += 1;
      L.at_start = 1;
      L.hx_done = 0;
    }
    __syncthreads();
    return true;
  };
  const float shift = (float)(a.rho + a.mu);
  for (;;) {
    if (V.at_start) {
      if (V.k >= a.K || V.stop) break;
      const bool due = V.k > 0 && (a.hx_refresh == 0 || V.k % a.hx_refresh == 0) && !V.hx_done;
      __syncthreads();
      if (due) {
        // ---- (H + rho I) x recomputed every hx_refresh iterations, every iteration for 0
        // (x = 0 at k = 0: hx = 0); the right-hand side follows once it is reduced
        if (tid == 0) {
          L.py = a.xc;
          L.pold = a.xc;
          L.pb = 0.f;
          L.mode = 0;
        }
        __syncthreads();
      } else {
        if (tid == 0) {
          double tk;
          int ta;
          fused_tol(a, L.k, L.eps_next, &tk, &ta);
          L.tolk = tk;
          L.tol_abs = ta;
          L.iters = 0;
          L.pstat = 0;
          L.fixedk = a.fixed ? a.fixed[L.k] : -1;
        }
        __syncthreads();
        // ---- right-hand side, warm-start residual w = r - (H + rho I) x, norms, U^T w partials
        {
          double v2[2] = {0.0, 0.0};
          for (int64_t j = V.j0 + tid; j < V.j1; j += NT) {
            const float rj = (float)fma(a.rho, a.z[j] - a.u[j], a.q[j]);
            const float wj = rj - a.hx[j];
            a.w[j] = wj;
            v2[0] += (double)wj * (double)wj;
            v2[1] += (double)rj * (double)rj;
          }
          fused_block_sum<2, NT>(v2, shv, V.nwa);
          if (tid == 0) {
            a.part[(int64_t)blockIdx.x * kPartW + kSlotW2] = v2[0];
            a.part[(int64_t)blockIdx.x * kPartW + kSlotR2] = v2[1];
          }
          utw_partials(a, a.w, V.j0, V.j1, nblk);
        }
        if (!barrier()) return;
        {
          double sums2[2];
          grid_sums<2>(a.part, nblk, kSlotW2, sums2, bc);
          if (tid == 0) {
            L.thresh2 = L.tol_abs ? L.tolk * L.tolk : L.tolk * L.tolk * sums2[1];
            // a step unless the warm start already meets the tolerance (or the replayed count is 0)
            L.step = L.fixedk >= 0 ? (L.fixedk != 0) : (sums2[0] > L.thresh2);
          }
          __syncthreads();
        }
        if (!V.step) {
          if (!finish_iter()) return;
          continue;
        }
        // ---- first direction p = y = P^{-1} w
        g_from_partials(a, nblk, gsh);
        {
          double wy[1] = {pinv_slice(a, V.j0, V.j1, gsh, redv, V.pcur)};
          fused_block_sum<1, NT>(wy, shv, V.nwa);
          if (tid == 0) a.part[(int64_t)blockIdx.x * kPartW + kSlotWy] = wy[0];
        }
        if (!barrier()) return;
        {
          double wyv[1];
          grid_sums<1>(a.part, nblk, kSlotWy, wyv, bc);
          if (tid == 0) {
            L.wy = wyv[0];
            L.py = L.pcur;
            L.pold = L.pcur;
            L.pb = 0.f;
            L.mode = 1;
            L.at_start = 0;
          }
          __syncthreads();
        }
      }
    }
    // ---- the pass: v = (H + rho I) p, or the recompute
    {
      const bool ok = ws_pass_float<DT, VPT, R, G>(a.pa, sm, smem, V.kbase, PSrcAxpy{V.py, V.pold, V.pb});
      __syncthreads();
      if (tid == 0) {
        L.kbase += ws_pass_steps(a.pa.n, R);
        L.passes += 1;
      }
      __syncthreads();
      if (!ok) return;
    }
    if (!barrier()) return;
    if (V.mode == 0) {
      (void)reduce_partials(a, a.xc, shift, a.hx, V.j0, V.j1, nblk, redv);
      if (tid == 0) L.hx_done = 1;
      __syncthreads();
      continue;
    }
    {
      double pv[1];
      pv[0] = reduce_partials(a, V.pcur, shift, a.v, V.j0, V.j1, nblk, redv);
      fused_block_sum<1, NT>(pv, shv, V.nwa);
      if (tid == 0) a.part[(int64_t)blockIdx.x * kPartW + kSlotPv] = pv[0];
    }
    if (!barrier()) return;
    double pvv[1];
    grid_sums<1>(a.part, nblk, kSlotPv, pvv, bc);
    const double pv = pvv[0];
    if (!(pv > 0.0) || !isfinite(pv)) {
      if (tid == 0) L.pstat = L.iters == 0 ? NYS_EBREAKDOWN : NYS_ENOCONV;
      __syncthreads();
      if (!finish_iter()) return;
      continue;
    }
    // ---- x += alpha p, w -= alpha v, (H + rho I) x += alpha v, ||w||^2, U^T w
    {
      const float al = (float)(V.wy / pv);
      const float* pc = V.pcur;
      double lw[1] = {0.0};
      for (int64_t j = V.j0 + tid; j < V.j1; j += NT) {
        const float vj = a.v[j];
        a.xc[j] = fmaf(al, pc[j], a.xc[j]);
        const float wj = fmaf(-al, vj, a.w[j]);
        a.w[j] = wj;
        a.hx[j] = fmaf(al, vj, a.hx[j]);
        lw[0] += (double)wj * (double)wj;
      }
      fused_block_sum<1, NT>(lw, shv, V.nwa);
      if (tid == 0) a.part[(int64_t)blockIdx.x * kPartW + kSlotW2b] = lw[0];
      utw_partials(a, a.w, V.j0, V.j1, nblk);
    }
    if (!barrier()) return;
    {
      double w2v[1];
      grid_sums<1>(a.part, nblk, kSlotW2b, w2v, bc);
      const double w2 = w2v[0];
      if (tid == 0) {
        int done = 0;
        if (!isfinite(w2)) {
          L.pstat = L.iters == 0 ? NYS_EBREAKDOWN : NYS_ENOCONV;
          done = 1;
        } else {
          L.iters += 1;
          if (L.fixedk >= 0) {
            done = L.iters >= L.fixedk;
          } else if (!(w2 > L.thresh2)) {
            done = 1;
          } else if (L.iters >= a.maxit) {
            done = 1;
            L.pstat = NYS_ENOCONV;
          }
        }
        L.step = done;
      }
      __syncthreads();
    }
    if (V.step) {
      if (!finish_iter()) return;
      continue;
    }
    // ---- y = P^{-1} w, beta, next direction p' = y + beta p
    g_from_partials(a, nblk, gsh);
    {
      double wyn[1] = {pinv_slice(a, V.j0, V.j1, gsh, redv, nullptr)};
      fused_block_sum<1, NT>(wyn, shv, V.nwa);
      if (tid == 0) a.part[(int64_t)blockIdx.x * kPartW + kSlotWyb] = wyn[0];
    }
    if (!barrier()) return;
    {
      double wynv[1];
      grid_sums<1>(a.part, nblk, kSlotWyb, wynv, bc);
      const float beta = (float)(wynv[0] / V.wy);
      const float* pc = V.pcur;
      float* pn = V.pnext;
      for (int64_t j = V.j0 + tid; j < V.j1; j += NT) pn[j] = fmaf(beta, pc[j], a.y[j]);
      __syncthreads();
      if (tid == 0) {
        L.wy = wynv[0];
        L.py = a.y;
        L.pold = L.pcur;
        L.pb = beta;
        L.pcur = L.pnext;
        L.pnext = const_cast<float*>(L.pold);
      }
      __syncthreads();
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    *a.k_out = L.k;
    *a.stop_out = L.stop;
    if (a.passes) *a.passes = L.passes;
  }
}

// Instantiated for the warp-specialised plans with two rows per stage (the planner's
// choice for rows of 8 to 64 KB); other plans run the graph-driven loop.  The pass keeps
// the stand-alone layout (kWsGroupWarps dot and update warps, the planner's vectors per
// thread), so the per-CTA partials are those of apass_ws_kernel bit for bit.
using FusedFn = void (*)(const FusedArgs);
// The shapes whose kernel keeps every role's working set in registers at kFusedRegs:
// FP32 with up to 10 vectors per thread, BF16 with 1-3 or 5, FP8 with 1-2.  The others
// run the graph-driven loop.
template <int DT>
FusedFn fused_kernel_for(int vpt) {
  constexpr int G = kWsGroupWarps;
  switch (vpt) {
    case 1: return admm_fused_kernel<DT, 1, 2, G>;
    case 2: return admm_fused_kernel<DT, 2, 2, G>;
    case 3:
      if constexpr (DT != NYS_FP8E4M3) return admm_fused_kernel<DT, 3, 2, G>;
      break;
    case 4:
      if constexpr (DT == NYS_F32) return admm_fused_kernel<DT, 4, 2, G>;
      break;
    case 5:
      if constexpr (DT != NYS_FP8E4M3) return admm_fused_kernel<DT, 5, 2, G>;
      break;
    case 6:
      if constexpr (DT == NYS_F32) return admm_fused_kernel<DT, 6, 2, G>;
      break;
    case 8:
      if constexpr (DT == NYS_F32) return admm_fused_kernel<DT, 8, 2, G>;
      break;
    case 10:
      if constexpr (DT == NYS_F32) return admm_fused_kernel<DT, 10, 2, G>;
      break;
    default: break;
  }
  return nullptr;
}

}  // namespace

nys_status admm_fused_try(const GraphLoopArgs& g, cudaStream_t st, GraphLoopResult* res, bool* ran) {
  *ran = false;
  const bool trace = std::getenv("NYS_TRACE") != nullptr;
  auto skip = [&](const char* why) {
    if (trace) std::fprintf(stderr, "[nys] fused loop not used: %s\n", why);
    return NYS_OK;
  };
  const char* env = std::getenv("NYS_ADMM_FUSED");
  if (env && std::atoi(env) == 0) return skip("NYS_ADMM_FUSED=0");
  const nys_matrix* A = g.pb.A;
  const ApassPlan& plan = g.pb.plan;
  if (!plan.ws || plan.rows_per_step != 2 || compute_is_f64(A->dtype)) return skip("pass plan");
  if (g.Aref || g.warm || g.warm_record || !g.allow_nostep || shard_comm().fn) return skip("solve options");
  const int s = g.P.s;
  if (s > kFusedMaxS || plan.grid > kFusedMaxGrid || plan.grid > sm_count() || g.K <= 0) return skip("sizes");
  FusedFn fn = nullptr;
  const int vpt = plan.vpt;
  switch (A->dtype) {
    case NYS_F32: fn = fused_kernel_for<NYS_F32>(vpt); break;
    case NYS_BF16: fn = fused_kernel_for<NYS_BF16>(vpt); break;
    case NYS_FP8E4M3: fn = fused_kernel_for<NYS_FP8E4M3>(vpt); break;
    default: break;
  }
  if (!fn) return skip("no kernel for this row width");
  const int threads = (2 * kWsGroupWarps + 2) * 32;
  if (ensure_max_dyn_smem((const void*)fn, kSmemBudget) != cudaSuccess) {
    cudaGetLastError();
    return skip("shared memory attribute");
  }
  int coop = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, current_device()) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, threads, plan.smem) != cudaSuccess ||
      !coop || per_sm < 1) {
    cudaGetLastError();
    if (trace) {
      cudaFuncAttributes fa_ = {};
      cudaFuncGetAttributes(&fa_, (const void*)fn);
      std::fprintf(stderr, "[nys] fused loop: %d regs, %zu static smem, %zu dynamic, %d per SM\n", fa_.numRegs,
                   fa_.sharedSizeBytes, plan.smem, per_sm);
    }
    return skip("occupancy");
  }
  *ran = true;
  const int64_t d = A->d;
  const int nblk = plan.grid;
  Pool pool(st);
  FusedArgs fa = {};
  fa.partial = reinterpret_cast<float*>(pool.alloc<unsigned char>(apass_partial_bytes(A, plan)));
  fa.part = pool.alloc<double>((size_t)nblk * kPartW);
  fa.part_g = pool.alloc<float>((size_t)nblk * std::max(1, s));
  fa.w = pool.alloc<float>(d);
  fa.y = pool.alloc<float>(d);
  fa.v = pool.alloc<float>(d);
  fa.pa_buf = pool.alloc<float>(d);
  fa.pb_buf = pool.alloc<float>(d);
  int* words = pool.alloc<int>(8);
  long long* passes = pool.alloc<long long>(1);
  int* fixed_dev = g.fixed_host ? pool.alloc<int>(g.K) : nullptr;
  if (!pool.ok()) return NYS_ENOMEM;
  FUSED_CU(cudaMemsetAsync(words, 0, 8 * sizeof(int), st));
  FUSED_CU(cudaMemsetAsync(g.hx, 0, d * sizeof(float), st));
  if (fixed_dev) FUSED_CU(cudaMemcpyAsync(fixed_dev, g.fixed_host, g.K * sizeof(int), cudaMemcpyHostToDevice, st));
  ApassKArgs& k = fa.pa;
  k.A = reinterpret_cast<const unsigned char*>(A->data);
  k.n = A->n;
  k.d = d;
  k.ld = A->ld;
  k.p = nullptr;
  k.D = g.pb.D;
  k.b = nullptr;
  k.D_out = nullptr;
  k.t_out = nullptr;
  k.mode = g.pb.D ? MODE_DIAG : MODE_ID;
  k.R = plan.rows_per_step;
  k.S = plan.stages;
  k.dpad = plan.dpad;
  k.partial = fa.partial;
  k.loss_part = nullptr;
  k.status = words;
  k.skip = nullptr;
  k.executed = nullptr;
  k.col_scale = A->col_scale;
  k.tm = stats_device_timer();
  k.bytes_alg = (double)A->n * (double)d * (double)dtype_size(A->dtype) + 4.0 * d + 4.0 * nblk * d +
                (g.pb.D ? 8.0 * A->n : 0.0);
  fa.d = d;
  fa.s = s;
  fa.U = reinterpret_cast<const float*>(g.P.U);
  fa.cvec = reinterpret_cast<const float*>(g.P.c);
  fa.q = g.q;
  fa.x = g.x;
  fa.z = g.z;
  fa.u = g.u;
  fa.xc = reinterpret_cast<float*>(g.xc);
  fa.hx = reinterpret_cast<float*>(g.hx);
  fa.bar = reinterpret_cast<unsigned*>(words + 1);
  fa.status = words;
  fa.k_out = words + 2;
  fa.stop_out = words + 3;
  fa.rho = g.rho;
  fa.mu = g.mu;
  fa.kappa = g.gamma / g.rho;
  fa.tol = g.tol;
  fa.tol_floor = g.tol_floor;
  fa.tol_mode = g.tol_mode;
  fa.maxit = g.maxit;
  fa.hx_refresh = g.hx_refresh;
  fa.K = g.K;
  fa.fixed = fixed_dev;
  fa.eps_abs = g.eps_abs;
  fa.eps_rel = g.eps_rel;
  fa.ztrace = g.ztrace;
  fa.rp = g.rp;
  fa.rd = g.rd;
  fa.pcg_it = g.pcg_it;
  fa.passes = passes;
  void* args[] = {(void*)&fa};
  count_launch();
  FUSED_CU(cudaLaunchCooperativeKernel((const void*)fn, dim3(nblk), dim3(threads), args, plan.smem, st));
  int h[4] = {0, 0, 0, 0};
  long long hp = 0;
  FUSED_CU(cudaMemcpyAsync(h, words, sizeof(h), cudaMemcpyDeviceToHost, st));
  FUSED_CU(cudaMemcpyAsync(&hp, passes, sizeof(hp), cudaMemcpyDeviceToHost, st));
  FUSED_CU(cudaStreamSynchronize(st));
  res->admm_iters = h[2];
  res->breakdown = h[3] == 2;
  return h[0] ? (nys_status)h[0] : NYS_OK;
}

}  // namespace nys
