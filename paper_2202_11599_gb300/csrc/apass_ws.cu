// Warp-specialised fused A-pass kernels: one pass y = A^T phi(A p) per launch (Table 1's
// T_mv, the H-matvec of Alg. Nystrom PCG), the same result layout as the kernels of
// apass.cu.  The roles and their per-stage mbarriers are described in apass_ws.cuh.
#include "apass_ws.cuh"

namespace nys {

// ------------------------------------------------------------------ float compute
template <int DT, int VPT, int R, int G>
__global__ void __launch_bounds__((2 * G + 2) * 32, 1) apass_ws_kernel(const ApassKArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) WsFloatSmem<R, G> sm;
  if (a.skip && *a.skip) return;
  if (a.executed && blockIdx.x == 0 && threadIdx.x == 0) *a.executed = 1;
  if (threadIdx.x == 0) {
    ws_init(sm.bars, a.S, G, G);
    sm.abort_flag = 0;
    sm.loss = 0.0;
  }
  __syncthreads();
  (void)ws_pass_float<DT, VPT, R, G>(a, sm, smem, 0, PSrcPlain{reinterpret_cast<const float*>(a.p)});
}

// ------------------------------------------------------------------ FP64 compute
// FP64 storage: the pass is bound by the FP64 FMA rate, so the roles are sized for the
// register file: G dot warps read p through L1 (it stays cached next to the stage ring),
// GU = 2G update warps hold the partial sums (VPT 16-byte vectors = 2 VPT doubles each).
template <int VPT, int R, int G>
__global__ void __launch_bounds__((3 * G + 2) * 32, 1) apass_ws64_kernel(const ApassKArgs a) {
  constexpr int GU = 2 * G;
  constexpr int TG = 32 * G;    // dot-group threads
  constexpr int TU = 32 * GU;   // update-group threads

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) WsBars bars;
  __shared__ double red[kWsMaxStages][G][R];
  __shared__ double us[kWsMaxStages][R];
  __shared__ int abort_flag;
  __shared__ double loss_sh;

  if (a.skip && *a.skip) return;
  if (a.executed && blockIdx.x == 0 && threadIdx.x == 0) *a.executed = 1;
  const int ts_slot = timer_begin(a);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nvec = (int)((a.d + 1) / 2);
  const uint32_t rowbytes = (uint32_t)(a.ld * 8);
  const int S = a.S;
  const uint32_t stage_bytes = (uint32_t)R * rowbytes;
  const int64_t r0 = a.n * (int64_t)blockIdx.x / gridDim.x;
  const int64_t r1 = a.n * (int64_t)(blockIdx.x + 1) / gridDim.x;
  const int nsteps = (int)((r1 - r0 + R - 1) / R);
  const int tail_vec = (int)(a.d / 2);   // the vector holding column d - 1 when d is odd
  const bool odd = (a.d & 1) != 0;
  const bool nodot = a.mode == MODE_CONST;
  const uint32_t sbase = smem_u32(smem);
  volatile int* abort_v = &abort_flag;

  if (tid == 0) {
    ws_init(bars, S, G, GU);
    abort_flag = 0;
    loss_sh = 0.0;
  }
  __syncthreads();

  double2 acc[VPT];
  int issued = 0;
  if (warp < G) {
    if (!nodot) {
      const double* p = reinterpret_cast<const double*>(a.p);
      const bool p16 = (reinterpret_cast<uintptr_t>(p) & 15u) == 0;   // 16-byte loads allowed
      const int nv_dot = (nvec + TG - 1) / TG;
      int st = 0;
      uint32_t ph = 0;
      for (int k = 0; k < nsteps; ++k, st = st + 1 == S ? 0 : st + 1, ph ^= st == 0 ? 1u : 0u) {
        if (!warp_wait(&bars.full[st], ph)) {
          *abort_v = 1;
          break;
        }
        const int rows_here = (int)min((int64_t)R, r1 - (r0 + (int64_t)k * R));
        const uint32_t sb = sbase + (uint32_t)st * stage_bytes;
        double dacc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) dacc[r] = 0.0;
        for (int kk = 0; kk < nv_dot; ++kk) {
          const int v = tid + kk * TG;
          if (v < nvec) {
            double p0, p1;
            if (odd && v == tail_vec) {
              p0 = __ldg(p + 2 * (int64_t)v);
              p1 = 0.0;
            } else if (!p16) {
              p0 = __ldg(p + 2 * (int64_t)v);
              p1 = __ldg(p + 2 * (int64_t)v + 1);
            } else {
              const double2 pv = __ldg(reinterpret_cast<const double2*>(p) + v);
              p0 = pv.x;
              p1 = pv.y;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
              if (r < rows_here) {
                uint4 x = lds128(sb + (uint32_t)r * rowbytes + (uint32_t)v * 16u);
                if (odd && v == tail_vec) x.z = x.w = 0u;
                dacc[r] = fma(__hiloint2double((int)x.y, (int)x.x), p0, dacc[r]);
                dacc[r] = fma(__hiloint2double((int)x.w, (int)x.z), p1, dacc[r]);
              }
            }
          }
        }
        double sums[R];
#pragma unroll
        for (int r = 0; r < R; ++r) sums[r] = dacc[r];
        const double tot = warp_sum_rows<R>(sums, lane);
        if ((lane & (32 / R - 1)) == 0) red[st][warp][lane / (32 / R)] = tot;
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.dotted[st]);
      }
    }
  } else if (warp < G + GU) {
    const int j = tid - TG;
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) acc[kk] = make_double2(0.0, 0.0);
    int st = 0;
    uint32_t ph = 0;
    for (int k = 0; k < nsteps; ++k, st = st + 1 == S ? 0 : st + 1, ph ^= st == 0 ? 1u : 0u) {
      if (!warp_wait(&bars.ready[st], ph) || !warp_wait(&bars.full[st], ph)) {
        *abort_v = 1;
        break;
      }
      const int rows_here = (int)min((int64_t)R, r1 - (r0 + (int64_t)k * R));
      const uint32_t sb = sbase + (uint32_t)st * stage_bytes;
      double u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = us[st][r];
#pragma unroll
      for (int kk = 0; kk < VPT; ++kk) {
        const int v = j + kk * TU;
        if (v < nvec) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            if (r < rows_here) {
              uint4 x = lds128(sb + (uint32_t)r * rowbytes + (uint32_t)v * 16u);
              if (odd && v == tail_vec) x.z = x.w = 0u;
              acc[kk].x = fma(__hiloint2double((int)x.y, (int)x.x), u[r], acc[kk].x);
              acc[kk].y = fma(__hiloint2double((int)x.w, (int)x.z), u[r], acc[kk].y);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.empty[st]);
    }
  } else if (warp == G + GU) {
    if (lane == 0) issued = ws_produce(a, bars, smem, nsteps, R, S, rowbytes, r0, r1, abort_v);
  } else {
    double l = ws_finish<double, R, G>(a, bars, red, us, nsteps, S, r0, r1, abort_v);
    l = warp_sum(l);
    if (lane == 0) loss_sh = l;
  }

  __syncthreads();
  if (abort_flag) {
    if (warp == G + GU && lane == 0) {
      for (int k = max(0, issued - S); k < issued; ++k)
        (void)mbar_wait_bounded(&bars.full[k % S], (uint32_t)((k / S) & 1));
      atomicExch(a.status, (int)NYS_ETIMEOUT);
    }
    return;
  }
  if (warp >= G && warp < G + GU) {
    double* part = reinterpret_cast<double*>(a.partial) + (int64_t)blockIdx.x * a.dpad;
    const int j = tid - TG;
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int v = j + kk * TU;
      if (v < nvec) *reinterpret_cast<double2*>(part + 2 * (int64_t)v) = acc[kk];
    }
  }
  if (tid == 0 && a.loss_part) a.loss_part[blockIdx.x] = loss_sh;
  timer_end(a, ts_slot, NYS_F64);
}

// ------------------------------------------------------------------ host side
namespace {

// Column vectors per thread of a group, from the instantiated set.
int ws_vpt(int64_t nvec, int group_threads, const int* set, int nset) {
  const int64_t need = (nvec + group_threads - 1) / group_threads;
  for (int i = 0; i < nset; ++i)
    if (need <= set[i]) return set[i];
  return -1;
}

constexpr int kVptF32[] = {1, 2, 3, 4, 5, 6, 8, 10};
constexpr int kVptBF16[] = {1, 2, 3, 4, 5, 6, 8};
constexpr int kVptFP8[] = {1, 2, 3, 4};
constexpr int kVptF64[] = {1, 2, 4, 6, 8, 10, 12};

template <typename K>
cudaError_t ws_launch_kernel(K fn, int threads, const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st,
                             bool prepare_only) {
  NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)fn, kSmemBudget));
  if (prepare_only) return cudaSuccess;
  count_launch();
  fn<<<plan.grid, threads, plan.smem, st>>>(k);
  return cudaGetLastError();
}

template <int DT, int VPT>
cudaError_t ws_float_r(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st, bool prep) {
  constexpr int G = kWsGroupWarps;
  switch (plan.rows_per_step) {
    case 1: return ws_launch_kernel(apass_ws_kernel<DT, VPT, 1, G>, (2 * G + 2) * 32, k, plan, st, prep);
    case 2: return ws_launch_kernel(apass_ws_kernel<DT, VPT, 2, G>, (2 * G + 2) * 32, k, plan, st, prep);
    case 4: return ws_launch_kernel(apass_ws_kernel<DT, VPT, 4, G>, (2 * G + 2) * 32, k, plan, st, prep);
    default: return cudaErrorInvalidValue;
  }
}

template <int DT>
cudaError_t ws_float(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st, bool prep) {
  switch (plan.vpt) {
    case 1: return ws_float_r<DT, 1>(k, plan, st, prep);
    case 2: return ws_float_r<DT, 2>(k, plan, st, prep);
    case 3: return ws_float_r<DT, 3>(k, plan, st, prep);
    case 4: return ws_float_r<DT, 4>(k, plan, st, prep);
    case 5:
      if constexpr (DT != NYS_FP8E4M3) return ws_float_r<DT, 5>(k, plan, st, prep);
      break;
    case 6:
      if constexpr (DT != NYS_FP8E4M3) return ws_float_r<DT, 6>(k, plan, st, prep);
      break;
    case 8:
      if constexpr (DT != NYS_FP8E4M3) return ws_float_r<DT, 8>(k, plan, st, prep);
      break;
    case 10:
      if constexpr (DT == NYS_F32) return ws_float_r<DT, 10>(k, plan, st, prep);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

template <int VPT>
cudaError_t ws64_r(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st, bool prep) {
  constexpr int G = kWs64DotWarps;
  switch (plan.rows_per_step) {
    case 1: return ws_launch_kernel(apass_ws64_kernel<VPT, 1, G>, (3 * G + 2) * 32, k, plan, st, prep);
    case 2: return ws_launch_kernel(apass_ws64_kernel<VPT, 2, G>, (3 * G + 2) * 32, k, plan, st, prep);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t ws64(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st, bool prep) {
  switch (plan.vpt) {
    case 1: return ws64_r<1>(k, plan, st, prep);
    case 2: return ws64_r<2>(k, plan, st, prep);
    case 4: return ws64_r<4>(k, plan, st, prep);
    case 6: return ws64_r<6>(k, plan, st, prep);
    case 8: return ws64_r<8>(k, plan, st, prep);
    case 10: return ws64_r<10>(k, plan, st, prep);
    case 12: return ws64_r<12>(k, plan, st, prep);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool apass_ws_layout(int dtype, int64_t d, int* threads, int* vpt) {
  switch (dtype) {
    case NYS_F32: *vpt = ws_vpt((d + 3) / 4, 32 * kWsGroupWarps, kVptF32, 8); break;
    case NYS_BF16: *vpt = ws_vpt((d + 7) / 8, 32 * kWsGroupWarps, kVptBF16, 7); break;
    case NYS_FP8E4M3: *vpt = ws_vpt((d + 15) / 16, 32 * kWsGroupWarps, kVptFP8, 4); break;
    case NYS_F64: *vpt = ws_vpt((d + 1) / 2, 32 * 2 * kWs64DotWarps, kVptF64, 7); break;
    default: return false;
  }
  if (*vpt < 0) return false;
  *threads = dtype == NYS_F64 ? (3 * kWs64DotWarps + 2) * 32 : (2 * kWsGroupWarps + 2) * 32;
  return true;
}

cudaError_t apass_ws_launch(const ApassKArgs& k, const ApassPlan& plan, int dtype, cudaStream_t st,
                            bool prepare_only) {
  if (plan.stages > kWsMaxStages || plan.stages < 2) return cudaErrorInvalidValue;
  switch (dtype) {
    case NYS_F32: return ws_float<NYS_F32>(k, plan, st, prepare_only);
    case NYS_BF16: return ws_float<NYS_BF16>(k, plan, st, prepare_only);
    case NYS_FP8E4M3: return ws_float<NYS_FP8E4M3>(k, plan, st, prepare_only);
    case NYS_F64: return ws64(k, plan, st, prepare_only);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nys
