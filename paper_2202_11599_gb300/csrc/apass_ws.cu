// Warp-specialised fused A-pass: y = A^T phi(A p) with one read of A (Table 1's T_mv,
// the H-matvec of Alg. Nystrom PCG), the same result layout as the kernels of apass.cu.
//
// The step of the classic pass makes every warp of the CTA wait twice per group of R
// rows for the cross-warp reduction of the row dots.  Here the CTA is split into roles
// that meet only through per-stage mbarriers, so no warp waits for the whole CTA while
// A streams:
//   * a producer warp (lane 0) issues the TMA bulk copy of each stage of R rows into a
//     ring of S stages and re-arms a stage once the update warps have released it;
//   * G "dot" warps form the partial row dots a_i . p of each stage (p in registers;
//     for FP64, where p does not fit in registers next to the partial sums, p is read
//     through the L1 cache), one warp reduction per row, and arrive on `dotted`;
//   * a finisher warp sums the G partials of each row in a fixed order (lane r takes
//     row r), applies the row mode phi (D_i t, the residual, the logistic weights),
//     writes the per-row side outputs and arrives on `ready`;
//   * GU "update" warps keep the CTA's partial of A^T u in registers, apply the rank-R
//     update of each stage from shared memory and release the stage on `empty`.
// The dot warps run up to S - 1 stages ahead of the update warps, so the reduction of
// one stage overlaps the dot products of the next.  Every wait is bounded: a role whose
// wait runs out raises the CTA's abort flag, all roles leave their loops, the producer
// drains its copies still in flight and the pass reports NYS_ETIMEOUT.
// Partial sums are written per CTA and summed in a fixed order by apass_reduce, so the
// result is bitwise reproducible from run to run.
#include <type_traits>

#include "apass_common.cuh"

namespace nys {

constexpr int kWsMaxStages = 12;

// Shared-memory ring control: one set of barriers per stage.
struct WsBars {
  uint64_t full[kWsMaxStages];    // TMA bytes landed (producer's expect_tx + copy)
  uint64_t dotted[kWsMaxStages];  // G dot warps wrote their partial row dots
  uint64_t ready[kWsMaxStages];   // finisher wrote u_i of the stage's rows
  uint64_t empty[kWsMaxStages];   // GU update warps are done reading the stage
};

__device__ __forceinline__ void ws_init(WsBars& b, int S, int G, int GU) {
  for (int st = 0; st < S; ++st) {
    mbar_init(&b.full[st], 1);
    mbar_init(&b.dotted[st], G);
    mbar_init(&b.ready[st], 1);
    mbar_init(&b.empty[st], GU);
  }
  fence_mbar_init();
}

// Warp sums of R per-lane values (R = 1, 2, 4) by a reduce-scatter over the lane bits:
// the first log2(R) exchanges split the rows between lane halves, the rest finish each
// row; the fixed order makes the sums bitwise reproducible.  Returns, in lane r (32 / R),
// the total of row r (every other lane holds a partial).
template <int R, typename T>
__device__ __forceinline__ T warp_sum_rows(const T (&v)[R], int lane) {
  constexpr unsigned F = 0xffffffffu;
  if constexpr (R == 1) {
    return warp_sum(v[0]);
  } else if constexpr (R == 2) {
    const bool hi = (lane & 16) != 0;
    T keep = hi ? v[1] : v[0];
    keep += __shfl_xor_sync(F, hi ? v[0] : v[1], 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(F, keep, o);
    return keep;
  } else {
    static_assert(R == 4, "rows per stage: 1, 2 or 4");
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
    T ka = b4 ? v[2] : v[0], kb = b4 ? v[3] : v[1];
    ka += __shfl_xor_sync(F, b4 ? v[0] : v[2], 16);
    kb += __shfl_xor_sync(F, b4 ? v[1] : v[3], 16);
    T keep = b3 ? kb : ka;
    keep += __shfl_xor_sync(F, b3 ? ka : kb, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) keep += __shfl_xor_sync(F, keep, o);
    return keep;
  }
}

// Producer (lane 0 of its warp): issues stage k once stage k - S has been released.
// Returns the number of stages issued.
__device__ __forceinline__ int ws_produce(const ApassKArgs& a, WsBars& b, unsigned char* smem, int nsteps, int R,
                                          int S, uint32_t rowbytes, int64_t r0, int64_t r1, volatile int* abort_flag) {
  const uint64_t pol = l2_evict_first_policy();  // A is streamed once per pass
  const uint32_t stage_bytes = (uint32_t)R * rowbytes;
  int issued = 0;
  for (int k = 0; k < nsteps; ++k) {
    const int st = k % S;
    if (k >= S && !mbar_wait_bounded(&b.empty[st], (uint32_t)(((k / S) - 1) & 1))) {
      *abort_flag = 1;
      break;
    }
    const int64_t row = r0 + (int64_t)k * R;
    const uint32_t bytes = (uint32_t)min((int64_t)R, r1 - row) * rowbytes;
    mbar_arrive_expect_tx(&b.full[st], bytes);
    tma_load_1d_hint(smem + (size_t)st * stage_bytes, a.A + row * (int64_t)rowbytes, bytes, &b.full[st], pol);
    issued = k + 1;
  }
  return issued;
}

// Finisher warp: u_i = phi(t_i) for the rows of each stage, t_i summed over the G dot
// warps' partials in a fixed order.  Returns this lane's share of the pass's loss term.
template <typename C, int R, int G>
__device__ __forceinline__ double ws_finish(const ApassKArgs& a, WsBars& b, const C (*red)[G][R], C (*us)[R],
                                            int nsteps, int S, int64_t r0, int64_t r1, volatile int* abort_flag) {
  const int lane = threadIdx.x & 31;
  const bool nodot = a.mode == MODE_CONST;
  double loss = 0.0;
  for (int k = 0; k < nsteps; ++k) {
    const int st = k % S;
    const uint32_t ph = (uint32_t)((k / S) & 1);
    const int64_t row0 = r0 + (int64_t)k * R;
    const int rows_here = (int)min((int64_t)R, r1 - row0);
    // the row's mode input (D_i or b_i) is loaded before the waits
    const double rin = (lane < R && lane < rows_here) ? row_input(a, row0 + lane) : 0.0;
    // waiting for the stage itself orders the writes of us[st] after its previous use
    // (the stage was re-armed only after the update warps released it)
    if (!warp_wait(&b.full[st], ph) || (!nodot && !warp_wait(&b.dotted[st], ph))) {
      *abort_flag = 1;
      break;
    }
    if (lane < R) {
      C u = C(0);
      if (lane < rows_here) {
        const int64_t i = row0 + lane;
        C t = C(0);
        if (!nodot) {
#pragma unroll
          for (int w = 0; w < G; ++w) t += red[st][w][lane];
        }
        if constexpr (sizeof(C) == 4) {
          u = row_phi(a, i, t, rin, loss);
        } else {
          u = (C)row_phi_d(a, i, (double)t, rin, loss);
        }
        if (!nodot && a.t_out) a.t_out[i] = (double)t;
      }
      us[st][lane] = u;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&b.ready[st]);
  }
  return loss;
}

// ------------------------------------------------------------------ float compute
// FP32 / BF16 / FP8 storage, FP32 vectors: G dot warps and G update warps, each thread
// of a group owning VPT 16-byte column vectors (slot j, vectors j + kk * 32 G).
template <int DT, int VPT, int R, int G>
__global__ void __launch_bounds__((2 * G + 2) * 32, 1) apass_ws_kernel(const ApassKArgs a) {
  constexpr int VEC = Stor<DT>::VEC;
  constexpr int ESZ = Stor<DT>::ESZ;
  constexpr int NP = VEC / 2;
  constexpr int TG = 32 * G;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) WsBars bars;
  __shared__ float red[kWsMaxStages][G][R];
  __shared__ float us[kWsMaxStages][R];
  __shared__ int abort_flag;
  __shared__ double loss_sh;

  if (a.skip && *a.skip) return;
  if (a.executed && blockIdx.x == 0 && threadIdx.x == 0) *a.executed = 1;
  const int ts_slot = timer_begin(a);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nvec = (int)((a.d + VEC - 1) / VEC);
  const uint32_t rowbytes = (uint32_t)(a.ld * ESZ);
  const int S = a.S;
  const uint32_t stage_bytes = (uint32_t)R * rowbytes;
  const int64_t r0 = a.n * (int64_t)blockIdx.x / gridDim.x;
  const int64_t r1 = a.n * (int64_t)(blockIdx.x + 1) / gridDim.x;
  const int nsteps = (int)((r1 - r0 + R - 1) / R);
  const int tail_n = (int)(a.d % VEC);
  const bool nodot = a.mode == MODE_CONST;
  const uint32_t sbase = smem_u32(smem);
  volatile int* abort_v = &abort_flag;
  // group slot j of this thread (dot: tid, update: tid - TG): its vectors j + kk TG exist
  // for kk < nfull, and the ragged last vector (when d is not a multiple of VEC) is kk = tail_kk
  const int jg = tid < TG ? tid : tid - TG;
  const int nfull = jg < nvec ? min(VPT, (nvec - 1 - jg) / TG + 1) : 0;
  const int tail_kk = (tail_n != 0 && (nvec - 1) % TG == jg) ? (nvec - 1) / TG : -1;

  if (tid == 0) {
    ws_init(bars, S, G, G);
    abort_flag = 0;
    loss_sh = 0.0;
  }
  __syncthreads();

  float2 acc[VPT][NP];
  int issued = 0;
  if (warp < G) {
    // ---------------- dot warps: t_i partials
    if (!nodot) {
      const int j = tid;
      const float* p = reinterpret_cast<const float*>(a.p);
      float2 pr[VPT][NP];
#pragma unroll
      for (int kk = 0; kk < VPT; ++kk) {
        const int v = j + kk * TG;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const int64_t e = (int64_t)v * VEC + 2 * q;
          float x0 = 0.f, x1 = 0.f;
          if (v < nvec) {
            if (e < a.d) x0 = p[e];
            if (e + 1 < a.d) x1 = p[e + 1];
            if (DT == NYS_FP8E4M3) {  // A_ij = s_j q_ij: a_i . p = q_i . (s o p)
              if (e < a.d) x0 *= a.col_scale[e];
              if (e + 1 < a.d) x1 *= a.col_scale[e + 1];
            }
          }
          pr[kk][q] = make_float2(x0, x1);
        }
      }
      for (int k = 0; k < nsteps; ++k) {
        const int st = k % S;
        if (!warp_wait(&bars.full[st], (uint32_t)((k / S) & 1))) {
          *abort_v = 1;
          break;
        }
        const int rows_here = (int)min((int64_t)R, r1 - (r0 + (int64_t)k * R));
        const uint32_t sbj = sbase + (uint32_t)st * stage_bytes + (uint32_t)j * 16u;
        float2 dacc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) dacc[r] = make_float2(0.f, 0.f);
        // full stages take the branch-free body; vector kk sits at a compile-time offset
        auto body = [&](auto full) {
#pragma unroll
          for (int kk = 0; kk < VPT; ++kk) {
            if (kk < nfull) {
              const bool tl = kk == tail_kk;
#pragma unroll
              for (int r = 0; r < R; ++r) {
                if (decltype(full)::value || r < rows_here) {
                  uint4 x = lds128(sbj + (uint32_t)r * rowbytes + (uint32_t)(kk * TG * 16));
                  if (tl) mask_tail<DT>(x, tail_n);
#pragma unroll
                  for (int q = 0; q < NP; ++q) dacc[r] = __ffma2_rn(unpack_pair<DT>(x, q), pr[kk][q], dacc[r]);
                }
              }
            }
          }
        };
        if (rows_here == R) body(std::true_type{});
        else body(std::false_type{});
        float sums[R];
#pragma unroll
        for (int r = 0; r < R; ++r) sums[r] = dacc[r].x + dacc[r].y;
        const float tot = warp_sum_rows<R>(sums, lane);
        if ((lane & (32 / R - 1)) == 0) red[st][warp][lane / (32 / R)] = tot;
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.dotted[st]);
      }
    }
  } else if (warp < 2 * G) {
    // ---------------- update warps: acc += sum_r u_r a_r over the stage's rows
    const int j = tid - TG;
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk)
#pragma unroll
      for (int q = 0; q < NP; ++q) acc[kk][q] = make_float2(0.f, 0.f);
    for (int k = 0; k < nsteps; ++k) {
      const int st = k % S;
      const uint32_t ph = (uint32_t)((k / S) & 1);
      if (!warp_wait(&bars.ready[st], ph) || !warp_wait(&bars.full[st], ph)) {
        *abort_v = 1;
        break;
      }
      const int rows_here = (int)min((int64_t)R, r1 - (r0 + (int64_t)k * R));
      const uint32_t sbj = sbase + (uint32_t)st * stage_bytes + (uint32_t)j * 16u;
      float2 u2[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float u = us[st][r];
        u2[r] = make_float2(u, u);
      }
      auto body = [&](auto full) {
#pragma unroll
        for (int kk = 0; kk < VPT; ++kk) {
          if (kk < nfull) {
            const bool tl = kk == tail_kk;
#pragma unroll
            for (int r = 0; r < R; ++r) {
              if (decltype(full)::value || r < rows_here) {
                uint4 x = lds128(sbj + (uint32_t)r * rowbytes + (uint32_t)(kk * TG * 16));
                if (tl) mask_tail<DT>(x, tail_n);
#pragma unroll
                for (int q = 0; q < NP; ++q) acc[kk][q] = __ffma2_rn(unpack_pair<DT>(x, q), u2[r], acc[kk][q]);
              }
            }
          }
        }
      };
      if (rows_here == R) body(std::true_type{});
      else body(std::false_type{});
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.empty[st]);
    }
  } else if (warp == 2 * G) {
    // ---------------- producer
    if (lane == 0) issued = ws_produce(a, bars, smem, nsteps, R, S, rowbytes, r0, r1, abort_v);
  } else {
    // ---------------- finisher
    double l = ws_finish<float, R, G>(a, bars, red, us, nsteps, S, r0, r1, abort_v);
    l = warp_sum(l);
    if (lane == 0) loss_sh = l;
  }

  __syncthreads();
  if (abort_flag) {
    if (warp == 2 * G && lane == 0) {
      // copies still in flight land in this CTA's shared memory: wait for them (bounded)
      for (int k = max(0, issued - S); k < issued; ++k)
        (void)mbar_wait_bounded(&bars.full[k % S], (uint32_t)((k / S) & 1));
      atomicExch(a.status, (int)NYS_ETIMEOUT);
    }
    return;
  }
  if (warp >= G && warp < 2 * G) {
    float* part = reinterpret_cast<float*>(a.partial) + (int64_t)blockIdx.x * a.dpad;
    const int j = tid - TG;
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int v = j + kk * TG;
      if (v < nvec) {
#pragma unroll
        for (int q = 0; q < NP; ++q) *reinterpret_cast<float2*>(part + (int64_t)v * VEC + 2 * q) = acc[kk][q];
      }
    }
  }
  if (tid == 0 && a.loss_part) a.loss_part[blockIdx.x] = loss_sh;
  timer_end(a, ts_slot, DT);
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
      for (int k = 0; k < nsteps; ++k) {
        const int st = k % S;
        if (!warp_wait(&bars.full[st], (uint32_t)((k / S) & 1))) {
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
    for (int k = 0; k < nsteps; ++k) {
      const int st = k % S;
      const uint32_t ph = (uint32_t)((k / S) & 1);
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
