// The warp-specialised fused A-pass as device code: y = A^T phi(A p) with one read of A
// (Table 1's T_mv, the H-matvec of Alg. Nystrom PCG), used by the pass kernels of
// apass_ws.cu.  The roles take a stage offset (`kbase`) so that a kernel running several
// passes could carry the stage ring and its barrier phases on from pass to pass.
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
// Partial sums are written per CTA and summed in a fixed order afterwards, so the
// result is bitwise reproducible from run to run.
#pragma once
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
// Returns the number of stages issued.  `kbase` counts the stages this CTA consumed in
// earlier passes of the same launch, so that ring slot and barrier phase carry on.
__device__ __forceinline__ int ws_produce(const ApassKArgs& a, WsBars& b, unsigned char* smem, int nsteps, int R,
                                          int S, uint32_t rowbytes, int64_t r0, int64_t r1, volatile int* abort_flag,
                                          int kbase = 0) {
  const uint64_t pol = l2_evict_first_policy();  // A is streamed once per pass
  const uint32_t stage_bytes = (uint32_t)R * rowbytes;
  int issued = 0;
  // ring slot and barrier phase of stage kbase + k, advanced without a division per stage
  int st = kbase % S;
  uint32_t ph = (uint32_t)((kbase / S) & 1);
  for (int k = 0; k < nsteps; ++k, st = st + 1 == S ? 0 : st + 1, ph ^= st == 0 ? 1u : 0u) {
    const int kg = kbase + k;
    if (kg >= S && !mbar_wait_bounded(&b.empty[st], ph ^ 1u)) {
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
                                            int nsteps, int S, int64_t r0, int64_t r1, volatile int* abort_flag,
                                            int kbase = 0) {
  const int lane = threadIdx.x & 31;
  const bool nodot = a.mode == MODE_CONST;
  double loss = 0.0;
  int st = kbase % S;
  uint32_t ph = (uint32_t)((kbase / S) & 1);
  for (int k = 0; k < nsteps; ++k, st = st + 1 == S ? 0 : st + 1, ph ^= st == 0 ? 1u : 0u) {
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


// Where the dot warps take p_j (read once per pass into registers): a vector written by an
// earlier launch.
struct PSrcPlain {
  const float* p;
  __device__ __forceinline__ float operator()(int64_t e) const { return p[e]; }
};

// Shared state of the float pass (beside the dynamic-memory stage ring).
template <int R, int G>
struct WsFloatSmem {
  WsBars bars;
  float red[kWsMaxStages][G][R];
  float us[kWsMaxStages][R];
  int abort_flag;
  double loss;
};

// One pass of the float-compute (FP32 / BF16 / FP8 storage) warp-specialised A-pass by
// this CTA over its slab of rows; the CTA's partial of A^T u goes to a.partial.  The
// barriers are initialised and abort_flag is 0 on entry; `kbase` = stages this CTA used
// in earlier passes of the launch.  G dot warps and G update warps, each thread of a
// group owning VPT 16-byte column vectors (slot j, vectors j + kk * 32 G).  Returns false
// if a wait ran out (copies drained, NYS_ETIMEOUT reported).
template <int DT, int VPT, int R, int G, class PSrc>
__device__ __forceinline__ bool ws_pass_float(const ApassKArgs& a, WsFloatSmem<R, G>& sm, unsigned char* smem,
                                              int kbase, const PSrc& psrc) {
  constexpr int VEC = Stor<DT>::VEC;
  constexpr int ESZ = Stor<DT>::ESZ;
  constexpr int NP = VEC / 2;
  constexpr int TG = 32 * G;
  WsBars& bars = sm.bars;
  const int ts_slot = timer_begin(a);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n_o = a.n, d_o = a.d, ld_o = a.ld;
  const int S_o = a.S;
  const int nvec = (int)((d_o + VEC - 1) / VEC);
  const uint32_t rowbytes = (uint32_t)(ld_o * ESZ);
  const int S = S_o;
  const uint32_t stage_bytes = (uint32_t)R * rowbytes;
  const int64_t r0 = a.row_split ? a.row_split[blockIdx.x] : n_o * (int64_t)blockIdx.x / gridDim.x;
  const int64_t r1 = a.row_split ? a.row_split[blockIdx.x + 1] : n_o * (int64_t)(blockIdx.x + 1) / gridDim.x;
  if (a.cta_time && tid == 0) a.cta_time[2 * blockIdx.x] = gtimer();
  const int nsteps = (int)((r1 - r0 + R - 1) / R);
  const int tail_n = (int)(d_o % VEC);
  const bool nodot = a.mode == MODE_CONST;
  const uint32_t sbase = smem_u32(smem);
  volatile int* abort_v = &sm.abort_flag;
  // group slot j of this thread (dot: tid, update: tid - TG): its vectors j + kk TG exist
  // for kk < nfull, and the ragged last vector (when d is not a multiple of VEC) is kk = tail_kk
  const int jg = tid < TG ? tid : tid - TG;
  const int nfull = jg < nvec ? min(VPT, (nvec - 1 - jg) / TG + 1) : 0;
  const int tail_kk = (tail_n != 0 && (nvec - 1) % TG == jg) ? (nvec - 1) / TG : -1;

  float2 acc[VPT][NP];
  int issued = 0;
  if (warp < G) {
    // ---------------- dot warps: t_i partials
    if (!nodot) {
      const int j = tid;
      float2 pr[VPT][NP];
#pragma unroll
      for (int kk = 0; kk < VPT; ++kk) {
        const int v = j + kk * TG;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const int64_t e = (int64_t)v * VEC + 2 * q;
          float x0 = 0.f, x1 = 0.f;
          if (v < nvec) {
            if (e < d_o) x0 = psrc(e);
            if (e + 1 < d_o) x1 = psrc(e + 1);
            if (DT == NYS_FP8E4M3) {  // A_ij = s_j q_ij: a_i . p = q_i . (s o p)
              if (e < d_o) x0 *= a.col_scale[e];
              if (e + 1 < d_o) x1 *= a.col_scale[e + 1];
            }
          }
          pr[kk][q] = make_float2(x0, x1);
        }
      }
      int st = kbase % S;
      uint32_t ph = (uint32_t)((kbase / S) & 1);
      for (int k = 0; k < nsteps; ++k, st = st + 1 == S ? 0 : st + 1, ph ^= st == 0 ? 1u : 0u) {
        if (!warp_wait(&bars.full[st], ph)) {
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
        if ((lane & (32 / R - 1)) == 0) sm.red[st][warp][lane / (32 / R)] = tot;
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
    int st = kbase % S;
    uint32_t ph = (uint32_t)((kbase / S) & 1);
    for (int k = 0; k < nsteps; ++k, st = st + 1 == S ? 0 : st + 1, ph ^= st == 0 ? 1u : 0u) {
      if (!warp_wait(&bars.ready[st], ph) || !warp_wait(&bars.full[st], ph)) {
        *abort_v = 1;
        break;
      }
      const int rows_here = (int)min((int64_t)R, r1 - (r0 + (int64_t)k * R));
      const uint32_t sbj = sbase + (uint32_t)st * stage_bytes + (uint32_t)j * 16u;
      float2 u2[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float u = sm.us[st][r];
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
    if (lane == 0) issued = ws_produce(a, bars, smem, nsteps, R, S, rowbytes, r0, r1, abort_v, kbase);
  } else {
    // ---------------- finisher
    double l = ws_finish<float, R, G>(a, bars, sm.red, sm.us, nsteps, S, r0, r1, abort_v, kbase);
    l = warp_sum(l);
    if (lane == 0) sm.loss = l;
  }

  __syncthreads();
  if (sm.abort_flag) {
    if (warp == 2 * G && lane == 0) {
      // copies still in flight land in this CTA's shared memory: wait for them (bounded)
      for (int k = max(0, issued - S); k < issued; ++k)
        (void)mbar_wait_bounded(&bars.full[(kbase + k) % S], (uint32_t)(((kbase + k) / S) & 1));
      atomicExch(a.status, (int)NYS_ETIMEOUT);
    }
    return false;
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
  if (tid == 0 && a.loss_part) a.loss_part[blockIdx.x] = sm.loss;
  timer_end(a, ts_slot, DT);
  if (a.cta_time) {
    __syncthreads();
    if (tid == 0) a.cta_time[2 * blockIdx.x + 1] = gtimer();
  }
  return true;
}

}  // namespace nys
