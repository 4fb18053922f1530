// Fused A-pass: y = A^T phi(A p) with ONE read of A from HBM.
//
// This is the T_mv of the paper's complexity model (Table 1) and the H-matvec
// v = (H + rho I) p of Alg. Nystrom PCG with H = A^T D A (Eq. ADMMSubProb; D from
// Sec. 3.2 for the logistic loss).  Its other modes build the ADMM right-hand
// sides A^T b (lasso) and A^T (w t + b01 - sigma(t)) (logistic, Sec. 3.2) and the
// residual A^T (A x - b) for the objective / KKT measures (Eq. 2, Eq. 31).
//
// GB300 design (one CTA of 512 threads per SM, persistent over a contiguous
// slab of rows):
//   * rows are streamed HBM -> shared memory by 1-D TMA bulk copies
//     (cp.async.bulk + mbarrier transaction counts), S stages of R rows each,
//     S-1 stages in flight while the CTA computes on the current one;
//   * every thread OWNS a fixed set of 16-byte column vectors, so p and the
//     CTA's partial of A^T phi(.) live in registers and the rank-1 update
//     y += a_i u_i needs no atomics;
//   * the row dot products t_i = a_i . p are reduced with warp shuffles plus one
//     __syncthreads_or per step (R rows), which also carries the bounded-wait
//     status;
//   * per-CTA partials go to a [grid x d] buffer that a second kernel sums in a
//     fixed order (deterministic, run-to-run bitwise identical) and adds rho p.
#include "apass_common.cuh"

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace nys {

template <int DT, int VPT>
__global__ void __launch_bounds__(kApassThreads, 1) apass_kernel(const ApassKArgs a) {
  using C = typename Stor<DT>::C;
  constexpr int VEC = Stor<DT>::VEC;
  constexpr int ESZ = Stor<DT>::ESZ;
  constexpr int T = kApassThreads;
  constexpr int NW = T / 32;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kMaxStages];
  __shared__ C red[2][NW][kRMax];

  if (a.skip && *a.skip) return;
  if (a.executed && blockIdx.x == 0 && threadIdx.x == 0) *a.executed = 1;
  const int ts_slot = timer_begin(a);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nvec = (a.d + VEC - 1) / VEC;
  const int64_t rowbytes = a.ld * ESZ;
  const int R = a.R, S = a.S;
  const int64_t stage_bytes = (int64_t)R * rowbytes;
  const int64_t r0 = a.n * (int64_t)blockIdx.x / gridDim.x;
  const int64_t r1 = a.n * (int64_t)(blockIdx.x + 1) / gridDim.x;
  const int nsteps = (int)((r1 - r0 + R - 1) / R);
  const int64_t tail_vec = a.d / VEC;           // vector holding the ragged end (if any)
  const int tail_n = (int)(a.d % VEC);          // valid elements in it

  const C* p = reinterpret_cast<const C*>(a.p);
  C pr[VPT][VEC];
  C acc[VPT][VEC];
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int64_t v = tid + (int64_t)k * T;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int64_t j = v * VEC + e;
      pr[k][e] = (a.mode != MODE_CONST && v < nvec && j < a.d) ? p[j] : C(0);
      acc[k][e] = C(0);
    }
  }

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const uint64_t pol = l2_evict_first_policy();  // A is streamed once per pass
  auto issue = [&](int step) {
    const int stage = step % S;
    const int64_t row = r0 + (int64_t)step * R;
    const int rows = (int)min((int64_t)R, r1 - row);
    const uint32_t bytes = (uint32_t)(rows * rowbytes);
    mbar_arrive_expect_tx(&bars[stage], bytes);
    tma_load_1d_hint(smem + stage * stage_bytes, a.A + row * rowbytes, bytes, &bars[stage], pol);
  };
  int issued = 0;
  if (tid == 0) {
    for (int st = 0; st < S && st < nsteps; ++st) issue(st);
    issued = min(S, nsteps);
  }

  double loss = 0.0;
  bool aborted = false;
  int k = 0;
  for (; k < nsteps; ++k) {
    const int stage = k % S;
    const unsigned char* sb = smem + stage * stage_bytes;
    const int64_t row0 = r0 + (int64_t)k * R;
    const int rows_here = (int)min((int64_t)R, r1 - row0);
    const bool ok = mbar_wait_bounded(&bars[stage], (uint32_t)((k / S) & 1));

    C dot[kRMax];
#pragma unroll
    for (int r = 0; r < kRMax; ++r) dot[r] = C(0);
    if (ok && a.mode != MODE_CONST) {
#pragma unroll
      for (int r = 0; r < kRMax; ++r) {
        if (r < rows_here) {
#pragma unroll
          for (int kk = 0; kk < VPT; ++kk) {
            const int64_t v = tid + (int64_t)kk * T;
            if (v < nvec) {
              const uint4 raw = *reinterpret_cast<const uint4*>(sb + r * rowbytes + v * 16);
              C val[VEC];
              unpack16<DT>(raw, val);
              if (v == tail_vec) {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                  if (e >= tail_n) val[e] = C(0);
              }
#pragma unroll
              for (int e = 0; e < VEC; ++e) dot[r] = fma(val[e], pr[kk][e], dot[r]);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kRMax; ++r) {
        const C s = warp_sum(dot[r]);
        if (lane == 0) red[k & 1][warp][r] = s;
      }
    }
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    // Stage (k-1) % S has been fully consumed by every thread: refill it.
    if (tid == 0 && k >= 1 && (k - 1 + S) < nsteps) {
      issue(k - 1 + S);
      ++issued;
    }
    C u[kRMax];
#pragma unroll
    for (int r = 0; r < kRMax; ++r) {
      u[r] = C(0);
      if (r < rows_here) {
        const int64_t i = row0 + r;
        if (a.mode == MODE_CONST) {
          u[r] = (C)a.b[i];
        } else {
          C t = C(0);
#pragma unroll
          for (int w = 0; w < NW; ++w) t += red[k & 1][w][r];
          if (a.mode == MODE_ID) {
            u[r] = t;
          } else if (a.mode == MODE_DIAG) {
            u[r] = (C)(a.D[i] * (double)t);
          } else if (a.mode == MODE_RESID) {
            const double rr = (double)t - a.b[i];
            u[r] = (C)rr;
            if (tid == 0) loss += 0.5 * rr * rr;
          } else if (a.mode == MODE_LGRAD) {
            const double td = (double)t;
            const double sg = sigmoid_d(td);
            const double b01 = 0.5 * (1.0 + a.b[i]);
            u[r] = (C)(sg - b01);
            if (tid == 0) loss += fmax(td, 0.0) + log1p(exp(-fabs(td))) - b01 * td;
          } else {  // MODE_LOGIT
            const double td = (double)t;
            const double sg = sigmoid_d(td);
            const double wv = sg * (1.0 - sg);
            const double b01 = 0.5 * (1.0 + a.b[i]);
            u[r] = (C)(wv * td + b01 - sg);
            if (tid == 0) {
              if (a.D_out) a.D_out[i] = wv;
              loss += fmax(td, 0.0) + log1p(exp(-fabs(td))) - b01 * td;
            }
          }
          if (tid == 0 && a.t_out) a.t_out[i] = (double)t;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kRMax; ++r) {
      if (r < rows_here) {
#pragma unroll
        for (int kk = 0; kk < VPT; ++kk) {
          const int64_t v = tid + (int64_t)kk * T;
          if (v < nvec) {
            const uint4 raw = *reinterpret_cast<const uint4*>(sb + r * rowbytes + v * 16);
            C val[VEC];
            unpack16<DT>(raw, val);
            if (v == tail_vec) {
#pragma unroll
              for (int e = 0; e < VEC; ++e)
                if (e >= tail_n) val[e] = C(0);
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[kk][e] = fma(val[e], u[r], acc[kk][e]);
          }
        }
      }
    }
  }

  if (aborted) {
    // Drain the copies still in flight into this CTA's shared memory (bounded), then report.
    if (tid == 0) {
      for (int st = k; st < issued; ++st) (void)mbar_wait_bounded(&bars[st % S], (uint32_t)((st / S) & 1));
      atomicExch(a.status, (int)NYS_ETIMEOUT);
    }
    return;
  }

  C* part = reinterpret_cast<C*>(a.partial) + (int64_t)blockIdx.x * a.dpad;
#pragma unroll
  for (int kk = 0; kk < VPT; ++kk) {
    const int64_t v = tid + (int64_t)kk * T;
    if (v < nvec) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) part[v * VEC + e] = acc[kk][e];
    }
  }
  if (tid == 0 && a.loss_part) a.loss_part[blockIdx.x] = loss;
  timer_end(a, ts_slot, DT);
}

// Float-compute variant (FP32 / BF16 storage).  Same streaming scheme, tuned for
// the instruction budget of a bandwidth-bound pass:
//   * the R rows of a stage are loaded from shared memory ONCE into registers (raw
//     16-byte vectors) and reused by both the dot product and the rank-1 update, so a
//     stage can be refilled by TMA as soon as every thread has loaded it (all S stages
//     stay in flight);
//   * dot products and updates use the packed FP32 FMA (two lanes per instruction);
//   * the row sums are finished by one warp per row (two barriers per step instead of
//     every thread re-reading all warp partials).
//
// Float-compute kernel.  Per step of R rows: every thread loads its slice of the
// stage from shared memory ONCE into registers (raw 16-byte vectors), forms its
// partial row dots with packed FP32 FMAs, and after the first barrier the stage is
// refilled by TMA at once (all S stages stay in flight); warps 0..R-1 finish the row
// sums and apply phi; after the second barrier every thread applies the rank-R
// update from the same registers.
// ONEBAR selects the finish of a step in the H-matvec modes: false = warps 0..R-1 finish
// one row sum each and a second barrier publishes them; true = every warp finishes all R
// row sums itself (one barrier per step, R warp reductions per warp).  A variant that
// re-read the stage from shared memory for the update instead of holding it in
// registers (refill one step later) measured slower in every configuration.
template <int DT, int VPT, int R, int T, bool ONEBAR>
__global__ void __launch_bounds__(T, 1) apass_f_kernel(const ApassKArgs a) {
  constexpr int VEC = Stor<DT>::VEC;
  constexpr int ESZ = Stor<DT>::ESZ;
  constexpr int NP = VEC / 2;
  constexpr int NW = T / 32;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kMaxStages];
  __shared__ float red[2][NW][R];
  __shared__ float us[2][R];
  __shared__ double lsh[NW];

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
  const int tail_vec = (int)(a.d / VEC);
  const int tail_n = (int)(a.d % VEC);
  const bool nodot = a.mode == MODE_CONST;
  const uint32_t sbase = smem_u32(smem);

  const float* p = reinterpret_cast<const float*>(a.p);
  float2 pr[VPT][NP], acc[VPT][NP];
#pragma unroll
  for (int kk = 0; kk < VPT; ++kk) {
    const int64_t v = tid + (int64_t)kk * T;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const int64_t j = v * VEC + 2 * q;
      float x0 = 0.f, x1 = 0.f;
      if (!nodot && v < nvec) {
        if (j < a.d) x0 = p[j];
        if (j + 1 < a.d) x1 = p[j + 1];
        if (DT == NYS_FP8E4M3) {  // A_ij = s_j q_ij: a_i . p = q_i . (s o p)
          if (j < a.d) x0 *= a.col_scale[j];
          if (j + 1 < a.d) x1 *= a.col_scale[j + 1];
        }
      }
      pr[kk][q] = make_float2(x0, x1);
      acc[kk][q] = make_float2(0.f, 0.f);
    }
  }

  if (tid == 0) {
    for (int st = 0; st < S; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const uint64_t pol = l2_evict_first_policy();  // A is streamed once per pass
  auto issue = [&](int step) {
    const int stage = step % S;
    const int64_t row = r0 + (int64_t)step * R;
    const int rows = (int)min((int64_t)R, r1 - row);
    const uint32_t bytes = (uint32_t)rows * rowbytes;
    mbar_arrive_expect_tx(&bars[stage], bytes);
    tma_load_1d_hint(smem + (size_t)stage * stage_bytes, a.A + row * (int64_t)rowbytes, bytes, &bars[stage], pol);
  };
  int issued = 0;
  if (tid == 0) {
    for (int st = 0; st < S && st < nsteps; ++st) issue(st);
    issued = min(S, nsteps);
  }

  double loss = 0.0;
  bool aborted = false;
  int k = 0;
  for (; k < nsteps; ++k) {
    const int stage = k % S;
    const uint32_t sb = sbase + (uint32_t)stage * stage_bytes;
    const int rows_here = (int)min((int64_t)R, r1 - (r0 + (int64_t)k * R));
    // per-row mode inputs: warp r (two-barrier finish) or every warp (one-barrier
    // finish) needs those of its rows; load them before waiting for the stage
    double rin[ONEBAR ? R : 1];
    if (ONEBAR && (a.mode == MODE_ID || a.mode == MODE_DIAG)) {
#pragma unroll
      for (int r = 0; r < (ONEBAR ? R : 1); ++r)
        rin[r] = r < rows_here ? row_input(a, r0 + (int64_t)k * R + r) : 0.0;
    } else {
      rin[0] = (warp < rows_here && lane == 0) ? row_input(a, r0 + (int64_t)k * R + warp) : 0.0;
    }
    const bool ok = mbar_wait_bounded(&bars[stage], (uint32_t)((k / S) & 1));

    uint4 raw[R][VPT];
    float2 dacc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dacc[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int v = tid + kk * T;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        if (ok && v < nvec && r < rows_here) x = lds128(sb + (uint32_t)r * rowbytes + (uint32_t)v * 16u);
        if (v == tail_vec) mask_tail<DT>(x, tail_n);
        raw[r][kk] = x;
        if (!nodot) {
#pragma unroll
          for (int q = 0; q < NP; ++q) dacc[r] = __ffma2_rn(unpack_pair<DT>(x, q), pr[kk][q], dacc[r]);
        }
      }
    }
    if (!nodot) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float sdot = warp_sum(dacc[r].x + dacc[r].y);
        if (lane == 0) red[k & 1][warp][r] = sdot;
      }
    }
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    // every thread holds its slice of this stage in registers: refill it now
    if (tid == 0 && k + S < nsteps) {
      issue(k + S);
      ++issued;
    }
    float2 u2[R];
    // ONEBAR (H-matvec modes): the per-warp finish below removes the second barrier
    // (FP32 storage, 512 threads: measured 5.8 -> 7.0 TB/s).  The host picks ONEBAR per
    // storage type and block size (register budget of raw[R][VPT]).
    if (ONEBAR && (a.mode == MODE_ID || a.mode == MODE_DIAG)) {
      // every warp finishes all R row sums itself (lanes 0..NW-1 hold
      // the warp partials of each row; a butterfly leaves the sum in every lane), so no
      // second barrier is needed.  Warp r's lane 0 writes row r's side outputs.
      float t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = warp_sum(lane < NW ? red[k & 1][lane][r] : 0.f);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float u = 0.f;
        if (r < rows_here) {
          const int64_t i = r0 + (int64_t)k * R + r;
          u = a.mode == MODE_ID ? t[r] : (float)(rin[r] * (double)t[r]);
          if (warp == r && lane == 0 && a.t_out) a.t_out[i] = (double)t[r];
        }
        u2[r] = make_float2(u, u);
      }
    } else {
      if (warp < R) {
        float t = 0.f;
        if (!nodot) t = warp_sum(lane < NW ? red[k & 1][lane][warp] : 0.f);
        if (lane == 0) {
          float u = 0.f;
          if (warp < rows_here) {
            const int64_t i = r0 + (int64_t)k * R + warp;
            u = row_phi(a, i, t, rin[0], loss);
            if (!nodot && a.t_out) a.t_out[i] = (double)t;
          }
          us[k & 1][warp] = u;
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float u = us[k & 1][r];
        u2[r] = make_float2(u, u);
      }
    }
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
#pragma unroll
      for (int q = 0; q < NP; ++q) {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[kk][q] = __ffma2_rn(unpack_pair<DT>(raw[r][kk], q), u2[r], acc[kk][q]);
      }
    }
  }

  if (aborted) {
    if (tid == 0) {
      for (int st = k; st < issued; ++st) (void)mbar_wait_bounded(&bars[st % S], (uint32_t)((st / S) & 1));
      atomicExch(a.status, (int)NYS_ETIMEOUT);
    }
    return;
  }

  float* part = reinterpret_cast<float*>(a.partial) + (int64_t)blockIdx.x * a.dpad;
#pragma unroll
  for (int kk = 0; kk < VPT; ++kk) {
    const int64_t v = tid + (int64_t)kk * T;
    if (v < nvec) {
#pragma unroll
      for (int q = 0; q < NP; ++q) *reinterpret_cast<float2*>(part + v * VEC + 2 * q) = acc[kk][q];
    }
  }
  if (a.loss_part) {
    if (lane == 0) lsh[warp] = loss;
    __syncthreads();
    if (tid == 0) {
      double sl = 0.0;
      for (int w = 0; w < NW; ++w) sl += lsh[w];
      a.loss_part[blockIdx.x] = sl;
    }
  }
  timer_end(a, ts_slot, DT);
}

// y_j = sum_g partial[g][j] (fixed order) + rho p_j; optional per-block partials of p^T y.
template <typename C>
__global__ void __launch_bounds__(kVecThreads) apass_reduce_kernel(const C* __restrict__ partial, int G,
                                                                   int64_t d, int64_t dpad, C rho,
                                                                   const C* __restrict__ p, C* __restrict__ y,
                                                                   double* dot_part, const int* skip,
                                                                   const float* __restrict__ cscale) {
  if (skip && *skip) return;
  __shared__ double sh[kVecThreads / 32];
  double dacc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    // fixed order over the CTAs' partials (increasing g)
    C s = sum_strided_fixed<false>(partial, G, dpad, j, C(0));
    if (cscale) s *= (C)cscale[j];  // FP8: sum_i q_ij u_i -> sum_i A_ij u_i
    const C pj = p ? p[j] : C(0);
    const C yj = fma(rho, pj, s);
    y[j] = yj;
    dacc += (double)pj * (double)yj;
  }
  if (dot_part) {
    const double t = block_sum_t0<kVecThreads>(dacc, sh);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = t;
  }
}

// Blocks of the vector kernels over d elements: one element per thread, at most 4 blocks
// per SM (measured: spreading a 10,000-element vector over 4x more blocks made the
// ADMM iteration slower, 78 -> 104 us of small-kernel time).
int reduce_blocks(int64_t d) {
  const int64_t b = (d + kVecThreads - 1) / kVecThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4 * (int64_t)sm_count()));
}

static int vpt_bucket(int64_t nvec, int threads = kApassThreads) {
  const int64_t need = (nvec + threads - 1) / threads;
  static const int buckets[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
  for (int b : buckets)
    if (need <= b) return b;
  return -1;
}

// Autotuned rows-per-stage, keyed by (device, dtype, columns per thread, row bytes): a
// choice timed on one GPU is not applied to another.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int64_t>, int> g_tuned_rows;

void apass_set_tuned_rows(const nys_matrix* A, int rows) {
  const int64_t esz = (int64_t)dtype_size(A->dtype);
  const int vb = vpt_bucket((A->d + (16 / esz) - 1) / (16 / esz));
  const int vpt = vb < 0 ? 99 : vb;   // the key apass_plan looks up
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (rows <= 0) g_tuned_rows.erase({dev, A->dtype, vpt, A->ld * esz});
  else g_tuned_rows[{dev, A->dtype, vpt, A->ld * esz}] = rows;
}

// Calibrated row splits of the warp-specialised float pass, keyed by (device, dtype, row
// bytes, rows, grid, rows per stage); device arrays of grid + 1 boundaries, owned here.
static std::map<std::tuple<int, int, int64_t, int64_t, int, int>, int64_t*> g_row_split;
static thread_local unsigned long long* g_cta_time = nullptr;   // set only while this thread calibrates

static const int64_t* row_split_lookup(int dtype, int64_t rowbytes, int64_t n, int grid, int R) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_row_split.find({dev, dtype, rowbytes, n, grid, R});
  return it == g_row_split.end() ? nullptr : it->second;
}

static cudaError_t row_split_store(int dtype, int64_t rowbytes, int64_t n, int grid, int R, const int64_t* host,
                                   cudaStream_t st) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const auto key = std::make_tuple(dev, dtype, rowbytes, n, grid, R);
  auto it = g_row_split.find(key);
  if (!host) {
    if (it != g_row_split.end()) {
      NYS_CUDA_TRY(cudaStreamSynchronize(st));
      NYS_CUDA_TRY(cudaFree(it->second));
      g_row_split.erase(it);
    }
    return cudaSuccess;
  }
  int64_t* buf = it == g_row_split.end() ? nullptr : it->second;
  if (!buf) {
    NYS_CUDA_TRY(cudaMalloc(&buf, (size_t)(grid + 1) * sizeof(int64_t)));
    g_row_split[key] = buf;
  }
  NYS_CUDA_TRY(cudaMemcpyAsync(buf, host, (size_t)(grid + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  return cudaStreamSynchronize(st);
}

static int tuned_rows(int dtype, int vpt, int64_t rowbytes) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_rows.find({dev, dtype, vpt, rowbytes});
  return it == g_tuned_rows.end() ? 0 : it->second;
}

// Float-path CTA size and vectors per thread.  BF16: where 512 threads would need 3
// vectors per thread but 640 need 2, the 640-thread CTA (R = 4) is used instead
// (d = 10,000 BF16, 100,000 rows: 4.03 -> 4.53 TB/s measured).  Tuning override:
// NYS_APASS_THREADS (512 or 640; 640 only where it needs <= 4 vectors per thread).
static void float_layout(const nys_matrix* A, int64_t nvec, int* threads, int* vpt) {
  *threads = kApassThreads;
  *vpt = vpt_bucket(nvec);
  int want = 0;
  if (A->dtype == NYS_BF16 && *vpt == 3 && vpt_bucket(nvec, kApassThreadsWide) == 2) want = kApassThreadsWide;
  if (const char* env = std::getenv("NYS_APASS_THREADS")) want = std::atoi(env);
  if (want == kApassThreadsWide && vpt_bucket(nvec, want) > 0 && vpt_bucket(nvec, want) <= 4) {
    *threads = want;
    *vpt = vpt_bucket(nvec, want);
  }
}

// Rows per step the float kernel is instantiated for at this many vectors per thread
// (register budget of raw[R][VPT]).
static bool float_rows_ok(int r, int vpt) { return r == 1 || (r == 2 && vpt <= 6) || (r == 4 && vpt <= 3); }

// Warp-specialised pass: used for wide rows, where the classic step's per-row block
// reductions dominate (NYS_APASS_WS = 0 / 1 overrides the choice).
static bool ws_wanted(const nys_matrix* A) {
  if (const char* env = std::getenv("NYS_APASS_WS")) return std::atoi(env) != 0;
  const int64_t rowbytes = A->ld * (int64_t)dtype_size(A->dtype);
  if (A->dtype == NYS_F64) return A->d >= 2048;
  return rowbytes >= 4096;
}

// Stages of the warp-specialised ring for R rows per stage (0 if fewer than two fit).
static int ws_stages(int64_t rowbytes, int R) {
  return (int)std::min<int64_t>(12, kSmemBudget / (R * rowbytes));
}

// Rows-per-stage values the kernels support for this matrix (float path: bounded by
// the register budget of the raw vectors; all: at least two stages must fit; the
// warp-specialised pass: 1, 2 or 4 rows with at least three stages, or two for 1 row).
int apass_row_candidates(const nys_matrix* A, int* out) {
  const int64_t esz = (int64_t)dtype_size(A->dtype);
  const int64_t nvec = (A->d + (16 / esz) - 1) / (16 / esz);
  const int64_t rowbytes = A->ld * esz;
  int n = 0;
  int wthreads = 0, wvpt = 0;
  if (ws_wanted(A) && apass_ws_layout(A->dtype, A->d, &wthreads, &wvpt)) {
    for (int r : {1, 2, 4}) {
      if (A->dtype == NYS_F64 && r == 4) continue;
      const int S = ws_stages(rowbytes, r);
      if (S >= (r == 1 ? 2 : 3)) out[n++] = r;
    }
    return n;
  }
  int threads = kApassThreads, vpt = vpt_bucket(nvec);
  if (A->dtype != NYS_F64) float_layout(A, nvec, &threads, &vpt);
  for (int r : {1, 2, 4}) {
    if (2 * r * rowbytes > kSmemBudget) continue;
    if (A->dtype != NYS_F64 && !float_rows_ok(r, vpt)) continue;
    out[n++] = r;
  }
  return n;
}

bool apass_plan(const nys_matrix* A, ApassPlan* plan) {
  const int64_t esz = (int64_t)dtype_size(A->dtype);
  const int vec = (int)(16 / esz);
  const int64_t nvec = (A->d + vec - 1) / vec;
  const int vkey = vpt_bucket(nvec);  // tuning key: vectors per thread at 512 threads
  const int64_t rowbytes = A->ld * esz;
  int wthreads = 0, wvpt = 0;
  if (ws_wanted(A) && apass_ws_layout(A->dtype, A->d, &wthreads, &wvpt)) {
    // warp-specialised: 2 rows per stage by default (1 for rows over 64 KB, 4 under 8 KB)
    int R = rowbytes > 64 * 1024 ? 1 : (rowbytes < 8 * 1024 ? 4 : 2);
    if (A->dtype == NYS_F64 && R > 2) R = 2;
    if (const int tr = tuned_rows(A->dtype, vkey < 0 ? 99 : vkey, rowbytes)) R = tr;
    if (R != 1 && R != 2 && R != 4) R = 2;
    if (A->dtype == NYS_F64 && R > 2) R = 2;
    if (const char* env = std::getenv("NYS_APASS_ROWS")) {
      const int r = std::atoi(env);
      if (r == 1 || r == 2 || (r == 4 && A->dtype != NYS_F64)) R = r;
    }
    while (R > 1 && ws_stages(rowbytes, R) < 3) R /= 2;
    const int S = ws_stages(rowbytes, R);
    if (S >= 2) {
      plan->ws = true;
      plan->rows_per_step = R;
      plan->stages = S;
      plan->threads = wthreads;
      plan->vpt = wvpt;
      plan->onebar = false;
      plan->smem = (size_t)S * R * rowbytes;
      plan->dpad = nvec * vec;
      const int64_t steps_total = (A->n + R - 1) / R;
      plan->grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(), steps_total));
      plan->fused = true;
      return true;
    }
  }
  if (vkey < 0) return false;
  if (A->dtype == NYS_F64 && vkey > 12) return false;
  int vpt = vkey;
  int R = (int)std::max<int64_t>(1, std::min<int64_t>(kRMax, (48 * 1024) / rowbytes));
  if (A->dtype == NYS_F64) {
    if (const int tr = tuned_rows(A->dtype, vkey, rowbytes)) R = tr;
  }
  int threads = kApassThreads;
  bool onebar = false;
  if (A->dtype != NYS_F64) {
    float_layout(A, nvec, &threads, &vpt);
    // float path: R is a template parameter bounded by the register budget of raw[R][VPT]
    R = vpt <= 3 ? 4 : (vpt <= 6 ? 2 : 1);
    if (const int tr = tuned_rows(A->dtype, vkey, rowbytes)) R = tr;
    // FP32: one barrier per step (every warp finishes the R row sums itself); BF16: two
    // barriers (its raw registers leave no room for R row sums in every warp: measured
    // 4.0 -> 3.1 TB/s with one barrier).  Tuning overrides: NYS_APASS_ROWS (rows per
    // stage; kept only if the instantiation exists for this width), NYS_APASS_ONEBAR (0/1).
    onebar = A->dtype == NYS_F32;
    if (const char* env = std::getenv("NYS_APASS_ROWS")) {
      const int r = std::atoi(env);
      if (float_rows_ok(r, vpt)) R = r;
    }
    if (const char* env = std::getenv("NYS_APASS_ONEBAR")) onebar = std::atoi(env) != 0;
    if (!float_rows_ok(R, vpt)) R = 1;
    while (R > 1 && 2 * R * rowbytes > kSmemBudget) R /= 2;
  }
  int S = (int)std::min<int64_t>(kMaxStages, kSmemBudget / (R * rowbytes));
  if (S < 2) {
    R = 1;
    S = (int)std::min<int64_t>(kMaxStages, kSmemBudget / rowbytes);
  }
  if (S < 2) return false;
  plan->ws = false;
  plan->rows_per_step = R;
  plan->stages = S;
  plan->threads = threads;
  plan->vpt = vpt;
  plan->onebar = onebar;
  plan->smem = (size_t)S * R * rowbytes;
  plan->dpad = nvec * vec;
  const int64_t steps_total = (A->n + R - 1) / R;
  plan->grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(), steps_total));
  plan->fused = true;
  return true;
}

size_t apass_partial_bytes(const nys_matrix* A, const ApassPlan& plan) {
  const size_t csz = compute_is_f64(A->dtype) ? 8 : 4;
  return (size_t)plan.grid * plan.dpad * csz;
}

static thread_local bool g_prepare_only = false;

template <int DT, int VPT>
static cudaError_t launch_vpt(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st) {
  auto fn = apass_kernel<DT, VPT>;
  NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)fn, kSmemBudget));
  if (g_prepare_only) return cudaSuccess;
  count_launch();
  fn<<<plan.grid, kApassThreads, plan.smem, st>>>(k);
  return cudaGetLastError();
}

template <int DT, int VPT, int R, int T, bool OB>
static cudaError_t launch_f(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st) {
  auto fn = apass_f_kernel<DT, VPT, R, T, OB>;
  NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)fn, kSmemBudget));
  if (g_prepare_only) return cudaSuccess;
  count_launch();
  fn<<<plan.grid, T, plan.smem, st>>>(k);
  return cudaGetLastError();
}

template <int DT, int VPT, int R, int T>
static cudaError_t launch_fo(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st) {
  if (plan.onebar) return launch_f<DT, VPT, R, T, true>(k, plan, st);
  return launch_f<DT, VPT, R, T, false>(k, plan, st);
}

template <int DT, int VPT, int T>
static cudaError_t launch_fr(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st) {
  switch (plan.rows_per_step) {
    case 4: if constexpr (VPT <= 3) return launch_fo<DT, VPT, 4, T>(k, plan, st); break;
    case 2: if constexpr (VPT <= 6) return launch_fo<DT, VPT, 2, T>(k, plan, st); break;
    case 1: return launch_fo<DT, VPT, 1, T>(k, plan, st);
    default: break;
  }
  return cudaErrorInvalidValue;
}

template <int DT>
static cudaError_t launch_float(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st) {
  if (plan.threads == kApassThreadsWide) {
    switch (plan.vpt) {
      case 1: return launch_fr<DT, 1, kApassThreadsWide>(k, plan, st);
      case 2: return launch_fr<DT, 2, kApassThreadsWide>(k, plan, st);
      case 3: return launch_fr<DT, 3, kApassThreadsWide>(k, plan, st);
      case 4: return launch_fr<DT, 4, kApassThreadsWide>(k, plan, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (plan.threads != kApassThreads) return cudaErrorInvalidValue;
  switch (plan.vpt) {
    case 1: return launch_fr<DT, 1, kApassThreads>(k, plan, st);
    case 2: return launch_fr<DT, 2, kApassThreads>(k, plan, st);
    case 3: return launch_fr<DT, 3, kApassThreads>(k, plan, st);
    case 4: return launch_fr<DT, 4, kApassThreads>(k, plan, st);
    case 5: return launch_fr<DT, 5, kApassThreads>(k, plan, st);
    case 6: return launch_fr<DT, 6, kApassThreads>(k, plan, st);
    case 8: return launch_fr<DT, 8, kApassThreads>(k, plan, st);
    case 10: return launch_fr<DT, 10, kApassThreads>(k, plan, st);
    case 12: return launch_fr<DT, 12, kApassThreads>(k, plan, st);
    case 16: return launch_fr<DT, 16, kApassThreads>(k, plan, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int DT>
static cudaError_t launch_dt(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st) {
  constexpr int VEC = Stor<DT>::VEC;
  const int64_t nvec = (k.d + VEC - 1) / VEC;
  switch (vpt_bucket(nvec)) {
    case 1: return launch_vpt<DT, 1>(k, plan, st);
    case 2: return launch_vpt<DT, 2>(k, plan, st);
    case 3: return launch_vpt<DT, 3>(k, plan, st);
    case 4: return launch_vpt<DT, 4>(k, plan, st);
    case 5: return launch_vpt<DT, 5>(k, plan, st);
    case 6: return launch_vpt<DT, 6>(k, plan, st);
    case 8: return launch_vpt<DT, 8>(k, plan, st);
    case 10: return launch_vpt<DT, 10>(k, plan, st);
    case 12: return launch_vpt<DT, 12>(k, plan, st);
    case 16:
      if constexpr (DT != NYS_F64) return launch_vpt<DT, 16>(k, plan, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t apass_run(const ApassArgs& a, const ApassPlan& plan, void* partial, double* loss_part,
                      int* dev_status, cudaStream_t st, bool allow_stats) {
  ApassKArgs k;
  k.A = reinterpret_cast<const unsigned char*>(a.A);
  k.n = a.n;
  k.d = a.d;
  k.ld = a.ld;
  k.p = a.p;
  k.D = a.D;
  k.b = a.b;
  k.D_out = a.D_out;
  k.t_out = a.t_out;
  k.mode = a.mode;
  k.R = plan.rows_per_step;
  k.S = plan.stages;
  k.dpad = plan.dpad;
  k.partial = partial;
  k.loss_part = loss_part;
  k.status = dev_status;
  k.skip = a.skip;
  k.executed = nullptr;
  k.col_scale = a.col_scale;
  k.row_split = nullptr;
  k.cta_time = nullptr;
  if (plan.ws && !compute_is_f64(a.dtype)) {
    k.row_split = row_split_lookup(a.dtype, a.ld * (int64_t)dtype_size(a.dtype), a.n, plan.grid, plan.rows_per_step);
    k.cta_time = g_cta_time;
  }
  {
    const double esz = (double)dtype_size(a.dtype), csz = compute_is_f64(a.dtype) ? 8.0 : 4.0;
    double bytes = (double)a.n * (double)a.d * esz + (double)a.d * csz + (double)plan.grid * a.d * csz;
    if (a.mode == MODE_DIAG || a.mode == MODE_RESID || a.mode == MODE_CONST) bytes += 8.0 * a.n;
    if (a.mode == MODE_LOGIT || a.mode == MODE_LGRAD) bytes += 16.0 * a.n;
    k.bytes_alg = bytes;
  }
  if (allow_stats && !g_prepare_only) k.tm = stats_device_timer();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int* flag = nullptr;
  // events cannot bracket a kernel node being captured into a graph; the in-kernel timer can
  const bool prof = allow_stats && !g_prepare_only && !launch_capturing() && stats_enabled() &&
                    stats_event_pair(&e0, &e1, &flag) == cudaSuccess;
  if (prof) {
    k.executed = flag;
    NYS_CUDA_TRY(cudaEventRecord(e0, st));
  }
  cudaError_t err;
  if (plan.ws) {
    err = apass_ws_launch(k, plan, a.dtype, st, g_prepare_only);
  } else switch (a.dtype) {
    case NYS_F64: err = launch_dt<NYS_F64>(k, plan, st); break;
    case NYS_F32: err = launch_float<NYS_F32>(k, plan, st); break;
    case NYS_BF16: err = launch_float<NYS_BF16>(k, plan, st); break;
    case NYS_FP8E4M3: err = launch_float<NYS_FP8E4M3>(k, plan, st); break;
    default: err = cudaErrorInvalidValue;
  }
  if (prof && err == cudaSuccess) {
    NYS_CUDA_TRY(cudaEventRecord(e1, st));
    // algorithmic bytes: A read once, p read, partials written, per-row vectors touched
    stats_record_apass(e0, e1, k.bytes_alg, a.dtype, flag);
  }
  return err;
}

// Balance the row slabs of the warp-specialised float pass over its CTAs (one read of A
// split over the SMs, Table 1's T_mv).  With equal slabs the CTAs on a few SMs finish ~3 %
// later on every pass (a group of SMs streams slower), and the pass waits for them.  Each
// CTA's time is measured, the rows are re-split in proportion to the measured speeds
// (boundaries on whole stages), up to three times, and a split is kept only while the pass
// gets faster.  The split fixes which rows each CTA sums, so for a given split the results
// stay bitwise repeatable.  ms_equal / ms_split: mean pass time before and after.
cudaError_t apass_balance_rows(const nys_matrix* A, const void* p, void* part, int* dstat, cudaStream_t st,
                               double* ms_equal, double* ms_split) {
  ApassPlan plan;
  if (ms_equal) *ms_equal = 0.0;
  if (ms_split) *ms_split = 0.0;
  if (compute_is_f64(A->dtype) || !apass_plan(A, &plan) || !plan.ws) return cudaSuccess;
  const int G = plan.grid, R = plan.rows_per_step;
  const int64_t n = A->n, rowbytes = A->ld * (int64_t)dtype_size(A->dtype);
  if (G < 2 || n < (int64_t)G * R * 8) return cudaSuccess;   // too few rows per CTA to matter
  ApassArgs a;
  a.A = A->data;
  a.n = A->n;
  a.d = A->d;
  a.ld = A->ld;
  a.dtype = A->dtype;
  a.col_scale = A->col_scale;
  a.p = p;
  a.D = nullptr;
  a.b = nullptr;
  a.D_out = nullptr;
  a.t_out = nullptr;
  a.mode = MODE_ID;
  NYS_CUDA_TRY(row_split_store(A->dtype, rowbytes, n, G, R, nullptr, st));   // start from the equal split
  unsigned long long* tbuf = nullptr;
  NYS_CUDA_TRY(cudaMalloc(&tbuf, (size_t)2 * G * sizeof(unsigned long long)));
  std::vector<unsigned long long> th((size_t)2 * G);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  auto time_passes = [&](double* ms) -> cudaError_t {
    NYS_CUDA_TRY(apass_run(a, plan, part, nullptr, dstat, st, false));   // warm-up
    NYS_CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < 5; ++r) NYS_CUDA_TRY(apass_run(a, plan, part, nullptr, dstat, st, false));
    NYS_CUDA_TRY(cudaEventRecord(e1, st));
    NYS_CUDA_TRY(cudaEventSynchronize(e1));
    float f = 0.f;
    NYS_CUDA_TRY(cudaEventElapsedTime(&f, e0, e1));
    *ms = f / 5.0;
    return cudaSuccess;
  };
  // per-CTA time (ns) from the pass's first start to the CTA's end, median of 5 passes
  auto cta_times = [&](std::vector<double>& T) -> cudaError_t {
    std::vector<std::vector<double>> rep((size_t)G);
    g_cta_time = tbuf;
    for (int r = 0; r < 5; ++r) {
      NYS_CUDA_TRY(cudaMemsetAsync(tbuf, 0, (size_t)2 * G * sizeof(unsigned long long), st));
      const cudaError_t e = apass_run(a, plan, part, nullptr, dstat, st, false);
      if (e != cudaSuccess) {
        g_cta_time = nullptr;
        return e;
      }
      NYS_CUDA_TRY(cudaMemcpyAsync(th.data(), tbuf, th.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      NYS_CUDA_TRY(cudaStreamSynchronize(st));
      unsigned long long t0 = ~0ull;
      for (int c = 0; c < G; ++c) t0 = std::min(t0, th[2 * c]);
      for (int c = 0; c < G; ++c) rep[c].push_back((double)(th[2 * c + 1] - t0));
    }
    g_cta_time = nullptr;
    T.resize(G);
    for (int c = 0; c < G; ++c) {
      std::sort(rep[c].begin(), rep[c].end());
      T[c] = rep[c][rep[c].size() / 2];
    }
    return cudaSuccess;
  };
  std::vector<int64_t> cur((size_t)G + 1), best_split;
  for (int c = 0; c <= G; ++c) cur[c] = n * c / G;
  double ms0 = 0.0, best = 0.0;
  if (err == cudaSuccess) err = time_passes(&ms0);
  best = ms0;
  for (int it = 0; it < 3 && err == cudaSuccess; ++it) {
    std::vector<double> T;
    err = cta_times(T);
    if (err != cudaSuccess) break;
    std::vector<double> speed((size_t)G);
    double tot = 0.0;
    for (int c = 0; c < G; ++c) {
      speed[c] = (double)(cur[c + 1] - cur[c]) / std::max(T[c], 1.0);
      tot += speed[c];
    }
    std::vector<int64_t> nxt((size_t)G + 1);
    nxt[0] = 0;
    double cum = 0.0;
    for (int c = 0; c + 1 < G; ++c) {
      cum += (double)n * speed[c] / tot;
      int64_t b = (int64_t)std::llround(cum / R) * R;
      b = std::max(b, nxt[c] + R);
      b = std::min(b, n - (int64_t)(G - 1 - c) * R);
      nxt[c + 1] = b;
    }
    nxt[G] = n;
    err = row_split_store(A->dtype, rowbytes, n, G, R, nxt.data(), st);
    double ms = 0.0;
    if (err == cudaSuccess) err = time_passes(&ms);
    if (err != cudaSuccess) break;
    if (ms < best * 0.998) {
      best = ms;
      best_split = nxt;
      cur = nxt;
    } else {
      break;
    }
  }
  if (err == cudaSuccess)
    err = row_split_store(A->dtype, rowbytes, n, G, R, best_split.empty() ? nullptr : best_split.data(), st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(tbuf);
  if (ms_equal) *ms_equal = ms0;
  if (ms_split) *ms_split = best;
  return err;
}

cudaError_t apass_prepare(const nys_matrix* A, const ApassPlan& plan) {
  ApassArgs a;
  a.A = A->data;
  a.n = A->n;
  a.d = A->d;
  a.ld = A->ld;
  a.dtype = A->dtype;
  a.col_scale = A->col_scale;
  a.p = nullptr;
  a.D = nullptr;
  a.b = nullptr;
  a.D_out = nullptr;
  a.t_out = nullptr;
  a.mode = MODE_ID;
  g_prepare_only = true;
  const cudaError_t e = apass_run(a, plan, nullptr, nullptr, nullptr, nullptr, false);
  g_prepare_only = false;
  return e;
}

cudaError_t apass_reduce(const ApassArgs& a, const ApassPlan& plan, const void* partial, double rho,
                         void* y, double* dot_part, int dot_blocks, cudaStream_t st) {
  const int nb = dot_blocks > 0 ? dot_blocks : reduce_blocks(a.d);
  if (compute_is_f64(a.dtype)) {
    count_launch();
    apass_reduce_kernel<double><<<nb, kVecThreads, 0, st>>>(
        reinterpret_cast<const double*>(partial), plan.grid, a.d, plan.dpad, rho,
        reinterpret_cast<const double*>(a.p), reinterpret_cast<double*>(y), dot_part, a.skip, nullptr);
  } else {
    count_launch();
    apass_reduce_kernel<float><<<nb, kVecThreads, 0, st>>>(
        reinterpret_cast<const float*>(partial), plan.grid, a.d, plan.dpad, (float)rho,
        reinterpret_cast<const float*>(a.p), reinterpret_cast<float*>(y), dot_part, a.skip,
        a.dtype == NYS_FP8E4M3 ? a.col_scale : nullptr);
  }
  return cudaGetLastError();
}

}  // namespace nys
