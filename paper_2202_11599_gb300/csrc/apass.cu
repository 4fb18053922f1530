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
#include "device_util.cuh"
#include "nys_internal.cuh"

#include <algorithm>

namespace nys {

constexpr int kMaxStages = 8;
constexpr int kRMax = 4;
constexpr int kSmemBudget = 200 * 1024;

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
};

__device__ __forceinline__ double sigmoid_d(double t) {
  // stable logistic function
  if (t >= 0) {
    const double e = exp(-t);
    return 1.0 / (1.0 + e);
  }
  const double e = exp(t);
  return e / (1.0 + e);
}

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

  auto issue = [&](int step) {
    const int stage = step % S;
    const int64_t row = r0 + (int64_t)step * R;
    const int rows = (int)min((int64_t)R, r1 - row);
    const uint32_t bytes = (uint32_t)(rows * rowbytes);
    mbar_arrive_expect_tx(&bars[stage], bytes);
    tma_load_1d(smem + stage * stage_bytes, a.A + row * rowbytes, bytes, &bars[stage]);
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
}

// y_j = sum_g partial[g][j] (fixed order) + rho p_j; optional per-block partials of p^T y.
template <typename C>
__global__ void __launch_bounds__(kVecThreads) apass_reduce_kernel(const C* __restrict__ partial, int G,
                                                                   int64_t d, int64_t dpad, C rho,
                                                                   const C* __restrict__ p, C* __restrict__ y,
                                                                   double* dot_part, const int* skip) {
  if (skip && *skip) return;
  __shared__ double sh[kVecThreads / 32];
  double dacc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    C s = C(0);
    for (int g = 0; g < G; ++g) s += partial[(int64_t)g * dpad + j];
    const C pj = p ? p[j] : C(0);
    const C yj = fma(rho, pj, s);
    y[j] = yj;
    dacc += (double)pj * (double)yj;
  }
  if (dot_part) {
    const double t = block_sum<kVecThreads>(dacc, sh);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = t;
  }
}

static int sm_count() {
  static int c = 0;
  if (c == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    if (c <= 0) c = 1;
  }
  return c;
}

int reduce_blocks(int64_t d) {
  const int64_t b = (d + kVecThreads - 1) / kVecThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4 * (int64_t)sm_count()));
}

static int vpt_bucket(int64_t nvec) {
  const int64_t need = (nvec + kApassThreads - 1) / kApassThreads;
  static const int buckets[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
  for (int b : buckets)
    if (need <= b) return b;
  return -1;
}

bool apass_plan(const nys_matrix* A, ApassPlan* plan) {
  const int64_t esz = (int64_t)dtype_size(A->dtype);
  const int vec = (int)(16 / esz);
  const int64_t nvec = (A->d + vec - 1) / vec;
  int vpt = vpt_bucket(nvec);
  if (vpt < 0) return false;
  if (A->dtype == NYS_F64 && vpt > 12) return false;
  const int64_t rowbytes = A->ld * esz;
  int R = (int)std::max<int64_t>(1, std::min<int64_t>(kRMax, (48 * 1024) / rowbytes));
  int S = (int)std::min<int64_t>(kMaxStages, kSmemBudget / (R * rowbytes));
  if (S < 2) {
    R = 1;
    S = (int)std::min<int64_t>(kMaxStages, kSmemBudget / rowbytes);
  }
  if (S < 2) return false;
  plan->rows_per_step = R;
  plan->stages = S;
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

template <int DT, int VPT>
static cudaError_t launch_vpt(const ApassKArgs& k, const ApassPlan& plan, cudaStream_t st) {
  auto fn = apass_kernel<DT, VPT>;
  static bool attr_set = false;
  if (!attr_set) {
    NYS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    attr_set = true;
  }
  fn<<<plan.grid, kApassThreads, plan.smem, st>>>(k);
  return cudaGetLastError();
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
                      int* dev_status, cudaStream_t st) {
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
  switch (a.dtype) {
    case NYS_F64: return launch_dt<NYS_F64>(k, plan, st);
    case NYS_F32: return launch_dt<NYS_F32>(k, plan, st);
    case NYS_BF16: return launch_dt<NYS_BF16>(k, plan, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t apass_reduce(const ApassArgs& a, const ApassPlan& plan, const void* partial, double rho,
                         void* y, double* dot_part, int dot_blocks, cudaStream_t st) {
  const int nb = dot_blocks > 0 ? dot_blocks : reduce_blocks(a.d);
  if (compute_is_f64(a.dtype)) {
    apass_reduce_kernel<double><<<nb, kVecThreads, 0, st>>>(
        reinterpret_cast<const double*>(partial), plan.grid, a.d, plan.dpad, rho,
        reinterpret_cast<const double*>(a.p), reinterpret_cast<double*>(y), dot_part, a.skip);
  } else {
    apass_reduce_kernel<float><<<nb, kVecThreads, 0, st>>>(
        reinterpret_cast<const float*>(partial), plan.grid, a.d, plan.dpad, (float)rho,
        reinterpret_cast<const float*>(a.p), reinterpret_cast<float*>(y), dot_part, a.skip);
  }
  return cudaGetLastError();
}

}  // namespace nys
