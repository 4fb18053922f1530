// Multi-right-hand-side Nystrom PCG for a lasso regularisation path.
//
// k lasso problems that share A, b and rho (and differ in gamma) share the
// x-subproblem matrix H + rho I of Eq. ADMMSubProb and therefore one Nystrom
// preconditioner.  Their k PCG solves (Alg. Nystrom PCG, one per column) are run
// side by side: every matvec reads A ONCE for all k columns as the two dense
// products W = A P (n x k) and V = A^T W + rho P (d x k), and the preconditioner is
// applied to the d x k block with two small GEMMs.  Each column keeps its own
// alpha, beta, residual and stop test; a converged column is frozen (alpha = 0).
// Vectors are d x k column-major in the PCG compute type; reductions are
// fixed-order per column.
#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "nys_internal.cuh"
#include "solver.cuh"

namespace nys {
namespace {

struct BCol {
  double wy, wy_new, pv, w2, r2, thresh2;
  float alpha, beta;
  int iters, done, status, pad;
};

template <typename C>
__global__ void b_matvec_finish_kernel(const C* __restrict__ part, int nz, int64_t len, C rho, const C* __restrict__ P,
                                       C* __restrict__ V) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    C s = C(0);
    for (int z = 0; z < nz; ++z) s += part[z * len + i];
    V[i] = fma(rho, P[i], s);
  }
}

// per-column partial dot products over a chunk of rows: warp w takes columns w, w+8, ...
template <typename C>
__global__ void __launch_bounds__(kVecThreads) b_coldot_kernel(const C* __restrict__ X, const C* __restrict__ Y,
                                                               int64_t d, int k, int chunk, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * chunk;
  const int64_t j1 = min(d, j0 + chunk);
  for (int c = warp; c < k; c += kVecThreads / 32) {
    const C* x = X + (int64_t)c * d;
    const C* y = Y + (int64_t)c * d;
    double acc = 0.0;
    for (int64_t j = j0 + lane; j < j1; j += 32) acc += (double)x[j] * (double)y[j];
    acc = warp_sum(acc);
    if (lane == 0) part[(int64_t)blockIdx.x * k + c] = acc;
  }
}

__global__ void b_colsum_kernel(const double* part, int nb, int k, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * k + c];
  out[c] = s;
}

// phase 0: init (r2, w2 -> threshold, done);  1: alpha from wy / pv;  2: stop test after the
// update (w2);  3: beta = wy_new / wy.  `sums` holds the column sums of the current dot.
__global__ void b_scalar_kernel(int phase, int k, BCol* col, const double* sums, const double* sums2, double tol,
                                int tol_abs, int maxit, int* ndone) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  BCol& s = col[c];
  if (phase == 0) {
    s.r2 = sums[c];
    s.w2 = sums2[c];
    s.thresh2 = tol_abs ? tol * tol : tol * tol * s.r2;
    s.iters = 0;
    s.status = 0;
    s.wy = 0.0;
    s.done = !(s.w2 > s.thresh2);
    s.alpha = 0.f;
    s.beta = 0.f;
  } else if (phase == 1) {
    s.pv = sums[c];
    if (s.done) {
      s.alpha = 0.f;
    } else if (!(s.pv > 0.0) || !isfinite(s.pv)) {
      s.alpha = 0.f;
      s.done = 1;
      s.status = s.iters == 0 ? NYS_EBREAKDOWN : NYS_ENOCONV;
    } else {
      s.alpha = (float)(s.wy / s.pv);
    }
  } else if (phase == 2) {
    if (!s.done) {
      s.w2 = sums[c];
      s.iters += 1;
      if (!(s.w2 > s.thresh2)) s.done = 1;
      else if (s.iters >= maxit) {
        s.done = 1;
        s.status = NYS_ENOCONV;
      }
    }
  } else {  // phase 3
    s.wy_new = sums[c];
    s.beta = s.wy > 0.0 ? (float)(s.wy_new / s.wy) : 0.f;
    s.wy = s.wy_new;
  }
  if (ndone && phase == 2) {
    // count converged columns (one writer per column; the host reads after the launch)
    if (s.done) atomicAdd(ndone, 1);
  }
}

template <typename C>
__global__ void b_init_w_kernel(int64_t len, const C* __restrict__ R, const C* __restrict__ V, C* __restrict__ W) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    W[i] = V ? R[i] - V[i] : R[i];
}

template <typename C>
__global__ void b_update_kernel(int64_t d, int k, C* __restrict__ X, C* __restrict__ W, const C* __restrict__ P,
                                const C* __restrict__ V, const BCol* col) {
  const int64_t len = d * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const C a = (C)col[i / d].alpha;
    X[i] = fma(a, P[i], X[i]);
    W[i] = fma(-a, V[i], W[i]);
  }
}

template <typename C>
__global__ void b_pupdate_kernel(int64_t d, int k, const C* __restrict__ Y, C* __restrict__ P, const BCol* col,
                                 int init) {
  const int64_t len = d * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    P[i] = init ? Y[i] : fma((C)col[i / d].beta, P[i], Y[i]);
}

// G (s x k) *= c_i row-wise
template <typename C>
__global__ void b_scale_rows_kernel(C* G, int s, int k, const C* __restrict__ cvec) {
  const int64_t len = (int64_t)s * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    G[i] *= cvec[i % s];
}

template <typename C>
__global__ void b_add_kernel(int64_t len, const C* __restrict__ W, C* __restrict__ Y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    Y[i] += W[i];
}

unsigned grid_for(int64_t len) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(8192, (len + 255) / 256)); }

}  // namespace

template <typename C>
nys_status batched_pcg_run(const PcgProblem& pb, const PrecondView& P, const C* R, C* X, int k, const PcgParams& prm,
                           cudaStream_t st, std::vector<int>* iters_out) {
  const int64_t d = pb.A->d, n = pb.A->n;
  const int s = P.s;
  const int64_t len = d * k;
  const int chunk = 1024;
  const int nbd = (int)((d + chunk - 1) / chunk);
  Pool pool(st);
  C* W = pool.alloc<C>(len);
  C* Y = pool.alloc<C>(len);
  C* Pd = pool.alloc<C>(len);
  C* V = pool.alloc<C>(len);
  C* Wn = pool.alloc<C>((size_t)n * k);
  const size_t atw_bytes = sketch_atw_work_bytes(pb.A, k);
  void* atw = pool.alloc<unsigned char>(atw_bytes);
  C* G = pool.alloc<C>((size_t)std::max(1, s) * k);
  C* gwork = pool.alloc<C>(std::max<size_t>(1, gemm_tn_work_elems<C>(d, std::max(1, s), k)));
  double* part = pool.alloc<double>((size_t)nbd * k);
  double* sums = pool.alloc<double>(k);
  double* sums2 = pool.alloc<double>(k);
  BCol* col = pool.alloc<BCol>(k);
  int* ndone = pool.alloc<int>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  const C* U = reinterpret_cast<const C*>(P.U);
  const C* cvec = reinterpret_cast<const C*>(P.c);
#define B_OK(x)                             \
  do {                                      \
    if ((x) != cudaSuccess) return NYS_ECUDA; \
  } while (0)
  auto launch_ok = [&]() { return cudaGetLastError() == cudaSuccess; };
  // BF16 storage: the k-column products run on the tensor cores (the same tcgen05 GEMMs
  // as the sketch, FP32 operand as three BF16 terms), with a transposed copy of A made
  // once for the whole solve
  TcPrepared tcp;
  bool use_tc = false;
  if constexpr (sizeof(C) == 4) {
    if (sketch_tc_supported(pb.A)) {
      void* tcs = pool.alloc<unsigned char>(tc_prepare_bytes(pb.A));
      if (!pool.ok()) return NYS_ENOMEM;
      if (tc_prepare(pb.A, tcs, &tcp, st) != cudaSuccess) return NYS_ECUDA;
      use_tc = true;
    }
  }
  // V = A^T (A P) + rho P for the k columns of P (reads A once)
  auto bmatvec = [&](const C* Pin, C* Vout) -> bool {
    if constexpr (sizeof(C) == 4) {
      if (use_tc) return tc_hmm(pb.A, tcp, pb.D, reinterpret_cast<const float*>(Pin), k, pb.rho,
                                reinterpret_cast<float*>(Vout), st) == cudaSuccess;
    }
    if (sketch_aw(pb.A, Pin, k, pb.D, Wn, st) != cudaSuccess) return false;
    int nz = 0;
    if (sketch_atw_partials(pb.A, Wn, k, atw, atw_bytes, &nz, st) != cudaSuccess) return false;
    count_launch();
    b_matvec_finish_kernel<C><<<grid_for(len), 256, 0, st>>>((const C*)atw, nz, len, (C)pb.rho, Pin, Vout);
    return launch_ok();
  };
  auto coldot = [&](const C* A_, const C* B_, double* out) -> bool {
    count_launch();
    b_coldot_kernel<C><<<nbd, kVecThreads, 0, st>>>(A_, B_, d, k, chunk, part);
    count_launch();
    b_colsum_kernel<<<(k + 127) / 128, 128, 0, st>>>(part, nbd, k, out);
    return launch_ok();
  };
  // Y = P^{-1} W = U diag(c) U^T W + W
  auto precond = [&]() -> bool {
    if (s == 0) return cudaMemcpyAsync(Y, W, len * sizeof(C), cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    if (gemm_tn<C>(U, W, d, s, k, G, gwork, st) != cudaSuccess) return false;
    count_launch();
    b_scale_rows_kernel<C><<<grid_for((int64_t)s * k), 256, 0, st>>>(G, s, k, cvec);
    if (gemm_nn_t<C>(U, d, s, G, k, Y, st) != cudaSuccess) return false;
    count_launch();
    b_add_kernel<C><<<grid_for(len), 256, 0, st>>>(len, W, Y);
    return launch_ok();
  };
  auto scalar = [&](int phase, const double* s1, const double* s2, int* nd) -> bool {
    count_launch();
    b_scalar_kernel<<<(k + 127) / 128, 128, 0, st>>>(phase, k, col, s1, s2, prm.tol, prm.tol_abs, prm.maxit, nd);
    return launch_ok();
  };

  // init: W = R - (H + rho I) X0, thresholds, Y = P^{-1} W, P = Y
  if (!prm.x0_zero) {
    if (!bmatvec(X, V)) return NYS_ECUDA;
  }
  count_launch();
  b_init_w_kernel<C><<<grid_for(len), 256, 0, st>>>(len, R, prm.x0_zero ? nullptr : V, W);
  if (!coldot(R, R, sums) || !coldot(W, W, sums2) || !scalar(0, sums, sums2, nullptr)) return NYS_ECUDA;
  if (!precond() || !coldot(W, Y, sums) || !scalar(3, sums, nullptr, nullptr)) return NYS_ECUDA;
  count_launch();
  b_pupdate_kernel<C><<<grid_for(len), 256, 0, st>>>(d, k, Y, Pd, col, 1);
  std::vector<BCol> hc(k);
  B_OK(cudaMemcpyAsync(hc.data(), col, k * sizeof(BCol), cudaMemcpyDeviceToHost, st));
  B_OK(cudaStreamSynchronize(st));
  int done_h = 0;
  for (const BCol& c : hc) done_h += c.done;
  const int cap = prm.fixed >= 0 ? prm.fixed : prm.maxit;
  for (int it = 0; it < cap && done_h < k; ++it) {
    if (!bmatvec(Pd, V) || !coldot(Pd, V, sums) || !scalar(1, sums, nullptr, nullptr)) return NYS_ECUDA;
    count_launch();
    b_update_kernel<C><<<grid_for(len), 256, 0, st>>>(d, k, X, W, Pd, V, col);
    B_OK(cudaMemsetAsync(ndone, 0, sizeof(int), st));
    if (!coldot(W, W, sums) || !scalar(2, sums, nullptr, ndone)) return NYS_ECUDA;
    if (!precond() || !coldot(W, Y, sums) || !scalar(3, sums, nullptr, nullptr)) return NYS_ECUDA;
    count_launch();
    b_pupdate_kernel<C><<<grid_for(len), 256, 0, st>>>(d, k, Y, Pd, col, 0);
    B_OK(cudaMemcpyAsync(&done_h, ndone, sizeof(int), cudaMemcpyDeviceToHost, st));
    B_OK(cudaStreamSynchronize(st));
  }
  B_OK(cudaMemcpyAsync(hc.data(), col, k * sizeof(BCol), cudaMemcpyDeviceToHost, st));
  B_OK(cudaStreamSynchronize(st));
#undef B_OK
  nys_status res = NYS_OK;
  if (iters_out) iters_out->assign(k, 0);
  for (int c = 0; c < k; ++c) {
    if (iters_out) (*iters_out)[c] = hc[c].iters;
    if (hc[c].status == NYS_EBREAKDOWN) res = NYS_EBREAKDOWN;
    else if (res == NYS_OK && (hc[c].status == NYS_ENOCONV || (!hc[c].done && prm.fixed < 0))) res = NYS_ENOCONV;
  }
  return res;
}
template nys_status batched_pcg_run<float>(const PcgProblem&, const PrecondView&, const float*, float*, int,
                                           const PcgParams&, cudaStream_t, std::vector<int>*);
template nys_status batched_pcg_run<double>(const PcgProblem&, const PrecondView&, const double*, double*, int,
                                            const PcgParams&, cudaStream_t, std::vector<int>*);

// ------------------------------------------------------------------ ADMM steps on d x k blocks
namespace {
template <typename C>
__global__ void b_rhs_kernel(int64_t d, int k, const double* __restrict__ q, const double* __restrict__ Z,
                             const double* __restrict__ Uu, double rho, C* __restrict__ R) {
  const int64_t len = d * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    R[i] = (C)fma(rho, Z[i] - Uu[i], q[i % d]);
}

// column c: z = S_{kappa_c}(x + u), u += x - z; partials of ||x - z||^2 and ||z - z_old||^2
template <typename C>
__global__ void __launch_bounds__(kVecThreads) b_zu_kernel(int64_t d, int k, int chunk, const C* __restrict__ Xc,
                                                           double* __restrict__ X, double* __restrict__ Z,
                                                           double* __restrict__ Uu, const double* __restrict__ kappa,
                                                           double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * chunk;
  const int64_t j1 = min(d, j0 + chunk);
  for (int c = warp; c < k; c += kVecThreads / 32) {
    const double kap = kappa[c];
    double a0 = 0.0, a1 = 0.0;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      const int64_t i = (int64_t)c * d + j;
      const double xj = (double)Xc[i];
      const double zo = Z[i];
      const double vj = xj + Uu[i];
      const double mag = fabs(vj) - kap;
      const double zj = mag > 0.0 ? copysign(mag, vj) : 0.0;
      X[i] = xj;
      Z[i] = zj;
      Uu[i] += xj - zj;
      a0 += (xj - zj) * (xj - zj);
      a1 += (zj - zo) * (zj - zo);
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    if (lane == 0) {
      part[((int64_t)blockIdx.x * k + c) * 2] = a0;
      part[((int64_t)blockIdx.x * k + c) * 2 + 1] = a1;
    }
  }
}
}  // namespace

template <typename C>
cudaError_t batched_rhs(int64_t d, int k, const double* q, const double* Z, const double* Uu, double rho, C* R,
                        cudaStream_t st) {
  count_launch();
  b_rhs_kernel<C><<<grid_for(d * k), 256, 0, st>>>(d, k, q, Z, Uu, rho, R);
  return cudaGetLastError();
}
template <typename C>
cudaError_t batched_zu(int64_t d, int k, const C* Xc, double* X, double* Z, double* Uu, const double* kappa,
                       double* part, int* nb_out, cudaStream_t st) {
  const int chunk = 1024;
  const int nb = (int)((d + chunk - 1) / chunk);
  count_launch();
  b_zu_kernel<C><<<nb, kVecThreads, 0, st>>>(d, k, chunk, Xc, X, Z, Uu, kappa, part);
  *nb_out = nb;
  return cudaGetLastError();
}
int batched_zu_blocks(int64_t d) { return (int)((d + 1023) / 1024); }
template cudaError_t batched_rhs<float>(int64_t, int, const double*, const double*, const double*, double, float*,
                                        cudaStream_t);
template cudaError_t batched_rhs<double>(int64_t, int, const double*, const double*, const double*, double, double*,
                                         cudaStream_t);
template cudaError_t batched_zu<float>(int64_t, int, const float*, double*, double*, double*, const double*, double*,
                                       int*, cudaStream_t);
template cudaError_t batched_zu<double>(int64_t, int, const double*, double*, double*, double*, const double*,
                                        double*, int*, cudaStream_t);

}  // namespace nys
