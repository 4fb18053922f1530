// C ABI of libnysadmm (include/nysadmm.h): argument checks, the Nystrom sketch
// driver (App. B), the preconditioner handle (Eq. Nystrom preconditioner), the
// PCG entry point (App. B, Alg. Nystrom PCG) and the NysADMM drivers
// (Alg. NysADMM for the lasso, Sec. 3.2 + App. C for l1-logistic regression).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "device_util.cuh"
#include "solver.cuh"

using namespace nys;

struct nys_precond_s {
  int64_t d = 0;
  int s = 0;
  double nu = 0.0;
  double* U64 = nullptr;  // d x s, column-major
  float* U32 = nullptr;   // FP32 copy, built on first FP32 use
  double* lam_d = nullptr;
  std::vector<double> lam;  // host copy, descending
};

namespace nys {

nys_status check_matrix(const nys_matrix* A) {
  if (!A || !A->data) return NYS_EINVAL;
  if (A->n <= 0 || A->d <= 0 || A->ld < A->d) return NYS_EINVAL;
  if (A->dtype != NYS_F64 && A->dtype != NYS_F32 && A->dtype != NYS_BF16 && A->dtype != NYS_FP8E4M3)
    return NYS_EINVAL;
  if ((A->dtype == NYS_FP8E4M3) != (A->col_scale != nullptr)) return NYS_EINVAL;  // scales iff FP8
  const size_t esz = dtype_size(A->dtype);
  if ((A->ld * esz) % 16 != 0) return NYS_EINVAL;
  if (reinterpret_cast<uintptr_t>(A->data) % 16 != 0) return NYS_EINVAL;
  ApassPlan plan;
  if (!apass_plan(A, &plan)) return NYS_EINVAL;
  return NYS_OK;
}

// Arguments of the H-matvec entry points (nys_hmatvec and its allocation-free variant).
nys_status check_hmatvec_args(const nys_matrix* A, double rho, const void* p, const void* y) {
  const nys_status s = check_matrix(A);
  if (s != NYS_OK) return s;
  if (!p || !y || p == y || !std::isfinite(rho)) return NYS_EINVAL;
  return NYS_OK;
}

}  // namespace nys

namespace {

constexpr int kMaxRank = 1024;

// Phase trace (set NYS_TRACE=1): wall time of each sketch / core phase, the stream
// synchronised at both ends, printed to stderr.
struct PhaseTimer {
  const char* name;
  cudaStream_t st;
  std::chrono::steady_clock::time_point t0;
  bool on;
  PhaseTimer(const char* n, cudaStream_t s) : name(n), st(s), on(std::getenv("NYS_TRACE") != nullptr) {
    if (on) {
      cudaStreamSynchronize(st);
      t0 = std::chrono::steady_clock::now();
    }
  }
  ~PhaseTimer() {
    if (!on) return;
    cudaStreamSynchronize(st);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::fprintf(stderr, "[nys] %-22s %9.3f ms\n", name, ms);
  }
};

cudaStream_t stream_of(const nys_opts* o) { return o ? reinterpret_cast<cudaStream_t>(o->stream) : nullptr; }

bool is_fin(double v) { return std::isfinite(v); }

nys_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return NYS_OK;
  if (e == cudaErrorMemoryAllocation) return NYS_ENOMEM;
  return NYS_ECUDA;
}

#define NYS_TRY(expr)                    \
  do {                                   \
    nys_status _s = (expr);              \
    if (_s != NYS_OK) return _s;         \
  } while (0)
#define NYS_CU(expr) NYS_TRY(cuda_status(expr))

double eps_host(double t, int mant_bits) {
  t = std::fabs(t);
  if (t == 0.0) return mant_bits == 52 ? std::ldexp(1.0, -1074) : std::ldexp(1.0, -149);
  int e = 0;
  std::frexp(t, &e);
  return std::ldexp(1.0, e - 1 - mant_bits);
}

// Thin QR of Omega (d x m, in place) by CholQR2: twice G = Om^T Om, C = chol(G), Om <- Om C^{-1}.
// fp32_class: the panel is rounded to BF16 values right after (the test matrix of an
// FP32-class sketch), so the second pass stops after its Gram when the first pass already
// left Om orthonormal to 2^-20 (max |Om^T Om - I|), far below that rounding's 2^-8 -- one
// CholQR pass does so for any well-conditioned panel (loss of orthogonality ~ cond^2 2^-53).
nys_status cholqr2(double* Om, int64_t d, int m, cudaStream_t st, bool fp32_class = false) {
  PhaseTimer pt("cholqr2", st);
  Pool pool(st);
  double* G = pool.alloc<double>((size_t)m * m);
  double* work = pool.alloc<double>(gram_work_bytes(d, m) / sizeof(double) + 1);
  int* info = pool.alloc<int>(1);
  double* gap = pool.alloc<double>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  for (int pass = 0; pass < 2; ++pass) {
    NYS_CU(gram_xty(Om, Om, d, m, G, work, st));
    if (pass == 1 && fp32_class) {
      NYS_CU(identity_gap(G, m, gap, st));
      double gap_h = 1.0;
      NYS_CU(cudaMemcpyAsync(&gap_h, gap, sizeof(double), cudaMemcpyDeviceToHost, st));
      NYS_CU(cudaStreamSynchronize(st));
      if (gap_h <= 0x1p-20) break;
    }
    // a pivot below 1e-10 of the largest column norm^2: columns dependent to ~1e-5, which
    // CholQR cannot orthonormalise -- refused as a bad test matrix
    NYS_CU(chol_upper(G, m, info, st, 1e-10));
    int info_h = 0;
    NYS_CU(cudaMemcpyAsync(&info_h, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    NYS_CU(cudaStreamSynchronize(st));
    if (info_h != 0) return NYS_EINVAL;  // Omega has (numerically) dependent columns
    NYS_CU(trsm_right_upper(G, m, Om, d, st));
  }
  return NYS_OK;
}

// Y (d x m, FP64) = (A^T diag(D) A + shift I) Om for an FP64 orthonormal panel Om.
// prep: tensor-core operands of A prepared once by the caller (repeated sketches of the
// same matrix), or NULL.  For a low-precision matrix (an FP32-class sketch) Om is first
// rounded in place to BF16 values; the caller's later steps use that rounded Om.
nys_status sketch_panel(const nys_matrix* A, const double* D, double shift, double* Om, int m, double* Y,
                        cudaStream_t st, const TcPrepared* prep = nullptr) {
  PhaseTimer pt("sketch Y = H Omega", st);
  Pool pool(st);
  const int64_t n = A->n, d = A->d;
  if (A->dtype != NYS_F64 && A->dtype != NYS_FP8E4M3) NYS_CU(round_panel_bf16(Om, d * m, st));
  if (A->dtype == NYS_FP8E4M3) {
    // FP8: sketch the dequantised matrix (s_j q_ij in FP32, exact products of the 4-bit
    // codes and the scales up to FP32 rounding) through the FP32 path
    float* A32 = pool.alloc<float>((size_t)n * A->ld);
    if (!pool.ok()) return NYS_ENOMEM;
    NYS_CU(dequantize_fp8(A, A32, st));
    nys_matrix M32 = *A;
    M32.data = A32;
    M32.dtype = NYS_F32;
    M32.col_scale = nullptr;
    return sketch_panel(&M32, D, shift, Om, m, Y, st, nullptr);
  }
  if (sketch_tc_supported(A)) {
    NYS_CU(prep ? sketch_tc_with(A, *prep, D, Om, m, Y, st) : sketch_tc(A, D, Om, m, Y, st));
    NYS_TRY(shard_sum(Y, d * m, NYS_F64, st));   // row-sharded: sum of the ranks' A_g^T D_g A_g Omega
    if (shift != 0.0) NYS_CU(axpy_panel(shift, Om, Y, d * m, st));
    return NYS_OK;
  }
  const size_t wbytes = sketch_atw_work_bytes(A, m);
  void* work = pool.alloc<unsigned char>(wbytes);
  if (A->dtype == NYS_F64) {
    double* W = pool.alloc<double>((size_t)n * m);
    if (!pool.ok()) return NYS_ENOMEM;
    NYS_CU(sketch_aw(A, Om, m, D, W, st));
    NYS_CU(sketch_atw(A, W, m, Y, work, wbytes, st));
  } else {
    float* Om32 = pool.alloc<float>((size_t)d * m);
    float* W = pool.alloc<float>((size_t)n * m);
    if (!pool.ok()) return NYS_ENOMEM;
    NYS_CU(convert_f64_to_f32(Om, Om32, d * m, st));
    NYS_CU(sketch_aw(A, Om32, m, D, W, st));
    NYS_CU(sketch_atw(A, W, m, Y, work, wbytes, st));
  }
  NYS_TRY(shard_sum(Y, d * m, NYS_F64, st));   // row-sharded: sum of the ranks' A_g^T D_g A_g Omega
  if (shift != 0.0) NYS_CU(axpy_panel(shift, Om, Y, d * m, st));
  return NYS_OK;
}

// FP64 core of App. B from the orthonormal Om and Y = H Om (both d x s):
// nu, Y_nu, C = chol(Om^T Y_nu) (retrying with 10x nu up to 3 times), B = Y_nu C^{-1},
// thin SVD of B via Jacobi on B^T B, U = B V Sigma^{-1}, lam = max(0, Sigma^2 - nu).
nys_status nystrom_core(const double* Om, const double* Y, int64_t d, int s, double shift_scale, int mant_bits,
                        double* U, double* lam_d, std::vector<double>& lam_h, double* nu_out, cudaStream_t st) {
  Pool pool(st);
  double* G = pool.alloc<double>((size_t)s * s);
  double* gw = pool.alloc<double>(gram_work_bytes(d, s) / sizeof(double) + 1);
  double* lmax = pool.alloc<double>(1);
  double* pw = pool.alloc<double>(2 * (size_t)s + 2);   // power iteration: two w buffers + barrier words
  double* Ynu = pool.alloc<double>((size_t)d * s);
  double* M = pool.alloc<double>((size_t)s * s);
  int* info = pool.alloc<int>(1);
  const int N = s + (s & 1);
  double* V = pool.alloc<double>((size_t)N * N);
  double* jw = pool.alloc<double>(jacobi_work_bytes(s) / sizeof(double) + 1);
  double* fw = pool.alloc<double>((size_t)s * s + s);
  if (!pool.ok()) return NYS_ENOMEM;

  PhaseTimer pt_all("nystrom core (total)", st);
  {
    PhaseTimer pt("core: Y^T Y + power", st);
    NYS_CU(gram_xty(Y, Y, d, s, G, gw, st));
    NYS_CU(power_lambda_max(G, s, lmax, pw, st));
  }
  double lmax_h = 0.0;
  NYS_CU(cudaMemcpyAsync(&lmax_h, lmax, sizeof(double), cudaMemcpyDeviceToHost, st));
  NYS_CU(cudaStreamSynchronize(st));
  if (!is_fin(lmax_h)) return NYS_EINVAL;
  double nu = shift_scale * eps_host(std::sqrt(std::max(lmax_h, 0.0)), mant_bits);
  bool ok = false;
  PhaseTimer* pt_chol = new PhaseTimer("core: shift + chol", st);
  for (int attempt = 0; attempt < 4; ++attempt) {
    NYS_CU(cudaMemcpyAsync(Ynu, Y, (size_t)d * s * sizeof(double), cudaMemcpyDeviceToDevice, st));
    NYS_CU(axpy_panel(nu, Om, Ynu, d * s, st));
    NYS_CU(gram_xty(Om, Ynu, d, s, M, gw, st));
    NYS_CU(chol_upper(M, s, info, st));
    int info_h = 0;
    NYS_CU(cudaMemcpyAsync(&info_h, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    NYS_CU(cudaStreamSynchronize(st));
    if (info_h == 0) {
      ok = true;
      break;
    }
    nu *= 10.0;
  }
  delete pt_chol;
  if (!ok) return NYS_ENOTSPD;
  {
    PhaseTimer pt("core: trsm + B^T B", st);
    NYS_CU(trsm_right_upper(M, s, Ynu, d, st));       // B = Y_nu C^{-1} (in Ynu)
    NYS_CU(gram_xty(Ynu, Ynu, d, s, G, gw, st));      // B^T B
  }
  int sweeps = 0;
  {
    // B^T B carries the sketch's rounding (unit roundoff 2^-(mant_bits + 1), relative): the
    // sweeps stop at that level, and at off(B^T B) <= 1e-12 ||B^T B||_F for an FP64 sketch
    PhaseTimer pt("core: jacobi", st);
    NYS_CU(jacobi_eig(G, V, s, jw, &sweeps, st, std::max(1e-12, std::ldexp(1.0, -mant_bits - 1))));
  }
  {
    PhaseTimer pt("core: finish (U = BV)", st);
    NYS_CU(nystrom_finish(Ynu, d, s, jw, V, nu, U, lam_d, fw, st));
  }
  if (std::getenv("NYS_TRACE")) std::fprintf(stderr, "[nys] jacobi sweeps %d (s = %d)\n", sweeps, s);
  lam_h.resize(s);
  NYS_CU(cudaMemcpyAsync(lam_h.data(), lam_d, s * sizeof(double), cudaMemcpyDeviceToHost, st));
  NYS_CU(cudaStreamSynchronize(st));
  if (nu_out) *nu_out = nu;
  return NYS_OK;
}

nys_status precond_alloc(nys_precond_s* P, int64_t d, int s) {
  P->d = d;
  P->s = s;
  if (cudaMalloc(&P->U64, (size_t)d * s * sizeof(double)) != cudaSuccess) return NYS_ENOMEM;
  if (cudaMalloc(&P->lam_d, (size_t)s * sizeof(double)) != cudaSuccess) return NYS_ENOMEM;
  return NYS_OK;
}

void precond_free(nys_precond_s* P) {
  if (!P) return;
  if (P->U64) cudaFree(P->U64);
  if (P->U32) cudaFree(P->U32);
  if (P->lam_d) cudaFree(P->lam_d);
  delete P;
}

// Device view of P^{-1} for one rho in the PCG compute type.
template <typename C>
nys_status precond_view(nys_precond_s* P, double rho, C* c, cudaStream_t st, PrecondView* out) {
  out->s = 0;
  out->U = nullptr;
  out->c = nullptr;
  if (!P || P->s == 0) return NYS_OK;
  const int s = P->s;
  std::vector<C> ch(s);
  const double lam_s = P->lam[s - 1];
  for (int i = 0; i < s; ++i) ch[i] = (C)((lam_s + rho) / (P->lam[i] + rho) - 1.0);
  NYS_CU(cudaMemcpyAsync(c, ch.data(), s * sizeof(C), cudaMemcpyHostToDevice, st));
  NYS_CU(cudaStreamSynchronize(st));  // ch goes out of scope
  if constexpr (sizeof(C) == 8) {
    out->U = P->U64;
  } else {
    if (!P->U32) {
      if (cudaMalloc(&P->U32, (size_t)P->d * s * sizeof(float)) != cudaSuccess) return NYS_ENOMEM;
      NYS_CU(convert_f64_to_f32(P->U64, P->U32, P->d * s, st));
    }
    out->U = P->U32;
  }
  out->c = c;
  out->s = s;
  return NYS_OK;
}

// Sketch of H = A^T diag(D) A + shift I with Omega blocks already orthonormalised:
// the panels Om (d x s) and Y (d x s) are given; builds/refreshes P.
nys_status precond_from_panels(const double* Om, const double* Y, int64_t d, int s, double shift_scale,
                               int mant_bits, nys_precond_s* P, cudaStream_t st) {
  if (P->s != s) {
    if (P->U64) cudaFree(P->U64);
    if (P->U32) cudaFree(P->U32);
    if (P->lam_d) cudaFree(P->lam_d);
    P->U64 = nullptr;
    P->U32 = nullptr;
    P->lam_d = nullptr;
    NYS_TRY(precond_alloc(P, d, s));
  } else if (P->U32) {
    cudaFree(P->U32);
    P->U32 = nullptr;
  }
  return nystrom_core(Om, Y, d, s, shift_scale, mant_bits, P->U64, P->lam_d, P->lam, &P->nu, st);
}

// Omega of a solve: the caller's panel (d x m, copied) or, when Omega is NULL, a panel drawn
// in the library from `seed` (Philox-4x32-10 + Box-Muller, nys_gaussian_test_matrix).
nys_status omega_panel(const double* Omega, uint64_t seed, int64_t d, int m, double* Om, cudaStream_t st) {
  if (Omega) return cuda_status(cudaMemcpyAsync(Om, Omega, (size_t)d * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return cuda_status(gaussian_panel(seed, d, m, Om, st));
}

int mant_bits_of(const nys_matrix* A) { return A->dtype == NYS_F64 ? 52 : 23; }

template <typename C>
nys_status hmatvec_t(const nys_matrix* A, const double* D, double rho, const void* p, void* y, cudaStream_t st) {
  ApassPlan plan;
  apass_plan(A, &plan);
  Pool pool(st);
  void* part = pool.alloc<unsigned char>(apass_partial_bytes(A, plan));
  int* dstat = pool.alloc<int>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  NYS_CU(cudaMemsetAsync(dstat, 0, sizeof(int), st));
  ApassArgs a;
  a.A = A->data;
  a.n = A->n;
  a.d = A->d;
  a.ld = A->ld;
  a.dtype = A->dtype;
  a.col_scale = A->col_scale;
  a.p = p;
  a.D = D;
  a.b = nullptr;
  a.D_out = nullptr;
  a.t_out = nullptr;
  a.mode = D ? MODE_DIAG : MODE_ID;
  NYS_CU(apass_run(a, plan, part, nullptr, dstat, st));
  NYS_CU(apass_reduce(a, plan, part, rho, y, nullptr, 0, st));
  int h = 0;
  NYS_CU(cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  NYS_CU(cudaStreamSynchronize(st));
  return h ? (nys_status)h : NYS_OK;
}

// y = A^T phi(A p) for an ADMM helper pass (modes CONST / RESID / LOGIT / LGRAD), rho = 0.
nys_status aux_pass(const nys_matrix* A, int mode, const void* p, const double* b, double* D_out, double* t_out,
                    void* y, double* loss_h, cudaStream_t st) {
  Pool pool(st);
  ApassPlan plan;
  apass_plan(A, &plan);
  void* part = pool.alloc<unsigned char>(apass_partial_bytes(A, plan));
  double* lp = pool.alloc<double>(plan.grid);
  int* dstat = pool.alloc<int>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  NYS_CU(cudaMemsetAsync(dstat, 0, sizeof(int), st));
  NYS_CU(cudaMemsetAsync(lp, 0, plan.grid * sizeof(double), st));
  ApassArgs a;
  a.A = A->data;
  a.n = A->n;
  a.d = A->d;
  a.ld = A->ld;
  a.dtype = A->dtype;
  a.col_scale = A->col_scale;
  a.p = p;
  a.D = nullptr;
  a.b = b;
  a.D_out = D_out;
  a.t_out = t_out;
  a.mode = mode;
  NYS_CU(apass_run(a, plan, part, lp, dstat, st));
  ApassArgs ar = a;
  ar.p = nullptr;
  NYS_CU(apass_reduce(ar, plan, part, 0.0, y, nullptr, 0, st));
  if (loss_h) {
    std::vector<double> h(plan.grid);
    NYS_CU(cudaMemcpyAsync(h.data(), lp, plan.grid * sizeof(double), cudaMemcpyDeviceToHost, st));
    NYS_CU(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : h) s += v;
    *loss_h = s;
  }
  int hs = 0;
  NYS_CU(cudaMemcpyAsync(&hs, dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  NYS_CU(cudaStreamSynchronize(st));
  return hs ? (nys_status)hs : NYS_OK;
}

// Result of a pass in A's compute type -> FP64 vector.
nys_status to_f64(const nys_matrix* A, const void* y, double* out, int64_t d, cudaStream_t st) {
  if (A->dtype == NYS_F64) {
    if (y != out) NYS_CU(cudaMemcpyAsync(out, y, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return NYS_OK;
  }
  NYS_CU(convert_f32_to_f64(reinterpret_cast<const float*>(y), out, d, st));
  return NYS_OK;
}

// PCG tolerance of ADMM iteration k (0-based): the decaying schedule ||r^k|| / k^beta of
// Sec. 5 (beta = tol, k counted from 1, a relative test) or the fixed tol.
double sched_tol(int mode, double tol, int k) {
  return mode == NYS_TOL_RNORM_POW ? std::pow((double)(k + 1), -tol) : tol;
}

// Alg. AdaptiveRandNysAppx (App. C): ranks s0, 2 s0, 4 s0, ... until (lam_s + rho)/rho <= Tol,
// extended once to s_max when doubling would pass it.  Each new block of the Gaussian Om
// (d x s_max) is orthonormalised on its own and its sketch H Om_block (H = A^T D A + shift I)
// is appended to Y; the approximation is rebuilt from all blocks so far.  *used_out: the rank.
nys_status adaptive_sketch(const nys_matrix* Ain, const double* D, double shift, double* Om, double* Y, int64_t d,
                           int rank, int smax, double ada_tol, double rho, double shs, const TcPrepared* tcpp,
                           nys_precond_s* P, int* used_out, cudaStream_t st) {
  int s0 = rank, m = rank, used = 0;
  auto add_block = [&](int cols) -> nys_status {
    NYS_TRY(cholqr2(Om + (int64_t)used * d, d, cols, st, Ain->dtype != NYS_F64));
    NYS_TRY(sketch_panel(Ain, D, shift, Om + (int64_t)used * d, cols, Y + (int64_t)used * d, st, tcpp));
    used += cols;
    return precond_from_panels(Om, Y, d, used, shs, mant_bits_of(Ain), P, st);
  };
  for (;;) {
    NYS_TRY(add_block(m));
    if ((P->lam.back() + rho) / rho <= ada_tol) break;
    m = s0;
    s0 = 2 * s0;
    if (s0 > smax) {
      s0 = s0 - m;
      m = smax - s0;
      if (m > 0) NYS_TRY(add_block(m));
      break;
    }
  }
  *used_out = used;
  return NYS_OK;
}

// A helper pass y = A^T phi(.) issued on a side stream and joined later (its buffers are
// allocated on the main stream before the fork and stay valid until the join).  With no side
// stream it runs on the main stream.
struct SidePass {
  cudaStream_t side = nullptr, main = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  void* part = nullptr;
  double* lp = nullptr;
  int* dstat = nullptr;
  ApassArgs a;
  ApassPlan plan;
  ~SidePass() {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (part) cudaFreeAsync(part, main);
    if (lp) cudaFreeAsync(lp, main);
    if (dstat) cudaFreeAsync(dstat, main);
  }
  nys_status start(const nys_matrix* A, int mode, const double* b, void* y, cudaStream_t side_st, cudaStream_t st) {
    main = st;
    side = side_st ? side_st : st;
    apass_plan(A, &plan);
    NYS_CU(cudaMallocAsync(&part, apass_partial_bytes(A, plan), st));
    NYS_CU(cudaMallocAsync((void**)&lp, plan.grid * sizeof(double), st));
    NYS_CU(cudaMallocAsync((void**)&dstat, sizeof(int), st));
    NYS_CU(cudaMemsetAsync(dstat, 0, sizeof(int), st));
    a.A = A->data;
    a.n = A->n;
    a.d = A->d;
    a.ld = A->ld;
    a.dtype = A->dtype;
    a.col_scale = A->col_scale;
    a.p = nullptr;
    a.D = nullptr;
    a.b = b;
    a.D_out = nullptr;
    a.t_out = nullptr;
    a.mode = mode;
    if (side != st) {
      NYS_CU(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
      NYS_CU(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
      NYS_CU(cudaEventRecord(fork, st));
      NYS_CU(cudaStreamWaitEvent(side, fork, 0));
    }
    NYS_CU(apass_run(a, plan, part, lp, dstat, side));
    ApassArgs ar = a;
    NYS_CU(apass_reduce(ar, plan, part, 0.0, y, nullptr, 0, side));
    if (side != st) NYS_CU(cudaEventRecord(join, side));
    return NYS_OK;
  }
  // Joins the pass; NYS_EINVAL when its result has a NaN or an infinity (a non-finite
  // entry of b or of A reaches A^T b).
  nys_status finish(cudaStream_t st, const void* y, int64_t d, bool f32) {
    if (join) NYS_CU(cudaStreamWaitEvent(st, join, 0));
    NYS_CU(cudaMemsetAsync(lp, 0, sizeof(int), st));
    NYS_CU(any_nonfinite(y, d, f32, reinterpret_cast<int*>(lp), st));
    int hs[2] = {0, 0};
    NYS_CU(cudaMemcpyAsync(&hs[0], dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
    NYS_CU(cudaMemcpyAsync(&hs[1], lp, sizeof(int), cudaMemcpyDeviceToHost, st));
    NYS_CU(cudaStreamSynchronize(st));
    if (hs[0]) return (nys_status)hs[0];
    return hs[1] ? NYS_EINVAL : NYS_OK;
  }
};

// ---------------------------------------------------------------- lasso / elastic-net NysADMM
// mu: H^g = mu I of a quadratic g (0 for the lasso; 1 - gamma for the elastic net of Eq. 6).
// The sketched Hessian is A^T A + mu I (Alg. NysADMM), the PCG matrix A^T A + (mu + rho) I,
// and the right-hand side stays q + rho (z - u) (the H^g x and grad g terms of Eq. ADMMSubProb cancel).
template <typename C>
nys_status lasso_admm(const nys_matrix* A, const nys_matrix* Ain, const double* b, double gamma, double mu,
                      double rho, int rank, double tol, const double* Omega, const nys_opts& o, double* x_out,
                      double* z_out, nys_info* info, cudaStream_t st) {
  const int64_t d = A->d;
  Pool pool(st);
  const bool refine = o.refine && (Ain != A);
  // Sketch on the PCG matrix (App. B; once for a quadratic loss, Thm. NysADMM convergence).
  // With opts.rank_max > rank the sketch size is chosen by Alg. AdaptiveRandNysAppx
  // (Alg. AdaNysADMM); it is fixed for all iterations afterwards.
  const int smax = o.rank_max > 0 ? std::max(o.rank_max, rank) : rank;
  nys_precond_s P;
  struct Guard {
    nys_precond_s* p;
    ~Guard() {
      if (p->U64) cudaFree(p->U64);
      if (p->U32) cudaFree(p->U32);
      if (p->lam_d) cudaFree(p->lam_d);
    }
  } guard{&P};
  double* Om = pool.alloc<double>((size_t)d * smax);
  double* Y = pool.alloc<double>((size_t)d * smax);
  double* q = pool.alloc<double>(d);
  void* ytmp = pool.alloc<unsigned char>(d * 8);
  if (!pool.ok()) return NYS_ENOMEM;
  // q = A^T b does not depend on the sketch: it runs on a side stream while the sketch and
  // the Nystrom core run on `st` (joined before the iterations).  Row-sharded solves keep it
  // on `st` (the reduction callback is ordered on one stream).
  SidePass qpass;
  NYS_TRY(qpass.start(A, MODE_CONST, b, ytmp, shard_comm().fn ? nullptr : side_stream(), st));
  NYS_TRY(omega_panel(Omega, o.seed, d, smax, Om, st));
  const double shs = o.shift_scale > 0 ? o.shift_scale : std::sqrt((double)d);
  if (smax > rank) {
    NYS_TRY(adaptive_sketch(Ain, nullptr, mu, Om, Y, d, rank, smax, o.ada_tol > 0 ? o.ada_tol : 2.0, rho, shs,
                            nullptr, &P, &rank, st));
  } else {
    NYS_TRY(cholqr2(Om, d, rank, st, Ain->dtype != NYS_F64));
    NYS_TRY(sketch_panel(Ain, nullptr, mu, Om, rank, Y, st));
    NYS_TRY(precond_from_panels(Om, Y, d, rank, shs, mant_bits_of(Ain), &P, st));
  }
  PrecondView view;
  C* cbuf = pool.alloc<C>(rank);
  if (!pool.ok()) return NYS_ENOMEM;
  {
    PhaseTimer pt("precond view", st);
    NYS_TRY(precond_view<C>(&P, rho, cbuf, st, &view));
  }

  double* x = pool.alloc<double>(d);
  double* z = pool.alloc<double>(d);
  double* u = pool.alloc<double>(d);
  double* yres = pool.alloc<double>(d);
  C* xc = pool.alloc<C>(d);
  C* rc = pool.alloc<C>(d);
  float* xA32 = pool.alloc<float>(d);
  const int K = std::max(1, o.admm_maxit);
  const int nb = admm_blocks(d);
  double* part5 = pool.alloc<double>((size_t)nb * 5);
  double* rp = pool.alloc<double>(K);
  double* rd = pool.alloc<double>(K);
  double* eps_next = pool.alloc<double>(1);
  int* stop = pool.alloc<int>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  NYS_CU(cudaMemsetAsync(x, 0, d * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(z, 0, d * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(u, 0, d * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(xc, 0, d * sizeof(C), st));
  NYS_CU(cudaMemsetAsync(stop, 0, sizeof(int), st));

  // q = A^T b: join the side pass
  {
    PhaseTimer pt("q = A^T b (join)", st);
    NYS_TRY(qpass.finish(st, ytmp, d, A->dtype != NYS_F64));
    NYS_TRY(to_f64(A, ytmp, q, d, st));
    NYS_TRY(shard_sum(q, d, NYS_F64, st));
  }

  PcgProblem pb;
  pb.A = Ain;
  pb.D = nullptr;
  pb.rho = rho + mu;
  apass_plan(Ain, &pb.plan);
  const int maxit = o.pcg_maxit > 0 ? o.pcg_maxit : (int)std::min<int64_t>(d, 1000);
  if (o.device_loop && (!refine || A->dtype == NYS_F64)) {
    // device-side loop: one CUDA graph launch for all K iterations
    GraphLoopArgs g;
    g.pb = pb;
    g.P = view;
    if (refine) {
      g.Aref = A;
      apass_plan(A, &g.plan_ref);
    }
    g.b = b;
    g.yres = yres;
    g.x = x;
    g.z = z;
    g.u = u;
    g.q = q;
    g.xc = xc;
    g.rc = rc;
    C* hx = pool.alloc<C>(d);
    int* pcg_it = pool.alloc<int>(K);
    if (!pool.ok()) return NYS_ENOMEM;
    g.hx = hx;
    g.gamma = gamma;
    g.rho = rho;
    g.mu = mu;
    g.K = K;
    g.eps_abs = o.eps_abs;
    g.eps_rel = o.eps_rel;
    g.tol = tol;
    g.tol_floor = (refine && sizeof(C) == 4) ? 1e-6 : 0.0;
    g.tol_mode = o.pcg_tol_mode;
    g.maxit = maxit;
    g.fixed_host = o.pcg_fixed_iters;
    g.hx_refresh = std::max(0, o.hx_refresh);
    g.ztrace = o.z_trace;
    g.rp = rp;
    g.rd = rd;
    g.pcg_it = pcg_it;
    g.warm = reinterpret_cast<const nys_mlp_s*>(o.warm_model);
    g.warm_record = o.warm_record;
    GraphLoopResult gr;
    nys_status gs = admm_graph_run<C>(g, st, &gr);
    if (gs != NYS_OK) return gs;
    const int done_k = std::min(gr.admm_iters, K);
    std::vector<int> its(std::max(1, done_k));
    if (done_k > 0) NYS_CU(cudaMemcpyAsync(its.data(), pcg_it, done_k * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (x_out) NYS_CU(cudaMemcpyAsync(x_out, x, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (z_out) NYS_CU(cudaMemcpyAsync(z_out, z, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (info && done_k > 0) {
      NYS_CU(cudaMemcpyAsync(&info->r_p, rp + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      NYS_CU(cudaMemcpyAsync(&info->r_d, rd + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    NYS_CU(cudaStreamSynchronize(st));
    int total = 0;
    bool capped = false;
    for (int i = 0; i < done_k; ++i) {
      if (o.pcg_trace) o.pcg_trace[i] = its[i];
      total += its[i];
      const int cap_i = o.pcg_fixed_iters ? o.pcg_fixed_iters[i] : maxit;
      if (!o.pcg_fixed_iters && its[i] >= cap_i) capped = true;
    }
    const nys_status result = gr.breakdown ? NYS_EBREAKDOWN : (capped ? NYS_ENOCONV : NYS_OK);
    if (info) {
      info->admm_iters = done_k;
      info->pcg_iters_total = total;
      info->final_rank = rank;
      info->status = result;
      info->nu = P.nu;
      info->emp_cond = P.lam.empty() ? 1.0 : (P.lam.back() + rho) / rho;
    }
    return result;
  }
  int total_pcg = 0;
  nys_status result = NYS_OK;
  int k = 0;
  for (; k < K; ++k) {
    PcgParams prm;
    prm.maxit = maxit;
    prm.tol = sched_tol(o.pcg_tol_mode, tol, k);
    prm.tol_abs = o.pcg_tol_mode == NYS_TOL_ABS;
    if (o.pcg_tol_mode == NYS_TOL_SQRT_RPRD && k > 0) prm.dev_tol = eps_next;
    if (o.pcg_fixed_iters) prm.fixed = o.pcg_fixed_iters[k];
    if (refine) {
      // exact residual of the x-subproblem at the current x with the FP64 problem matrix
      const void* xa = x;
      if (A->dtype != NYS_F64) {
        NYS_CU(convert_f64_to_f32(x, xA32, d, st));
        xa = xA32;
      }
      NYS_TRY(aux_pass(A, MODE_RESID, xa, b, nullptr, nullptr, ytmp, nullptr, st));
      NYS_TRY(to_f64(A, ytmp, yres, d, st));
      NYS_TRY(shard_sum(yres, d, NYS_F64, st));
      NYS_CU(admm_rhs<C>(d, q, z, u, rho, x, yres, rc, st, mu));
      NYS_CU(cudaMemsetAsync(xc, 0, d * sizeof(C), st));
      prm.x0_zero = true;
      if (sizeof(C) == 4 && !prm.tol_abs) prm.tol = std::max(prm.tol, 1e-6);
    } else {
      NYS_CU(admm_rhs<C>(d, q, z, u, rho, nullptr, nullptr, rc, st));
      prm.x0_zero = (k == 0);
    }
    int it = 0;
    nys_status s = pcg_run<C>(pb, view, rc, xc, prm, st, &it, nullptr);
    total_pcg += it;
    if (o.pcg_trace) o.pcg_trace[k] = it;
    if (s == NYS_ENOCONV) {
      result = NYS_ENOCONV;
    } else if (s != NYS_OK) {
      result = s;
      break;
    }
    double* zt = o.z_trace ? o.z_trace + (int64_t)k * d : nullptr;
    NYS_CU(admm_zu<C>(d, xc, refine ? 1 : 0, x, z, u, gamma / rho, zt, part5, st));
    NYS_CU(admm_scalar(d, part5, rho, k, rp, rd, eps_next, o.eps_abs, o.eps_rel, stop, st));
    if (o.eps_rel > 0) {
      int stop_h = 0;
      NYS_CU(cudaMemcpyAsync(&stop_h, stop, sizeof(int), cudaMemcpyDeviceToHost, st));
      NYS_CU(cudaStreamSynchronize(st));
      if (stop_h) {
        ++k;
        break;
      }
    }
  }
  const int done_k = std::min(k, K);
  if (x_out) NYS_CU(cudaMemcpyAsync(x_out, x, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (z_out) NYS_CU(cudaMemcpyAsync(z_out, z, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (info) {
    info->admm_iters = done_k;
    info->pcg_iters_total = total_pcg;
    info->final_rank = rank;
    info->status = result;
    info->nu = P.nu;
    info->emp_cond = P.lam.empty() ? 1.0 : (P.lam.back() + rho) / rho;
    if (done_k > 0) {
      NYS_CU(cudaMemcpyAsync(&info->r_p, rp + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      NYS_CU(cudaMemcpyAsync(&info->r_d, rd + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
  }
  NYS_CU(cudaStreamSynchronize(st));
  return result;
}

// ---------------------------------------------------------------- lasso regularisation path (k gammas)
template <typename C>
nys_status lasso_path(const nys_matrix* A, const nys_matrix* Ain, const double* b, const double* gammas, int k,
                      double rho, int rank, double tol, const double* Omega, const nys_opts& o, double* X_out,
                      double* Z_out, nys_info* info, int32_t* iters_out, cudaStream_t st) {
  const int64_t d = A->d;
  Pool pool(st);
  nys_precond_s P;
  struct Guard {
    nys_precond_s* p;
    ~Guard() {
      if (p->U64) cudaFree(p->U64);
      if (p->U32) cudaFree(p->U32);
      if (p->lam_d) cudaFree(p->lam_d);
    }
  } guard{&P};
  double* Om = pool.alloc<double>((size_t)d * rank);
  double* Y = pool.alloc<double>((size_t)d * rank);
  if (!pool.ok()) return NYS_ENOMEM;
  NYS_TRY(omega_panel(Omega, o.seed, d, rank, Om, st));
  NYS_TRY(cholqr2(Om, d, rank, st, Ain->dtype != NYS_F64));
  NYS_TRY(sketch_panel(Ain, nullptr, 0.0, Om, rank, Y, st));
  const double shs = o.shift_scale > 0 ? o.shift_scale : std::sqrt((double)d);
  NYS_TRY(precond_from_panels(Om, Y, d, rank, shs, mant_bits_of(Ain), &P, st));
  C* cbuf = pool.alloc<C>(rank);
  const int64_t len = d * k;
  double* X = pool.alloc<double>(len);
  double* Z = pool.alloc<double>(len);
  double* Uu = pool.alloc<double>(len);
  double* q = pool.alloc<double>(d);
  double* kappa = pool.alloc<double>(k);
  C* Xc = pool.alloc<C>(len);
  C* Rc = pool.alloc<C>(len);
  void* ytmp = pool.alloc<unsigned char>(d * 8);
  double* part = pool.alloc<double>((size_t)batched_zu_blocks(d) * k * 2);
  if (!pool.ok()) return NYS_ENOMEM;
  PrecondView view;
  NYS_TRY(precond_view<C>(&P, rho, cbuf, st, &view));
  std::vector<double> kap(k);
  for (int c = 0; c < k; ++c) kap[c] = gammas[c] / rho;
  NYS_CU(cudaMemcpyAsync(kappa, kap.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
  NYS_CU(cudaMemsetAsync(X, 0, len * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(Z, 0, len * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(Uu, 0, len * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(Xc, 0, len * sizeof(C), st));
  NYS_TRY(aux_pass(A, MODE_CONST, nullptr, b, nullptr, nullptr, ytmp, nullptr, st));
  NYS_TRY(to_f64(A, ytmp, q, d, st));
  PcgProblem pb;
  pb.A = Ain;
  pb.D = nullptr;
  pb.rho = rho;
  apass_plan(Ain, &pb.plan);
  const int maxit = o.pcg_maxit > 0 ? o.pcg_maxit : (int)std::min<int64_t>(d, 1000);
  const int K = std::max(1, o.admm_maxit);
  nys_status result = NYS_OK;
  std::vector<int> its, tot(k, 0);
  int nbz = 0;
  for (int it = 0; it < K; ++it) {
    NYS_CU(batched_rhs<C>(d, k, q, Z, Uu, rho, Rc, st));
    PcgParams prm;
    prm.tol = sched_tol(o.pcg_tol_mode, tol, it);
    prm.tol_abs = o.pcg_tol_mode == NYS_TOL_ABS;
    prm.maxit = maxit;
    prm.x0_zero = it == 0;
    if (o.pcg_fixed_iters) prm.fixed = o.pcg_fixed_iters[it];
    nys_status s = batched_pcg_run<C>(pb, view, Rc, Xc, k, prm, st, &its);
    if (s == NYS_ENOCONV) result = NYS_ENOCONV;
    else if (s != NYS_OK) return s;
    for (int c = 0; c < k; ++c) tot[c] += its[c];
    NYS_CU(batched_zu<C>(d, k, Xc, X, Z, Uu, kappa, part, &nbz, st));
  }
  if (X_out) NYS_CU(cudaMemcpyAsync(X_out, X, len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (Z_out) NYS_CU(cudaMemcpyAsync(Z_out, Z, len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  std::vector<double> hp((size_t)nbz * k * 2);
  if (nbz) NYS_CU(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  NYS_CU(cudaStreamSynchronize(st));
  if (iters_out)
    for (int c = 0; c < k; ++c) iters_out[c] = tot[c];
  if (info) {
    double rp = 0, rd = 0;  // worst column
    for (int c = 0; c < k; ++c) {
      double a0 = 0, a1 = 0;
      for (int bb = 0; bb < nbz; ++bb) {
        a0 += hp[((size_t)bb * k + c) * 2];
        a1 += hp[((size_t)bb * k + c) * 2 + 1];
      }
      rp = std::max(rp, std::sqrt(a0));
      rd = std::max(rd, rho * std::sqrt(a1));
    }
    int total = 0;
    for (int c = 0; c < k; ++c) total += tot[c];
    info->admm_iters = K;
    info->pcg_iters_total = total;
    info->final_rank = rank;
    info->status = result;
    info->r_p = rp;
    info->r_d = rd;
    info->nu = P.nu;
    info->emp_cond = (P.lam.back() + rho) / rho;
  }
  return result;
}

// ---------------------------------------------------------------- batch of independent lasso instances
// Every instance is sketched eagerly, then all device-side ADMM loops run as parallel
// branches of ONE CUDA graph launch.
template <typename C>
nys_status lasso_batch(int count, const nys_lasso_instance* in, double rho, double tol, const nys_opts& o,
                       nys_info* infos, cudaStream_t st) {
  Pool pool(st);
  std::vector<nys_precond_s> Ps(count);
  struct Guard {
    std::vector<nys_precond_s>* v;
    ~Guard() {
      for (auto& p : *v) {
        if (p.U64) cudaFree(p.U64);
        if (p.U32) cudaFree(p.U32);
        if (p.lam_d) cudaFree(p.lam_d);
      }
    }
  } guard{&Ps};
  const int K = std::max(1, o.admm_maxit);
  std::vector<GraphLoopArgs> gs(count);
  std::vector<int*> pcg_its(count);
  for (int i = 0; i < count; ++i) {
    const nys_matrix* A = in[i].A;
    const int64_t d = A->d;
    const int rank = in[i].rank;
    double* Om = pool.alloc<double>((size_t)d * rank);
    double* Y = pool.alloc<double>((size_t)d * rank);
    C* cbuf = pool.alloc<C>(rank);
    double* x = pool.alloc<double>(d);
    double* z = pool.alloc<double>(d);
    double* u = pool.alloc<double>(d);
    double* q = pool.alloc<double>(d);
    C* xc = pool.alloc<C>(d);
    C* rc = pool.alloc<C>(d);
    C* hx = pool.alloc<C>(d);
    void* ytmp = pool.alloc<unsigned char>(d * 8);
    double* rp = pool.alloc<double>(K);
    double* rd = pool.alloc<double>(K);
    int* pit = pool.alloc<int>(K);
    if (!pool.ok()) return NYS_ENOMEM;
    NYS_CU(cudaMemcpyAsync(Om, in[i].Omega, (size_t)d * rank * sizeof(double), cudaMemcpyDeviceToDevice, st));
    NYS_TRY(cholqr2(Om, d, rank, st, A->dtype != NYS_F64));
    NYS_TRY(sketch_panel(A, nullptr, 0.0, Om, rank, Y, st));
    const double shs = o.shift_scale > 0 ? o.shift_scale : std::sqrt((double)d);
    NYS_TRY(precond_from_panels(Om, Y, d, rank, shs, mant_bits_of(A), &Ps[i], st));
    PrecondView view;
    NYS_TRY(precond_view<C>(&Ps[i], rho, cbuf, st, &view));
    NYS_CU(cudaMemsetAsync(x, 0, d * sizeof(double), st));
    NYS_CU(cudaMemsetAsync(z, 0, d * sizeof(double), st));
    NYS_CU(cudaMemsetAsync(u, 0, d * sizeof(double), st));
    NYS_CU(cudaMemsetAsync(xc, 0, d * sizeof(C), st));
    NYS_TRY(aux_pass(A, MODE_CONST, nullptr, in[i].b, nullptr, nullptr, ytmp, nullptr, st));
    NYS_TRY(to_f64(A, ytmp, q, d, st));
    GraphLoopArgs& g = gs[i];
    g.pb.A = A;
    g.pb.D = nullptr;
    g.pb.rho = rho;
    apass_plan(A, &g.pb.plan);
    g.P = view;
    g.b = in[i].b;
    g.x = x;
    g.z = z;
    g.u = u;
    g.q = q;
    g.xc = xc;
    g.rc = rc;
    g.hx = hx;
    g.gamma = in[i].gamma;
    g.rho = rho;
    g.K = K;
    g.eps_abs = o.eps_abs;
    g.eps_rel = o.eps_rel;
    g.tol = tol;
    g.tol_mode = o.pcg_tol_mode;
    g.maxit = o.pcg_maxit > 0 ? o.pcg_maxit : (int)std::min<int64_t>(d, 1000);
    g.fixed_host = o.pcg_fixed_iters;
    g.hx_refresh = std::max(0, o.hx_refresh);
    g.rp = rp;
    g.rd = rd;
    g.pcg_it = pit;
    pcg_its[i] = pit;
  }
  std::vector<GraphInstance> insts(count);
  std::vector<GraphLoopResult> res(count);
  NYS_TRY(admm_graph_run_many<C>(gs.data(), count, st, insts.data(), res.data()));
  nys_status worst = NYS_OK;
  for (int i = 0; i < count; ++i) {
    const int64_t d = in[i].A->d;
    const int done_k = std::min(res[i].admm_iters, K);
    std::vector<int> its(std::max(1, done_k));
    if (done_k > 0) NYS_CU(cudaMemcpyAsync(its.data(), pcg_its[i], done_k * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (in[i].x_out) NYS_CU(cudaMemcpyAsync(in[i].x_out, gs[i].x, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (in[i].z_out) NYS_CU(cudaMemcpyAsync(in[i].z_out, gs[i].z, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    nys_info inf;
    std::memset(&inf, 0, sizeof(inf));
    if (done_k > 0) {
      NYS_CU(cudaMemcpyAsync(&inf.r_p, gs[i].rp + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      NYS_CU(cudaMemcpyAsync(&inf.r_d, gs[i].rd + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    NYS_CU(cudaStreamSynchronize(st));
    int total = 0;
    for (int j = 0; j < done_k; ++j) total += its[j];
    inf.admm_iters = done_k;
    inf.pcg_iters_total = total;
    inf.final_rank = in[i].rank;
    inf.status = res[i].breakdown ? NYS_EBREAKDOWN : NYS_OK;
    inf.nu = Ps[i].nu;
    inf.emp_cond = (Ps[i].lam.back() + rho) / rho;
    if (res[i].breakdown) worst = NYS_EBREAKDOWN;
    if (infos) infos[i] = inf;
  }
  return worst;
}

// ---------------------------------------------------------------- logistic (Sec. 3.2) + AdaRandNysAppx (App. C)
template <typename C>
nys_status logistic_admm(const nys_matrix* A, const nys_matrix* Ain, const double* b, double gamma, double rho,
                         int rank, double tol, const double* Omega, const nys_opts& o, double* x_out,
                         double* z_out, nys_info* info, cudaStream_t st) {
  const int64_t d = A->d, n = A->n;
  const int smax = o.rank_max > 0 ? std::max(o.rank_max, rank) : rank;
  const double ada_tol = o.ada_tol > 0 ? o.ada_tol : 2.0;
  const double shs = o.shift_scale > 0 ? o.shift_scale : std::sqrt((double)d);
  Pool pool(st);
  double* Om = pool.alloc<double>((size_t)d * smax);
  double* Y = pool.alloc<double>((size_t)d * smax);
  double* Dw = pool.alloc<double>(n);
  C* cbuf = pool.alloc<C>(smax);
  double* x = pool.alloc<double>(d);
  double* z = pool.alloc<double>(d);
  double* u = pool.alloc<double>(d);
  double* q = pool.alloc<double>(d);
  C* xc = pool.alloc<C>(d);
  C* rc = pool.alloc<C>(d);
  void* ytmp = pool.alloc<unsigned char>(d * 8);
  float* xA32 = pool.alloc<float>(d);
  const int K = std::max(1, o.admm_maxit);
  const int nb = admm_blocks(d);
  double* part5 = pool.alloc<double>((size_t)nb * 5);
  double* rp = pool.alloc<double>(K);
  double* rd = pool.alloc<double>(K);
  double* eps_next = pool.alloc<double>(1);
  int* stop = pool.alloc<int>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  NYS_TRY(omega_panel(Omega, o.seed, d, smax, Om, st));
  NYS_CU(cudaMemsetAsync(x, 0, d * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(z, 0, d * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(u, 0, d * sizeof(double), st));
  NYS_CU(cudaMemsetAsync(xc, 0, d * sizeof(C), st));
  NYS_CU(cudaMemsetAsync(stop, 0, sizeof(int), st));

  nys_precond_s P;
  struct Guard {
    nys_precond_s* p;
    ~Guard() {
      if (p->U64) cudaFree(p->U64);
      if (p->U32) cudaFree(p->U32);
      if (p->lam_d) cudaFree(p->lam_d);
    }
  } guard{&P};

  PcgProblem pb;
  pb.A = Ain;
  pb.D = Dw;
  pb.rho = rho;
  apass_plan(Ain, &pb.plan);
  const int maxit = o.pcg_maxit > 0 ? o.pcg_maxit : (int)std::min<int64_t>(d, 1000);
  int total_pcg = 0, cur_rank = 0;
  nys_status result = NYS_OK;
  // the curvature D changes every iteration but A does not: prepare its tensor-core
  // operands once for all re-sketches
  TcPrepared tcp;
  const TcPrepared* tcpp = nullptr;
  if (sketch_tc_supported(Ain)) {
    void* tcs = pool.alloc<unsigned char>(tc_prepare_bytes(Ain));
    if (!pool.ok()) return NYS_ENOMEM;
    NYS_CU(tc_prepare(Ain, tcs, &tcp, st));
    tcpp = &tcp;
  }
  int k = 0;
  for (; k < K; ++k) {
    // t = A x~, w, and the right-hand side A^T (w t + b01 - sigma(t)) in one pass (Sec. 3.2)
    const void* xa = x;
    if (A->dtype != NYS_F64) {
      NYS_CU(convert_f64_to_f32(x, xA32, d, st));
      xa = xA32;
    }
    NYS_TRY(aux_pass(A, MODE_LOGIT, xa, b, Dw, nullptr, ytmp, nullptr, st));
    NYS_TRY(to_f64(A, ytmp, q, d, st));
    if (k == 0) {
      NYS_TRY(adaptive_sketch(Ain, Dw, 0.0, Om, Y, d, rank, smax, ada_tol, rho, shs, tcpp, &P, &cur_rank, st));
    } else if (o.resketch_every > 0 && k % o.resketch_every == 0) {
      // same orthonormal blocks, new curvature D
      NYS_TRY(sketch_panel(Ain, Dw, 0.0, Om, cur_rank, Y, st, tcpp));
      NYS_TRY(precond_from_panels(Om, Y, d, cur_rank, shs, mant_bits_of(Ain), &P, st));
    }
    PrecondView view;
    NYS_TRY(precond_view<C>(&P, rho, cbuf, st, &view));
    NYS_CU(admm_rhs<C>(d, q, z, u, rho, nullptr, nullptr, rc, st));
    PcgParams prm;
    prm.maxit = maxit;
    prm.tol = sched_tol(o.pcg_tol_mode, tol, k);
    prm.tol_abs = o.pcg_tol_mode == NYS_TOL_ABS;
    if (o.pcg_tol_mode == NYS_TOL_SQRT_RPRD && k > 0) prm.dev_tol = eps_next;
    if (o.pcg_fixed_iters) prm.fixed = o.pcg_fixed_iters[k];
    prm.x0_zero = (k == 0);
    int it = 0;
    nys_status s = pcg_run<C>(pb, view, rc, xc, prm, st, &it, nullptr);
    total_pcg += it;
    if (o.pcg_trace) o.pcg_trace[k] = it;
    if (s == NYS_ENOCONV) {
      result = NYS_ENOCONV;
    } else if (s != NYS_OK) {
      result = s;
      break;
    }
    double* zt = o.z_trace ? o.z_trace + (int64_t)k * d : nullptr;
    NYS_CU(admm_zu<C>(d, xc, 0, x, z, u, gamma / rho, zt, part5, st));
    NYS_CU(admm_scalar(d, part5, rho, k, rp, rd, eps_next, o.eps_abs, o.eps_rel, stop, st));
    if (o.eps_rel > 0) {
      int stop_h = 0;
      NYS_CU(cudaMemcpyAsync(&stop_h, stop, sizeof(int), cudaMemcpyDeviceToHost, st));
      NYS_CU(cudaStreamSynchronize(st));
      if (stop_h) {
        ++k;
        break;
      }
    }
  }
  const int done_k = std::min(k, K);
  if (x_out) NYS_CU(cudaMemcpyAsync(x_out, x, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (z_out) NYS_CU(cudaMemcpyAsync(z_out, z, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (info) {
    info->admm_iters = done_k;
    info->pcg_iters_total = total_pcg;
    info->final_rank = cur_rank;
    info->status = result;
    info->nu = P.nu;
    info->emp_cond = P.lam.empty() ? 1.0 : (P.lam.back() + rho) / rho;
    if (done_k > 0) {
      NYS_CU(cudaMemcpyAsync(&info->r_p, rp + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      NYS_CU(cudaMemcpyAsync(&info->r_d, rd + done_k - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
  }
  NYS_CU(cudaStreamSynchronize(st));
  return result;
}

// ---------------------------------------------------------------- objective helpers
// g: gradient of the loss term; mu x (g = mu/2 ||x||^2, elastic net) is added to it here
__global__ void obj_vec_kernel(int64_t d, const double* __restrict__ x, const double* __restrict__ g, double gamma,
                               double mu, double* part4) {
  __shared__ double sh[kVecThreads / 32];
  double l1 = 0, l2 = 0, kk = 0, gm = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    const double xj = x[j], gj = fma(mu, xj, g[j]);
    l1 += fabs(xj);
    l2 += xj * xj;
    const double v = xj - gj;
    const double mag = fabs(v) - gamma;
    const double pj = mag > 0 ? copysign(mag, v) : 0.0;
    kk += (xj - pj) * (xj - pj);
    gm = fmax(gm, fabs(gj));
  }
  l1 = block_sum<kVecThreads>(l1, sh);
  l2 = block_sum<kVecThreads>(l2, sh);
  kk = block_sum<kVecThreads>(kk, sh);
  for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  __shared__ double mx[kVecThreads / 32];
  if ((threadIdx.x & 31) == 0) mx[threadIdx.x >> 5] = gm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0;
    for (int i = 0; i < kVecThreads / 32; ++i) m = fmax(m, mx[i]);
    double* o = part4 + (int64_t)blockIdx.x * 4;
    o[0] = l1;
    o[1] = l2;
    o[2] = kk;
    o[3] = m;
  }
}

__global__ void obj_row_kernel(int64_t n, const double* __restrict__ t, const double* __restrict__ b, double* part2) {
  __shared__ double sh[kVecThreads / 32];
  double bres = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bres += b[i] * (t[i] - b[i]);
    bb += b[i] * b[i];
  }
  bres = block_sum<kVecThreads>(bres, sh);
  bb = block_sum<kVecThreads>(bb, sh);
  if (threadIdx.x == 0) {
    part2[2 * blockIdx.x] = bres;
    part2[2 * blockIdx.x + 1] = bb;
  }
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

void nys_opts_default(nys_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->shift_scale = 0.0;
  o->pcg_tol_mode = NYS_TOL_REL;
  o->pcg_maxit = 0;
  o->pcg_fixed_iters = nullptr;
  o->admm_maxit = 200;
  o->eps_abs = 0.0;
  o->eps_rel = 0.0;
  o->A_inner = nullptr;
  o->refine = 1;
  o->z_trace = nullptr;
  o->rank_max = 0;
  o->ada_tol = 2.0;
  o->resketch_every = 1;
  o->stream = nullptr;
  o->device_loop = 1;
  o->hx_refresh = 0;
  o->warm_model = nullptr;
  o->warm_record = nullptr;
  o->seed = 0;
  o->allreduce = nullptr;
  o->allreduce_ctx = nullptr;
  o->pcg_trace = nullptr;
}

nys_status nys_gaussian_test_matrix(uint64_t seed, int64_t d, int32_t s, double* Omega, void* stream) {
  if (d < 1 || s < 1 || !Omega) return NYS_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  NYS_CU(gaussian_panel(seed, d, s, Omega, st));
  NYS_CU(cudaStreamSynchronize(st));
  return NYS_OK;
}

const char* nys_strerror(int32_t s) {
  switch (s) {
    case NYS_OK: return "ok";
    case NYS_EINVAL: return "invalid argument";
    case NYS_ENOTSPD: return "Nystrom core matrix not positive definite after shift retries";
    case NYS_EBREAKDOWN: return "PCG breakdown (p^T (H + rho I) p <= 0 or not finite)";
    case NYS_ENOCONV: return "iteration cap reached before the tolerance";
    case NYS_ETIMEOUT: return "device-side wait exceeded its bound";
    case NYS_ECUDA: return "CUDA runtime error";
    case NYS_ENOMEM: return "device memory allocation failed";
    default: return "unknown status";
  }
}

nys_status nys_hmatvec(const nys_matrix* A, const double* D, double rho, const void* p, void* y, void* stream) {
  NYS_TRY(check_hmatvec_args(A, rho, p, y));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return A->dtype == NYS_F64 ? hmatvec_t<double>(A, D, rho, p, y, st) : hmatvec_t<float>(A, D, rho, p, y, st);
}

nys_status nys_sketch(const nys_matrix* A, const double* D, double diag_shift, int32_t s, const double* Omega,
                      const nys_opts* opts, nys_precond* out) {
  if (!out) return NYS_EINVAL;
  *out = nullptr;
  NYS_TRY(check_matrix(A));
  if (s < 1 || s > A->d || s > kMaxRank || !is_fin(diag_shift) || diag_shift < 0) return NYS_EINVAL;
  cudaStream_t st = stream_of(opts);
  const int64_t d = A->d;
  ShardScope shard(opts);
  nys_precond_s* P = new (std::nothrow) nys_precond_s();
  if (!P) return NYS_ENOMEM;
  nys_status r;
  {
    Pool pool(st);
    double* Om = pool.alloc<double>((size_t)d * s);
    double* Y = pool.alloc<double>((size_t)d * s);
    if (!pool.ok()) {
      precond_free(P);
      return NYS_ENOMEM;
    }
    r = omega_panel(Omega, opts ? opts->seed : 0, d, s, Om, st);
    if (r == NYS_OK) r = cholqr2(Om, d, s, st, A->dtype != NYS_F64);
    if (r == NYS_OK) r = sketch_panel(A, D, diag_shift, Om, s, Y, st);
    const double shs = (opts && opts->shift_scale > 0) ? opts->shift_scale : std::sqrt((double)d);
    if (r == NYS_OK) r = precond_from_panels(Om, Y, d, s, shs, mant_bits_of(A), P, st);
    cudaStreamSynchronize(st);
  }
  if (r != NYS_OK) {
    precond_free(P);
    return r;
  }
  *out = P;
  return NYS_OK;
}

nys_status nys_precond_get(nys_precond P, double* U_out, double* lam_out, int32_t* s_out, int64_t* d_out,
                           double* nu_out, void* stream) {
  if (!P) return NYS_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (U_out)
    NYS_CU(cudaMemcpyAsync(U_out, P->U64, (size_t)P->d * P->s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (lam_out) std::memcpy(lam_out, P->lam.data(), P->s * sizeof(double));
  if (s_out) *s_out = P->s;
  if (d_out) *d_out = P->d;
  if (nu_out) *nu_out = P->nu;
  NYS_CU(cudaStreamSynchronize(st));
  return NYS_OK;
}

nys_status nys_precond_apply(nys_precond P, double rho, const void* V, void* Yv, int64_t k, int32_t dtype,
                             void* stream) {
  if (!P || !V || !Yv || k < 1 || !(rho > 0) || !is_fin(rho)) return NYS_EINVAL;
  if (dtype != NYS_F64 && dtype != NYS_F32) return NYS_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Pool pool(st);
  void* cbuf = pool.alloc<double>(P->s);
  if (!pool.ok()) return NYS_ENOMEM;
  PrecondView view;
  if (dtype == NYS_F64) {
    NYS_TRY(precond_view<double>(P, rho, (double*)cbuf, st, &view));
    return precond_apply_run<double>(view, P->d, (const double*)V, (double*)Yv, k, st);
  }
  NYS_TRY(precond_view<float>(P, rho, (float*)cbuf, st, &view));
  return precond_apply_run<float>(view, P->d, (const float*)V, (float*)Yv, k, st);
}

nys_status pcg_solve(const nys_matrix* A, const double* D, double rho, nys_precond P, const void* r, void* x,
                     double tol, const nys_opts* opts, int32_t* iters, double* resnorm) {
  NYS_TRY(check_matrix(A));
  if (!r || !x || !(rho > 0) || !is_fin(rho) || !(tol >= 0) || !is_fin(tol)) return NYS_EINVAL;
  if (P && P->d != A->d) return NYS_EINVAL;
  nys_opts o;
  if (opts) o = *opts;
  else nys_opts_default(&o);
  // no ADMM iteration here: the schedules of Sec. 5 do not apply
  if (o.pcg_tol_mode < NYS_TOL_REL || o.pcg_tol_mode >= NYS_TOL_RNORM_POW) return NYS_EINVAL;
  cudaStream_t st = stream_of(&o);
  ShardScope shard(&o);
  PcgProblem pb;
  pb.A = A;
  pb.D = D;
  pb.rho = rho;
  apass_plan(A, &pb.plan);
  PcgParams prm;
  prm.tol = tol;
  prm.tol_abs = o.pcg_tol_mode == NYS_TOL_ABS;
  prm.maxit = o.pcg_maxit > 0 ? o.pcg_maxit : (int)std::min<int64_t>(A->d, 1000);
  if (o.pcg_fixed_iters) prm.fixed = o.pcg_fixed_iters[0];
  Pool pool(st);
  void* cbuf = pool.alloc<double>(P ? P->s : 1);
  int* bad = pool.alloc<int>(1);
  if (!pool.ok()) return NYS_ENOMEM;
  {
    // a NaN or an infinity in r or in x0 is a bad argument, not a breakdown of the iteration
    int bad_h = 0;
    NYS_CU(cudaMemsetAsync(bad, 0, sizeof(int), st));
    NYS_CU(any_nonfinite(r, A->d, A->dtype != NYS_F64, bad, st));
    NYS_CU(any_nonfinite(x, A->d, A->dtype != NYS_F64, bad, st));
    NYS_CU(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    NYS_CU(cudaStreamSynchronize(st));
    if (bad_h) return NYS_EINVAL;
  }
  PrecondView view;
  int it = 0;
  nys_status s;
  if (A->dtype == NYS_F64) {
    NYS_TRY(precond_view<double>(P, rho, (double*)cbuf, st, &view));
    s = pcg_run<double>(pb, view, (const double*)r, (double*)x, prm, st, &it, resnorm);
  } else {
    NYS_TRY(precond_view<float>(P, rho, (float*)cbuf, st, &view));
    s = pcg_run<float>(pb, view, (const float*)r, (float*)x, prm, st, &it, resnorm);
  }
  if (iters) *iters = it;
  return s;
}

nys_status nysadmm_solve(int32_t loss, const nys_matrix* A, const double* b, double gamma, double rho, int32_t rank,
                         double tol, const double* Omega, const nys_opts* opts, double* x_out, double* z_out,
                         nys_info* info) {
  NYS_TRY(check_matrix(A));
  if (loss != NYS_LASSO && loss != NYS_LOGISTIC && loss != NYS_ELASTIC_NET) return NYS_EINVAL;
  if (!b || !(gamma >= 0) || !is_fin(gamma) || !(rho > 0) || !is_fin(rho)) return NYS_EINVAL;
  if (loss == NYS_ELASTIC_NET && !(gamma > 0 && gamma <= 1)) return NYS_EINVAL;  // Eq. 6: 0 < gamma <= 1
  if (rank < 1 || rank > A->d || rank > kMaxRank || !(tol >= 0) || !is_fin(tol)) return NYS_EINVAL;
  nys_opts o;
  if (opts) o = *opts;
  else nys_opts_default(&o);
  if (o.admm_maxit < 1) return NYS_EINVAL;
  if (o.rank_max > A->d || o.rank_max > kMaxRank) return NYS_EINVAL;
  if (o.pcg_tol_mode < NYS_TOL_REL || o.pcg_tol_mode > NYS_TOL_RNORM_POW) return NYS_EINVAL;
  // row-sharded solves run the host-driven loop (the device-side graph cannot call back)
  if (o.allreduce && (loss == NYS_LOGISTIC || o.device_loop || o.warm_model || o.warm_record)) return NYS_EINVAL;
  ShardScope shard(&o);
  const nys_matrix* Ain = o.A_inner ? o.A_inner : A;
  if (o.A_inner) {
    NYS_TRY(check_matrix(Ain));
    if (Ain->n != A->n || Ain->d != A->d) return NYS_EINVAL;
  }
  cudaStream_t st = stream_of(&o);
  if (info) std::memset(info, 0, sizeof(*info));
  if (loss == NYS_LASSO || loss == NYS_ELASTIC_NET) {
    const double mu = loss == NYS_ELASTIC_NET ? 1.0 - gamma : 0.0;
    return Ain->dtype == NYS_F64
               ? lasso_admm<double>(A, Ain, b, gamma, mu, rho, rank, tol, Omega, o, x_out, z_out, info, st)
               : lasso_admm<float>(A, Ain, b, gamma, mu, rho, rank, tol, Omega, o, x_out, z_out, info, st);
  }
  return Ain->dtype == NYS_F64 ? logistic_admm<double>(A, Ain, b, gamma, rho, rank, tol, Omega, o, x_out, z_out, info, st)
                               : logistic_admm<float>(A, Ain, b, gamma, rho, rank, tol, Omega, o, x_out, z_out, info, st);
}

nys_status nysadmm_solve_path(const nys_matrix* A, const double* b, const double* gammas, int32_t k, double rho,
                              int32_t rank, double tol, const double* Omega, const nys_opts* opts, double* X_out,
                              double* Z_out, nys_info* info, int32_t* pcg_iters) {
  NYS_TRY(check_matrix(A));
  if (!b || !gammas || k < 1 || k > 4096 || !(rho > 0) || !is_fin(rho)) return NYS_EINVAL;
  for (int c = 0; c < k; ++c)
    if (!(gammas[c] >= 0) || !is_fin(gammas[c])) return NYS_EINVAL;
  if (rank < 1 || rank > A->d || rank > kMaxRank || !(tol >= 0) || !is_fin(tol)) return NYS_EINVAL;
  nys_opts o;
  if (opts) o = *opts;
  else nys_opts_default(&o);
  if (o.pcg_tol_mode < NYS_TOL_REL || o.pcg_tol_mode > NYS_TOL_RNORM_POW) return NYS_EINVAL;
  if (o.allreduce) return NYS_EINVAL;   // the path is not row-sharded
  const nys_matrix* Ain = o.A_inner ? o.A_inner : A;
  if (o.A_inner) {
    NYS_TRY(check_matrix(Ain));
    if (Ain->n != A->n || Ain->d != A->d) return NYS_EINVAL;
  }
  if (A->dtype == NYS_FP8E4M3 || Ain->dtype == NYS_FP8E4M3) return NYS_EINVAL;  // multi-RHS: F64/F32/BF16
  cudaStream_t st = stream_of(&o);
  if (info) std::memset(info, 0, sizeof(*info));
  return Ain->dtype == NYS_F64
             ? lasso_path<double>(A, Ain, b, gammas, k, rho, rank, tol, Omega, o, X_out, Z_out, info, pcg_iters, st)
             : lasso_path<float>(A, Ain, b, gammas, k, rho, rank, tol, Omega, o, X_out, Z_out, info, pcg_iters, st);
}

nys_status nysadmm_solve_batch(int32_t count, const nys_lasso_instance* inst, double rho, double tol,
                               const nys_opts* opts, nys_info* infos) {
  if (count < 1 || count > 4096 || !inst || !(rho > 0) || !is_fin(rho) || !(tol >= 0) || !is_fin(tol))
    return NYS_EINVAL;
  const bool f64 = inst[0].A && inst[0].A->dtype == NYS_F64;
  for (int i = 0; i < count; ++i) {
    NYS_TRY(check_matrix(inst[i].A));
    if ((inst[i].A->dtype == NYS_F64) != f64) return NYS_EINVAL;  // one compute type per batch
    if (inst[i].A->dtype == NYS_FP8E4M3) return NYS_EINVAL;
    if (!inst[i].b || !inst[i].Omega || !(inst[i].gamma >= 0) || !is_fin(inst[i].gamma)) return NYS_EINVAL;
    if (inst[i].rank < 1 || inst[i].rank > inst[i].A->d || inst[i].rank > kMaxRank) return NYS_EINVAL;
  }
  nys_opts o;
  if (opts) o = *opts;
  else nys_opts_default(&o);
  if (o.allreduce) return NYS_EINVAL;   // independent instances are not row-sharded
  if (o.admm_maxit < 1) return NYS_EINVAL;
  if (o.pcg_tol_mode < NYS_TOL_REL || o.pcg_tol_mode > NYS_TOL_RNORM_POW) return NYS_EINVAL;
  cudaStream_t st = stream_of(&o);
  return f64 ? lasso_batch<double>(count, inst, rho, tol, o, infos, st)
             : lasso_batch<float>(count, inst, rho, tol, o, infos, st);
}

nys_status nys_objective(int32_t loss, const nys_matrix* A, const double* b, double gamma, const double* x,
                         double* out, void* stream) {
  NYS_TRY(check_matrix(A));
  if (!b || !x || !out || !(gamma >= 0) || !is_fin(gamma)) return NYS_EINVAL;
  if (loss != NYS_LASSO && loss != NYS_LOGISTIC && loss != NYS_ELASTIC_NET) return NYS_EINVAL;
  if (loss == NYS_ELASTIC_NET && !(gamma > 0 && gamma <= 1)) return NYS_EINVAL;
  const double mu = loss == NYS_ELASTIC_NET ? 1.0 - gamma : 0.0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t d = A->d, n = A->n;
  Pool pool(st);
  double* g = pool.alloc<double>(d);
  double* t = pool.alloc<double>(n);
  void* ytmp = pool.alloc<unsigned char>(d * 8);
  const int nbd = reduce_blocks(d), nbn = reduce_blocks(n);
  double* p4 = pool.alloc<double>((size_t)nbd * 4);
  double* p2 = pool.alloc<double>((size_t)nbn * 2);
  if (!pool.ok()) return NYS_ENOMEM;
  float* x32 = pool.alloc<float>(d);
  if (!pool.ok()) return NYS_ENOMEM;
  const void* xa = x;
  if (A->dtype != NYS_F64) {
    NYS_CU(convert_f64_to_f32(x, x32, d, st));
    xa = x32;
  }
  double lossv = 0.0;
  NYS_TRY(aux_pass(A, loss == NYS_LOGISTIC ? MODE_LGRAD : MODE_RESID, xa, b, nullptr, t, ytmp, &lossv, st));
  NYS_TRY(to_f64(A, ytmp, g, d, st));
  count_launch();
  obj_vec_kernel<<<nbd, kVecThreads, 0, st>>>(d, x, g, gamma, mu, p4);
  NYS_CU(cudaGetLastError());
  count_launch();
  obj_row_kernel<<<nbn, kVecThreads, 0, st>>>(n, t, b, p2);
  NYS_CU(cudaGetLastError());
  std::vector<double> h4((size_t)nbd * 4), h2((size_t)nbn * 2);
  NYS_CU(cudaMemcpyAsync(h4.data(), p4, h4.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  NYS_CU(cudaMemcpyAsync(h2.data(), p2, h2.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  NYS_CU(cudaStreamSynchronize(st));
  double l1 = 0, l2 = 0, kk = 0, gm = 0, bres = 0, bb = 0;
  for (int i = 0; i < nbd; ++i) {
    l1 += h4[4 * i];
    l2 += h4[4 * i + 1];
    kk += h4[4 * i + 2];
    gm = std::max(gm, h4[4 * i + 3]);
  }
  for (int i = 0; i < nbn; ++i) {
    bres += h2[2 * i];
    bb += h2[2 * i + 1];
  }
  const double F = lossv + 0.5 * mu * l2 + gamma * l1;
  out[0] = F;
  if (loss != NYS_LOGISTIC) {
    // lasso dual at the scaled residual; the elastic net as the lasso of the stacked data
    // [A; sqrt(mu) I], [b; 0], whose residual adds -sqrt(mu) x (squared norm mu ||x||^2)
    const double res2 = 2.0 * lossv;
    out[1] = std::sqrt(kk) / (1.0 + std::sqrt(l2) + std::sqrt(res2));
    const double c = gm > gamma ? gamma / gm : 1.0;
    const double dual = -c * bres - 0.5 * c * c * (res2 + mu * l2);
    out[2] = F - dual;
  } else {
    out[1] = gm;
    out[2] = 0.0;
  }
  return NYS_OK;
}

nys_status nys_autotune_apass(const nys_matrix* A, int32_t* rows_out, double* ms_out, void* stream) {
  NYS_TRY(check_matrix(A));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int cand[3];
  const int nc = apass_row_candidates(A, cand);
  if (nc == 0) return NYS_EINVAL;
  const bool f64 = A->dtype == NYS_F64;
  Pool pool(st);
  void* p = pool.alloc<unsigned char>((size_t)A->d * 8);
  int* dstat = pool.alloc<int>(1);
  ApassPlan big;
  apass_plan(A, &big);
  // partials for the largest grid any candidate can use
  void* part = pool.alloc<unsigned char>((size_t)big.dpad * 8 * 256);
  cudaEvent_t e0, e1;
  if (!pool.ok()) return NYS_ENOMEM;
  NYS_CU(cudaMemsetAsync(p, 0, (size_t)A->d * 8, st));
  NYS_CU(cudaMemsetAsync(dstat, 0, sizeof(int), st));
  NYS_CU(cudaEventCreate(&e0));
  NYS_CU(cudaEventCreate(&e1));
  int best = cand[0];
  double best_ms = 1e300;
  for (int c = 0; c < nc; ++c) {
    apass_set_tuned_rows(A, cand[c]);
    ApassPlan plan;
    if (!apass_plan(A, &plan) || plan.grid > 256) continue;
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
    NYS_CU(apass_run(a, plan, part, nullptr, dstat, st, false));  // warm-up
    NYS_CU(cudaEventRecord(e0, st));
    for (int rep = 0; rep < 3; ++rep) NYS_CU(apass_run(a, plan, part, nullptr, dstat, st, false));
    NYS_CU(cudaEventRecord(e1, st));
    NYS_CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    NYS_CU(cudaEventElapsedTime(&ms, e0, e1));
    if (ms / 3.0 < best_ms) {
      best_ms = ms / 3.0;
      best = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)f64;
  apass_set_tuned_rows(A, best);
  // then the row slabs of the warp-specialised float pass, balanced over the CTAs
  double ms_eq = 0.0, ms_split = 0.0;
  NYS_CU(apass_balance_rows(A, p, part, dstat, st, &ms_eq, &ms_split));
  if (ms_split > 0.0 && ms_split < best_ms) best_ms = ms_split;
  if (std::getenv("NYS_TRACE"))
    std::fprintf(stderr, "[nys] autotune: rows %d, pass %.4f ms (equal slabs %.4f ms, balanced %.4f ms)\n", best, best_ms,
                 ms_eq, ms_split);
  if (rows_out) *rows_out = best;
  if (ms_out) *ms_out = best_ms;
  return NYS_OK;
}

void nys_precond_destroy(nys_precond P) { precond_free(P); }

}  // extern "C"
