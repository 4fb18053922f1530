// Internal declarations shared by the CUDA translation units of libnysadmm.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "nysadmm.h"

namespace nys {

constexpr int kApassThreads = 512;       // threads of the fused A-pass CTA
constexpr int kApassThreadsWide = 640;   // float-path CTA for narrow rows (<= 4 vectors per thread)
constexpr int kVecThreads = 256;         // threads of the vector kernels
constexpr int kMaxDevices = 64;          // device ordinals the per-device caches cover

// Per-device runtime state (runtime.cu): the device current at the call selects the entry.
int current_device();                                       // -1 if none
int sm_count();                                             // SMs of the current device
cudaError_t ensure_max_dyn_smem(const void* fn, int bytes); // once per (kernel, device)
cudaStream_t capture_stream();                              // private capture stream per (thread, device)
cudaStream_t side_stream();                                 // second work stream per (thread, device)

// Row modes of the fused A-pass: u_i = phi(t_i), t = A p.
enum ApassMode : int {
  MODE_ID = 0,        // u = t                        (H = A^T A)
  MODE_DIAG = 1,      // u = D_i t                    (H = A^T D A)
  MODE_LOGIT = 2,     // sigma = sigmoid(t), w = sigma(1-sigma), D_out = w,
                      // u = w t + b01 - sigma; loss += softplus(t) - b01 t
  MODE_RESID = 3,     // u = t - b_i; loss += (t - b_i)^2 / 2
  MODE_CONST = 4,     // u = b_i (no dot product: A^T b)
  MODE_LGRAD = 5      // u = sigma(t) - b01; loss += softplus(t) - b01 t (logistic gradient)
};

struct ApassArgs {
  const void* A;        // row-major n x ld
  int64_t n, d, ld;
  int dtype;            // nys_dtype
  const void* p;        // length d, compute type
  const double* D;      // length n (MODE_DIAG) or NULL
  const double* b;      // length n (RESID / CONST / LOGIT labels in {-1,+1})
  double* D_out;        // length n (MODE_LOGIT) or NULL
  double* t_out;        // length n or NULL: t = A p
  int mode;
  const int* skip = nullptr;  // if non-null and *skip != 0 the pass is skipped
  const float* col_scale = nullptr;  // FP8: per-column scales (A_ij = col_scale[j] q_ij)
};

// Workspace-carrying handle for repeated A-passes on one matrix.
struct ApassPlan {
  int grid = 0;          // CTAs (partials)
  int rows_per_step = 1; // R
  int stages = 2;        // S
  size_t smem = 0;       // dynamic shared memory bytes
  int64_t dpad = 0;      // partial row stride (elements of compute type)
  bool fused = true;     // false -> two-pass fallback
  int threads = 512;     // CTA size (float path: 512 or 640)
  int vpt = 0;           // 16-byte column vectors owned per thread
  bool onebar = false;   // float path, H-matvec modes: one barrier per step
  bool ws = false;       // warp-specialised pass (apass_ws.cu): threads / vpt / R / S of its layout
};

bool apass_plan(const nys_matrix* A, ApassPlan* plan);
// Argument checks shared by the entry points (capi.cu): NYS_EINVAL for a malformed matrix
// (null data, bad sizes, unknown dtype, col_scale present iff FP8, unaligned rows, no pass
// plan) and, for the H-matvec entry points, null / aliased vectors or a non-finite rho.
nys_status check_matrix(const nys_matrix* A);
nys_status check_hmatvec_args(const nys_matrix* A, double rho, const void* p, const void* y);
void apass_set_tuned_rows(const nys_matrix* A, int rows);   // rows <= 0 clears
int apass_row_candidates(const nys_matrix* A, int* out);      // out: up to 3 values
size_t apass_partial_bytes(const nys_matrix* A, const ApassPlan& plan);
// Calibrate unequal row slabs for the warp-specialised float pass of A (kept per device,
// dtype, row bytes, rows, grid and stage depth; used by every later pass of that shape).
// p: a device vector of A's compute type (d entries), part: partial scratch of the plan.
cudaError_t apass_balance_rows(const nys_matrix* A, const void* p, void* part, int* dstat, cudaStream_t st,
                               double* ms_equal, double* ms_split);

// y = sum of partials + rho * p (+ beta * y_prev?) -- y in compute type.
// dot_part (optional): per-block partials of p^T y (double), count returned via nblk.
// allow_stats = false keeps the launch off the instrumentation path (which may allocate).
cudaError_t apass_run(const ApassArgs& a, const ApassPlan& plan, void* partial, double* loss_part,
                      int* dev_status, cudaStream_t st, bool allow_stats = true);
cudaError_t apass_reduce(const ApassArgs& a, const ApassPlan& plan, const void* partial, double rho,
                         void* y, double* dot_part, int dot_blocks, cudaStream_t st);
int reduce_blocks(int64_t d);

// ---------------------------------------------------------------- small dense FP64 kernels
// C (s x s, col-major, ldc = s) = X^T Y for X, Y d x s col-major FP64 (ld = d); deterministic.
cudaError_t gram_xty(const double* X, const double* Y, int64_t d, int s, double* C, double* work,
                     cudaStream_t st);
size_t gram_work_bytes(int64_t d, int s);
// In-place upper Cholesky of a symmetric s x s matrix (col-major): C^T C = M. info[0] = 0 ok,
// k+1 if the k-th pivot is not positive, or not above rel_tol times the largest diagonal
// entry of M (numerically dependent columns).  M is symmetrised as (M + M^T)/2 first.
cudaError_t chol_upper(double* M, int s, int* info, cudaStream_t st, double rel_tol = 0.0);
// B (d x s) = Y C^{-1} with C upper (s x s); B may alias Y.
cudaError_t trsm_right_upper(const double* C, int s, double* Y, int64_t d, cudaStream_t st);
// Y += nu * X  (d x s)
cudaError_t axpy_panel(double nu, const double* X, double* Y, int64_t n, cudaStream_t st);
// lambda_max of a symmetric s x s matrix by power iteration (device scalar out)
cudaError_t power_lambda_max(const double* G, int s, double* out, double* work, cudaStream_t st);
// Symmetric eigendecomposition by parallel cyclic Jacobi: G (s x s, overwritten) -> V (s x s),
// eigenvalues in the diagonal.  Sweeps stop once off(A) <= tol ||A||_F.  Returns sweeps used
// in *sweeps (host).
cudaError_t jacobi_eig(double* G, double* V, int s, double* work, int* sweeps, cudaStream_t st, double tol = 1e-12);
size_t jacobi_work_bytes(int s);
// *out (device) = max_ij |G_ij - delta_ij| of the m x m matrix G.
cudaError_t identity_gap(const double* G, int m, double* out, cudaStream_t st);
// After Jacobi: sort eigenpairs descending, U = B V Sigma^{-1}, lam = max(0, sigma^2 - nu).
cudaError_t nystrom_finish(const double* B, int64_t d, int s, const double* G, const double* V,
                           double nu, double* U, double* lam, double* work, cudaStream_t st);

// ---------------------------------------------------------------- sketch GEMMs
// W (n x s, col-major, ld n) = diag(D) (A Omega) with Omega d x s col-major (ld d) in compute type
cudaError_t sketch_aw(const nys_matrix* A, const void* Omega, int s, const double* D, void* W,
                      cudaStream_t st);
// Y (d x s, col-major FP64) = A^T W (+ shift * Omega64)
cudaError_t sketch_atw(const nys_matrix* A, const void* W, int s, double* Y, void* work,
                       size_t work_bytes, cudaStream_t st);
size_t sketch_atw_work_bytes(const nys_matrix* A, int s);
// Tensor-core (tcgen05) products for BF16 storage and for FP32 storage (split exactly into
// three BF16 terms): tc_prepare builds the operands once (transposed copy of A; for FP32
// also the terms) in caller-owned scratch of tc_prepare_bytes(A) bytes.
struct TcPrepared {
  int at = 1;                    // A terms: 1 (BF16) or 3 (FP32 split)
  const uint16_t* A = nullptr;   // row-major terms, n x lda, term stride aterm
  int64_t lda = 0, aterm = 0;
  const uint16_t* At = nullptr;  // transposed terms, d x nP, term stride atterm
  int64_t nP = 0, atterm = 0;
};
bool sketch_tc_supported(const nys_matrix* A);
size_t tc_prepare_bytes(const nys_matrix* A);
cudaError_t tc_prepare(const nys_matrix* A, void* scratch, TcPrepared* prep, cudaStream_t st);
// Y (d x m, col-major FP64) = A^T diag(D) A Om (the sketch of App. B) on the tensor cores.
// Om must hold BF16 values (round_panel_bf16): the first product takes it as one term.
cudaError_t sketch_tc(const nys_matrix* A, const double* D, const double* Om, int m, double* Y, cudaStream_t st);
cudaError_t sketch_tc_with(const nys_matrix* A, const TcPrepared& prep, const double* D, const double* Om, int m,
                           double* Y, cudaStream_t st);
// X (n values, FP64) <- each entry rounded to the nearest BF16 value through FP32 (to nearest,
// ties to even): the test matrix of an FP32-class sketch.
cudaError_t round_panel_bf16(double* X, int64_t n, cudaStream_t st);
// Y (d x k) = A^T diag(D) A X + rho X, FP32 X and Y column-major (multi-RHS H-matvec).
cudaError_t tc_hmm(const nys_matrix* A, const TcPrepared& prep, const double* D, const float* X, int k, double rho,
                   float* Y, cudaStream_t st);
cudaError_t sketch_atw_partials(const nys_matrix* A, const void* W, int s, void* work, size_t work_bytes, int* nz_out,
                                cudaStream_t st);
// small dense GEMMs in compute type T (column-major)
template <typename T>
cudaError_t gemm_tn(const T* X, const T* Y, int64_t K, int M, int N, T* C, T* work, cudaStream_t st);
template <typename T>
size_t gemm_tn_work_elems(int64_t K, int M, int N);
template <typename T>
cudaError_t gemm_nn_t(const T* B, int64_t M, int K, const T* V, int N, T* C, cudaStream_t st);

// ---------------------------------------------------------------- helpers
// Omega (d x s column-major FP64) ~ N(0,1) from Philox-4x32-10 + Box-Muller (random.cu).
cudaError_t gaussian_panel(uint64_t seed, int64_t d, int s, double* Omega, cudaStream_t st);
cudaError_t convert_f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t st);
// *flag |= 1 (device int, caller-zeroed) if any of x[0..n) (FP64, or FP32) is NaN or infinite
cudaError_t any_nonfinite(const void* x, int64_t n, bool f32, int* flag, cudaStream_t st);
// FP8 E4M3 matrix with per-column scales -> FP32 values (n x ld, same layout)
cudaError_t dequantize_fp8(const nys_matrix* A, float* out, cudaStream_t st);
cudaError_t convert_f32_to_f64(const float* x, double* y, int64_t n, cudaStream_t st);

// Instrumentation (nys_stats_* in the C ABI): every kernel launch is counted; the
// fused A-pass launches are bracketed by CUDA events on their stream when enabled.
void count_launch();
void count_launch_suspend(bool on);     // while capturing a graph: launches are counted on execution
void count_launch_add(long long n);     // executed graph kernel nodes
bool launch_capturing();                // true between count_launch_suspend(true) and (false)
// Set the launch attributes of the A-pass instantiation for this matrix (outside capture).
cudaError_t apass_prepare(const nys_matrix* A, const ApassPlan& plan);
bool stats_enabled();
void stats_record_apass(cudaEvent_t start, cudaEvent_t stop, double bytes, int dtype, int* executed);

// In-kernel timing of A-pass launches (works inside CUDA graphs): the first CTA to
// start stamps %globaltimer into start[slot] (atomicMin), every CTA stamps its end
// (atomicMax), and the last CTA to finish advances *count.
struct DevTimer {
  unsigned long long* start = nullptr;
  unsigned long long* end = nullptr;
  double* bytes = nullptr;
  int* dtype = nullptr;
  int* count = nullptr;
  int* done = nullptr;
  int cap = 0;
};
DevTimer stats_device_timer();
// An event pair plus a zeroed device flag that the pass sets when it runs.
cudaError_t stats_event_pair(cudaEvent_t* start, cudaEvent_t* stop, int** executed);

inline size_t dtype_size(int dt) { return dt == NYS_F64 ? 8 : (dt == NYS_F32 ? 4 : (dt == NYS_BF16 ? 2 : 1)); }
inline bool compute_is_f64(int dt) { return dt == NYS_F64; }

}  // namespace nys

#define NYS_CUDA_TRY(expr)                          \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return _e;               \
  } while (0)
