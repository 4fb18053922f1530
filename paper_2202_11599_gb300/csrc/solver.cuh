// Host-side solver structures shared by pcg.cu and capi.cu.
#pragma once
#include <vector>

#include "nys_internal.cuh"

namespace nys {

struct PcgState {
  double wy;       // w^T y of the previous iteration (denominator of beta)
  double w2;       // ||w||^2 of the current residual
  double r2;       // ||r||^2
  double thresh2;  // stop when ||w||^2 <= thresh2
  double tol;
  int tol_abs;
  int iters;
  int done;
  int status;
  int maxit;
  int fixed;       // >= 0: run exactly this many iterations
  unsigned int ticket[2];  // last-block election of the fused update / tail kernels (zero between launches)
  unsigned int bar_count, bar_gen;  // grid barrier of pcg_post_kernel (zeroed once per solve)
};

// Stream-ordered device allocations freed when the pool goes out of scope.
void keep_mempool_cached();

class Pool {
 public:
  explicit Pool(cudaStream_t st) : st_(st) { keep_mempool_cached(); }
  ~Pool() {
    for (void* p : ptrs_) cudaFreeAsync(p, st_);
  }
  template <typename T>
  T* alloc(size_t count) {
    if (count == 0) count = 1;
    void* p = nullptr;
    if (cudaMallocAsync(&p, count * sizeof(T), st_) != cudaSuccess) {
      ok_ = false;
      cudaGetLastError();
      return nullptr;
    }
    ptrs_.push_back(p);
    return reinterpret_cast<T*>(p);
  }
  bool ok() const { return ok_; }

 private:
  cudaStream_t st_;
  std::vector<void*> ptrs_;
  bool ok_ = true;
};

// Row-sharded operation: the communicator of the calling thread's current entry point
// (set from nys_opts for the duration of the call).  shard_sum is a no-op without one.
struct ShardComm {
  nys_allreduce_fn fn = nullptr;
  void* ctx = nullptr;
};
ShardComm& shard_comm();
nys_status shard_sum(void* buf, int64_t count, int dtype, cudaStream_t st);
struct ShardScope {
  explicit ShardScope(const nys_opts* o);
  ~ShardScope();
  ShardComm saved;
};

struct PcgProblem {
  const nys_matrix* A;
  const double* D;    // NULL: H = A^T A
  double rho;
  ApassPlan plan;
};

// Preconditioner in the PCG compute type: U (d x s column-major) and
// c_i = (lam_s + rho)/(lam_i + rho) - 1 (Eq. Nystrom preconditioner).  s = 0: P = I.
struct PrecondView {
  const void* U = nullptr;
  const void* c = nullptr;
  int s = 0;
};

struct PcgParams {
  double tol = 1e-8;
  int tol_abs = 0;
  int maxit = 1000;
  int fixed = -1;
  bool x0_zero = false;
  const double* dev_tol = nullptr;  // device tolerance (absolute), overrides tol
};

template <typename C>
nys_status pcg_run(const PcgProblem& pb, const PrecondView& P, const C* r, C* x, const PcgParams& prm,
                   cudaStream_t stream, int* iters_out, double* resnorm_out);

template <typename C>
nys_status precond_apply_run(const PrecondView& P, int64_t d, const C* V, C* Y, int64_t k, cudaStream_t stream);

template <typename C>
cudaError_t admm_rhs(int64_t d, const double* q, const double* z, const double* u, double rho, const double* x,
                     const double* yres, C* r, cudaStream_t st, double mu = 0.0);
template <typename C>
cudaError_t admm_zu(int64_t d, const C* xc, int accumulate, double* x, double* z, double* u, double kappa,
                    double* ztrace, double* part5, cudaStream_t st);
cudaError_t admm_scalar(int64_t d, const double* part5, double rho, int k, double* rp, double* rd, double* eps_next,
                        double eps_abs, double eps_rel, int* stop, cudaStream_t st);
int admm_blocks(int64_t d);
int pcg_nb3(int64_t d);

PcgState* host_state();

// Multi-RHS PCG (k columns sharing H + rho I and P); R, X: d x k column-major.
template <typename C>
nys_status batched_pcg_run(const PcgProblem& pb, const PrecondView& P, const C* R, C* X, int k, const PcgParams& prm,
                           cudaStream_t st, std::vector<int>* iters_out);
template <typename C>
cudaError_t batched_rhs(int64_t d, int k, const double* q, const double* Z, const double* Uu, double rho, C* R,
                        cudaStream_t st);
template <typename C>
cudaError_t batched_zu(int64_t d, int k, const C* Xc, double* X, double* Z, double* Uu, const double* kappa,
                       double* part, int* nb_out, cudaStream_t st);
int batched_zu_blocks(int64_t d);

// Device-side lasso ADMM loop (one CUDA graph with conditional WHILE nodes).
struct GraphLoopArgs {
  PcgProblem pb;             // PCG matrix (A_inner or A), D, rho, plan
  PrecondView P;
  const nys_matrix* Aref = nullptr;  // refined step: exact residual with this (FP64) matrix
  ApassPlan plan_ref;
  const double* b = nullptr;
  double* yres = nullptr;    // d, FP64 (refined step)
  double *x = nullptr, *z = nullptr, *u = nullptr, *q = nullptr;
  void *xc = nullptr, *rc = nullptr, *hx = nullptr;  // compute type, length d
  double gamma = 0, rho = 1;
  double mu = 0;             // H^g = mu I (elastic net): the H-matvec shift is rho + mu
  int K = 1;
  double eps_abs = 0, eps_rel = 0;
  double tol = 1e-8;          // beta for NYS_TOL_RNORM_POW
  double tol_floor = 0;       // lower bound of a relative PCG tolerance (FP32 refined step)
  int tol_mode = NYS_TOL_REL;
  int maxit = 1000;
  const int* fixed_host = nullptr;
  int hx_refresh = 0;
  double* ztrace = nullptr;
  double *rp = nullptr, *rd = nullptr;
  int* pcg_it = nullptr;     // device, K
  const nys_mlp_s* warm = nullptr;   // learned warm start model, or null
  float* warm_record = nullptr;      // K x (2 s + 3) feature/target rows, or null
  bool allow_nostep = true;          // fused no-PCG-step iterations (off for graph branches that
                                     // run concurrently: its grid barrier wants the grid co-resident)
};
struct GraphLoopResult {
  int admm_iters = 0;
  bool breakdown = false;
};
struct AdmmCtl;
// MLP forward on device buffers (no allocation or synchronisation: capturable)
cudaError_t mlp_forward_dev(const nys_mlp_s* M, const float* X, int B, float* z1, float* h1, float* z2, float* h2,
                            float* Y, cudaStream_t st);
int mlp_dims(const nys_mlp_s* M, int* ni, int* nh, int* no);
struct GraphInstance {
  AdmmCtl* ctl = nullptr;
  int* dstat = nullptr;
};
template <typename C>
nys_status admm_graph_run(const GraphLoopArgs& g, cudaStream_t stream, GraphLoopResult* res);
// Several independent instances as parallel branches of ONE graph launch.
template <typename C>
nys_status admm_graph_run_many(const GraphLoopArgs* gs, int count, cudaStream_t stream, GraphInstance* insts,
                               GraphLoopResult* res);

}  // namespace nys
