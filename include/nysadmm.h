/*
 * nysadmm.h -- C ABI of the GB300 NysADMM hot path.
 *
 * The library solves  minimize  l(Ax; b) + gamma ||x||_1   (Eq. 1 / Eq. 2 /
 * Eq. 9 of "NysADMM: faster composite convex optimization via low-rank
 * approximation") by inexact linearised ADMM whose x-subproblem
 *     (A^T D A + rho I) x = r            (Eq. ADMMSubProb; D = I for the lasso,
 *                                         D = diag(sigma(1-sigma)) for Eq. 9)
 * is solved by conjugate gradients preconditioned with a randomised Nystrom
 * approximation (App. B: Alg. Randomized Nystrom Approximation, Alg. Nystrom PCG).
 *
 * Conventions shared by every entry point
 *  - Every array argument is a DEVICE pointer on the current CUDA device,
 *    caller-owned, unless the comment says "host".  The caller keeps it valid
 *    until the call returns; all work is issued on `stream` (NULL = legacy
 *    default stream) and every entry point synchronises `stream` before it
 *    returns, so outputs are ready on return.
 *  - Matrices (nys_matrix) are dense and ROW-major: element (i, j) of A is at
 *    data + i*ld + j.  ld >= d, ld * sizeof(element) must be a multiple of 16
 *    bytes and data must be 16-byte aligned (rows are streamed by TMA bulk
 *    copies).  Entries j in [d, ld) are never read as data.
 *  - d x s panels (Omega, U) are COLUMN-major with leading dimension d.
 *  - Vector precision ("compute type") follows the matrix that PCG runs on:
 *    FP64 vectors for an NYS_F64 matrix, FP32 vectors for NYS_F32 / NYS_BF16 /
 *    NYS_FP8E4M3.
 *    ADMM state (x, z, u, residuals) is always FP64.
 *  - Errors are returned, never trapped: NYS_EINVAL for bad arguments (checked
 *    before any launch; NaN or infinite data -- in b, in A, in Omega, in the PCG
 *    right-hand side or start -- is detected on the device where it first enters a
 *    reduction and also gives NYS_EINVAL), NYS_ENOTSPD if the Nystrom core matrix stays
 *    indefinite after shift retries, NYS_EBREAKDOWN if p^T (H + rho I) p <= 0
 *    or is not finite in PCG, NYS_ENOCONV when an iteration cap is reached
 *    (the last iterate is still written), NYS_ETIMEOUT if a device-side wait
 *    exceeded its bound, NYS_ECUDA for a CUDA runtime error, NYS_ENOMEM if a
 *    workspace allocation failed.
 *  - The library allocates its own workspace with cudaMallocAsync on `stream`
 *    and frees it before returning; nys_precond handles own device memory
 *    until nys_precond_destroy.
 */
#ifndef NYSADMM_H
#define NYSADMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NYS_OK = 0,
  NYS_EINVAL = 1,
  NYS_ENOTSPD = 2,
  NYS_EBREAKDOWN = 3,
  NYS_ENOCONV = 4,
  NYS_ETIMEOUT = 5,
  NYS_ECUDA = 6,
  NYS_ENOMEM = 7
} nys_status;

/* Loss l(Ax; b): the lasso (Eq. 2, D = I) or l1-regularised logistic
 * regression (Eq. 9 with labels b in {-1,+1} mapped to (1+b)/2). */
typedef enum { NYS_LASSO = 0, NYS_LOGISTIC = 1, NYS_ELASTIC_NET = 2 } nys_loss;

/* Storage of A.  NYS_FP8E4M3: 8-bit E4M3 codes q with one FP32 scale per column,
 * A_ij = col_scale[j] * q_ij (the per-column-scaled FP8 form of the mixed precision
 * variant); accepted where A is the matrix PCG runs on (nys_hmatvec, nys_sketch,
 * pcg_solve, opts->A_inner of nysadmm_solve), with FP32 vectors. */
typedef enum { NYS_F64 = 0, NYS_F32 = 1, NYS_BF16 = 2, NYS_FP8E4M3 = 3 } nys_dtype;

/* PCG stopping test at the top of each iteration (Alg. Nystrom PCG):
 * REL: ||w|| <= tol ||r||;  ABS: ||w|| <= tol (as printed);
 * SQRT_RPRD: inside ADMM, tol_k = sqrt(r_p r_d) of the previous ADMM
 * iteration (Sec. 5 experiments), REL with `tol` at the first iteration;
 * RNORM_POW: inside ADMM, ||w|| <= ||r^k|| / k^beta with beta = `tol` and k = 1, 2, ...
 * the ADMM iteration (the decaying schedule of Sec. 5); pcg_solve rejects it. */
typedef enum { NYS_TOL_REL = 0, NYS_TOL_ABS = 1, NYS_TOL_SQRT_RPRD = 2, NYS_TOL_RNORM_POW = 3 } nys_tol_mode;

typedef struct {
  const void* data;        /* device, row-major n x ld, 16-byte aligned */
  int32_t dtype;           /* nys_dtype */
  int64_t n, d, ld;
  const float* col_scale;  /* NYS_FP8E4M3: device, length d; NULL for the other types */
} nys_matrix;

/* Opaque Nystrom preconditioner: U (d x s, orthonormal columns), the
 * eigenvalue estimates lam (descending) and the shift nu (App. B). */
typedef struct nys_precond_s* nys_precond;

/* Sum over the ranks of a row-sharded solve, completed in place on buf (device, count
 * values of dtype NYS_F64 or NYS_F32), ordered on `stream`: the callback either enqueues
 * the reduction on that stream or synchronises it.  Returns NYS_OK or an error status. */
typedef int32_t (*nys_allreduce_fn)(void* buf, int64_t count, int32_t dtype, void* stream, void* ctx);

typedef struct {
  double shift_scale;          /* nu = shift_scale * eps(||Y||_2); <= 0 -> sqrt(d) */
  int32_t pcg_tol_mode;        /* nys_tol_mode */
  int32_t pcg_maxit;           /* <= 0 -> min(d, 1000) */
  const int32_t* pcg_fixed_iters; /* host, length admm_maxit, or NULL: run exactly
                                      this many PCG iterations at ADMM iteration k */
  int32_t admm_maxit;          /* ADMM iterations (upper bound when eps_rel > 0) */
  double eps_abs, eps_rel;     /* residual stop of Sec. 2.1; eps_rel <= 0 -> off */
  const nys_matrix* A_inner;   /* optional lower-precision copy of A used for the
                                  sketch and inside PCG (mixed form); NULL -> A */
  int32_t refine;              /* mixed form: each x-step solves for the correction
                                  of the exact residual r - (A^T D A + rho I) x
                                  computed with A (1) or runs PCG on A_inner alone (0) */
  double* z_trace;             /* device, admm_maxit x d (row k = z after iteration
                                  k), or NULL */
  int32_t rank_max;            /* adaptive rank cap (logistic); <= 0 -> rank */
  double ada_tol;              /* adaptive stop (lam_s + rho)/rho <= ada_tol; <= 0 -> 2 */
  int32_t resketch_every;      /* logistic: re-sketch period in outer iterations (0 = never) */
  void* stream;                /* cudaStream_t */
  int32_t device_loop;         /* lasso: 1 = run the ADMM and PCG loops on the device as one
                                  CUDA graph with conditional WHILE nodes (no host
                                  synchronisation inside the solve); 0 = host-driven loop.
                                  Both launch the same kernels in the same order. */
  int32_t hx_refresh;          /* PCG warm start w0 = r - (A^T D A + rho I) x0: 0 = recompute
                                  it with one pass over A at every ADMM iteration (as printed
                                  in Alg. Nystrom PCG); M >= 1 = carry (A^T D A + rho I) x
                                  along the PCG updates and recompute it every M ADMM
                                  iterations (device_loop only; same value in exact arithmetic) */
  void* warm_model;            /* nys_mlp or NULL (lasso, device_loop): learned warm start,
                                  PCG starts at x_prev + U c with c = model(features) (see
                                  nys_mlp_create); the model needs n_in = rank + 3, n_out = rank */
  float* warm_record;          /* device, admm_maxit x (2 rank + 3) FP32, or NULL (lasso,
                                  device_loop): row k = [features (rank + 3), target (rank)] of
                                  ADMM iteration k, the training pairs for the model */
  uint64_t seed;               /* Omega == NULL in nys_sketch / nysadmm_solve / nysadmm_solve_path:
                                  the Gaussian test matrix is drawn in the library from this seed
                                  (nys_gaussian_test_matrix); default 0 */
  nys_allreduce_fn allreduce;  /* row-sharded operation (Table 1's T_mv and the sketch are sums
                                  over row blocks, A^T D A = sum_g A_g^T D_g A_g): each process
                                  passes its own contiguous block of rows A_g, b_g; every sum
                                  over rows -- the sketch A^T D A Omega (one d x s reduction),
                                  A^T b, each PCG matvec (one d-vector reduction per iteration),
                                  the refined step's residual -- is completed by this callback;
                                  all d-space state is replicated and stays identical on every
                                  rank.  Supported by nys_sketch, pcg_solve and nysadmm_solve
                                  (lasso / elastic net, device_loop = 0, no warm_model); other
                                  calls with a callback return NYS_EINVAL.  NULL: unsharded. */
  void* allreduce_ctx;         /* passed to allreduce */
  int32_t* pcg_trace;          /* host, admm_maxit, or NULL: PCG iterations of each ADMM
                                  iteration of nysadmm_solve (lasso / elastic net) */
} nys_opts;

typedef struct {
  int32_t admm_iters;          /* ADMM iterations run */
  int32_t pcg_iters_total;     /* sum of PCG iterations */
  int32_t final_rank;          /* sketch size of the last preconditioner */
  int32_t status;              /* nys_status of the solve */
  double r_p, r_d;             /* last primal / dual residual norms (Sec. 2.1) */
  double emp_cond;             /* (lam_s + rho)/rho of the last preconditioner (Eq. empCondNum) */
  double nu;                   /* shift of the last sketch */
} nys_info;

/* Fills *o with the defaults documented in nys_opts. */
void nys_opts_default(nys_opts* o);

/* H-matvec (Table 1, T_mv; the product inside Alg. Nystrom PCG):
 *   y = A^T diag(D) A p + rho p,  one read of A per call.
 * D: device, length n, FP64, or NULL for D = I.  p, y: device, length d, in the
 * compute type of A (FP64 for NYS_F64, else FP32).  y must not alias p. */
nys_status nys_hmatvec(const nys_matrix* A, const double* D, double rho, const void* p,
                       void* y, void* stream);

/* Allocation-free variant of nys_hmatvec (the paper has no counterpart; this is a
 * deployment convenience).  Same arguments, same checks and the same result, bit for
 * bit, for every storage type nys_hmatvec accepts (FP8 E4M3 included), but it allocates
 * no device memory: its scratch (the per-block partial sums and a status word) is a
 * fixed 16 MiB array compiled into the library, which every GPU that loads the library
 * holds until the process exits.  It is meant for callers that cannot call
 * cudaMalloc/cudaFree on the request path: for example a service whose device memory is
 * entirely owned by another allocator (a framework's caching allocator or a
 * preallocated arena), or a latency-critical caller that cannot take the device-wide
 * synchronisation cudaFree implies.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current).
 *  - Like every entry point it ends by reading the status word back and synchronising
 *    `stream`, so it cannot be called while `stream` is being captured into a graph.
 *  - Scratch needed = (#blocks of the pass, at most the SM count) x d rounded up
 *    to 16 bytes x (8 for NYS_F64, else 4) bytes; a call that needs more than
 *    16 MiB returns NYS_EINVAL without launching anything.
 *  - All calls share the one array, so calls that overlap on the GPU (different
 *    streams, or host threads) race and corrupt each other's partial sums:
 *    serialise them.  Each call overwrites every partial it reads and clears the
 *    status word itself. */
nys_status nys_hmatvec_noalloc(const nys_matrix* A, const double* D, double rho, const void* p,
                               void* y, void* stream);

/* Gaussian test matrix of the sketch (App. B, Alg. Randomized Nystrom Approximation draws
 * Omega with independent N(0,1) entries), drawn on the device: Omega (device, d x s
 * column-major FP64) from the counter-based generator Philox-4x32-10 (Salmon et al., SC 2011)
 * and the Box-Muller transform.  Element e = i + j d is member e mod 2 of pair m = e / 2,
 * drawn with counter (lo32(m), hi32(m), 0, 0) and key (lo32(seed), hi32(seed)); the 4 output
 * words give u1 = (((w0 2^32 + w1) >> 11) + 1) 2^-53 and u2 = ((w2 2^32 + w3) >> 11) 2^-53, and
 * the pair is sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).  The panel depends only on (seed, d, s)
 * (a d x s draw is the first d s values of a (d s) x 1 draw).  NYS_EINVAL for d < 1, s < 1 or a
 * NULL Omega. */
nys_status nys_gaussian_test_matrix(uint64_t seed, int64_t d, int32_t s, double* Omega, void* stream);

/* Randomized Nystrom approximation of H = A^T diag(D) A + diag_shift I
 * (App. B, Alg. Randomized Nystrom Approximation): Omega (device, d x s,
 * column-major FP64 Gaussian test matrix drawn by the caller) is
 * orthonormalised (CholQR2), Y = H Omega is sketched (in FP64 for an NYS_F64
 * matrix, FP32 otherwise), and the FP64 core gives U, lam.  Omega is not
 * modified.  opts may be NULL (defaults; opts->stream supplies the stream). */
nys_status nys_sketch(const nys_matrix* A, const double* D, double diag_shift, int32_t s,
                      const double* Omega, const nys_opts* opts, nys_precond* out);

/* Copies the factors out: U_out (device, d x s column-major FP64) and
 * lam_out (host, length s, descending) may be NULL.  *s_out, *d_out, *nu_out
 * (host) are set when non-NULL. */
nys_status nys_precond_get(nys_precond P, double* U_out, double* lam_out, int32_t* s_out,
                           int64_t* d_out, double* nu_out, void* stream);

/* P^{-1} applied to k vectors (Eq. Nystrom preconditioner):
 *   Y = (lam_s + rho) U (Lam + rho I)^{-1} U^T V + (I - U U^T) V,
 * V, Y: device, d x k column-major, dtype NYS_F64 or NYS_F32.  Y may alias V. */
nys_status nys_precond_apply(nys_precond P, double rho, const void* V, void* Y, int64_t k,
                             int32_t dtype, void* stream);

/* Nystrom PCG (App. B, Alg. Nystrom PCG) for (A^T diag(D) A + rho I) x = r.
 * r, x: device, length d, compute type of A; x holds x0 on entry and the
 * solution on return.  P may be NULL (plain CG).  tol with opts->pcg_tol_mode
 * (REL or ABS; SQRT_RPRD acts as REL outside ADMM, RNORM_POW and unknown modes give
 * NYS_EINVAL); opts->pcg_fixed_iters[0], when set, fixes the iteration count.
 * *iters and *resnorm (host, may be NULL) receive the iteration count and ||w||. */
nys_status pcg_solve(const nys_matrix* A, const double* D, double rho, nys_precond P,
                     const void* r, void* x, double tol, const nys_opts* opts,
                     int32_t* iters, double* resnorm);

/* NysADMM (Alg. NysADMM; Alg. AdaNysADMM with opts->rank_max > rank):
 * loss NYS_LASSO: sketch once, then opts->admm_maxit ADMM iterations with
 * PCG tolerance `tol` (mode opts->pcg_tol_mode), warm-started at the previous
 * x, z-update by soft-thresholding at gamma/rho.
 * With opts->rank_max > rank (lasso, elastic net) the sketch size is chosen once,
 * before the iterations, by Alg. AdaptiveRandNysAppx from `rank` up to rank_max with
 * stop (lam_s + rho)/rho <= opts->ada_tol (Alg. AdaNysADMM); info->final_rank reports it.
 * loss NYS_ELASTIC_NET (Sec. 3.1, Eq. 6; 0 < gamma <= 1, else NYS_EINVAL):
 * as NYS_LASSO with g(x) = (1 - gamma)/2 ||x||^2, so the sketched Hessian is
 * A^T A + (1 - gamma) I, the PCG matrix A^T A + (1 - gamma + rho) I, and the
 * z-update soft-thresholds at gamma/rho.
 * loss NYS_LOGISTIC: D and the right-hand side are refreshed from
 * t = A x~ at every outer iteration (Sec. 3.2); the rank is chosen by
 * Alg. AdaptiveRandNysAppx from `rank` up to opts->rank_max at the first
 * iteration and re-sketched every opts->resketch_every iterations.
 * PCG tolerance schedules (opts->pcg_tol_mode, nys_tol_mode): with RNORM_POW `tol`
 * is beta.  An unknown mode gives NYS_EINVAL.
 * b: device, length n, FP64 (labels in {-1,+1} for NYS_LOGISTIC).
 * Omega: device, d x max(rank, rank_max) column-major FP64 Gaussian, or NULL: drawn in the
 * library by nys_gaussian_test_matrix with opts->seed.
 * x_out, z_out: device, length d, FP64 (z is the sparse iterate; either may be
 * NULL).  info: host, may be NULL. */
nys_status nysadmm_solve(int32_t loss, const nys_matrix* A, const double* b, double gamma,
                         double rho, int32_t rank, double tol, const double* Omega,
                         const nys_opts* opts, double* x_out, double* z_out, nys_info* info);

/* Lasso regularisation path: k NysADMM lasso solves (Alg. NysADMM) that share A,
 * b, rho and the Nystrom preconditioner and differ in gamma (gammas: host, k).
 * Because the x-subproblem matrix A^T A + rho I (Eq. ADMMSubProb) is common to
 * all k problems, the k PCG solves run side by side: each matvec reads A (or
 * opts->A_inner) once for all k right-hand sides as two dense products, and each
 * column keeps its own PCG scalars and stop test.  opts->admm_maxit ADMM
 * iterations are run for every gamma (opts->refine and device_loop do not apply).
 * X_out, Z_out: device, d x k column-major FP64 (column c = problem c), may be
 * NULL.  pcg_iters: host, k (total PCG iterations per column), may be NULL. */
nys_status nysadmm_solve_path(const nys_matrix* A, const double* b, const double* gammas, int32_t k, double rho,
                              int32_t rank, double tol, const double* Omega, const nys_opts* opts, double* X_out,
                              double* Z_out, nys_info* info, int32_t* pcg_iters);

/* One independent lasso instance of a batch (device pointers). */
typedef struct {
  const nys_matrix* A;   /* problem matrix; all instances of a batch share its compute type */
  const double* b;       /* length n */
  double gamma;
  int32_t rank;          /* Nystrom sketch size of this instance */
  const double* Omega;   /* d x rank column-major Gaussian test matrix */
  double* x_out;         /* length d FP64, or NULL */
  double* z_out;         /* length d FP64, or NULL */
} nys_lasso_instance;

/* A batch of independent lasso problems of different sizes, each solved by
 * NysADMM (Alg. NysADMM) with its own sketch and preconditioner.  The sketches are
 * built first; then every instance's device-side ADMM/PCG loop (conditional WHILE
 * nodes, as with opts->device_loop) becomes one branch of a single CUDA graph, so
 * the whole batch runs as one graph launch and the GPU overlaps the instances.
 * Shared: rho, the PCG tolerance tol and opts (admm_maxit, tolerance mode, stops,
 * hx_refresh).  infos: host array of count entries, may be NULL. */
nys_status nysadmm_solve_batch(int32_t count, const nys_lasso_instance* inst, double rho, double tol,
                               const nys_opts* opts, nys_info* infos);

/* Objective and optimality measures at x (FP64, one read of A):
 * out[0] = l(Ax; b) + g(x) + gamma ||x||_1 (Eq. 2, Eq. 6 or Eq. 9);
 * out[1] = relative KKT residual eta (Eq. 31, with the gradient of g added for the
 *          elastic net) or ||A^T(sigma(Ax)-b01)||_inf (logistic);
 * out[2] = duality gap at the scaled-residual dual point (lasso; the elastic net as
 *          the lasso of the stacked data [A; sqrt(1-gamma) I], [b; 0]) or 0 (logistic).
 * x: device, length d, FP64; out: host, length 3. */
nys_status nys_objective(int32_t loss, const nys_matrix* A, const double* b, double gamma,
                         const double* x, double* out, void* stream);

/* Instrumentation (no counterpart in the paper; used to report measured
 * bandwidth).  nys_stats_enable(1) resets the counters and starts recording:
 * every kernel launch of the library is counted, and each fused A-pass launch
 * (the H-matvec / right-hand-side pass) is bracketed by CUDA events on the
 * stream it runs on.  nys_stats_read waits for the recorded events and fills
 * *out (host).  apass_bytes is the algorithmic traffic of those launches:
 * n*d*sizeof(element) for A plus the vectors read and the partials written. */
typedef struct {
  int64_t launches;           /* kernel launches since the last enable */
  int64_t apass_launches[4];  /* fused A-pass launches that ran (a launch issued after
                                 PCG converged returns at once and is not counted),
                                 by nys_dtype of A */
  double apass_ms[4];         /* summed device time of those launches (ms) */
  double apass_bytes[4];      /* summed algorithmic bytes of those launches */
  /* The same quantities from the kernels' own %globaltimer stamps (earliest CTA
   * start to latest CTA end of each launch).  These also cover passes launched
   * inside the device-side solve loop (a CUDA graph), where no event can
   * bracket an individual kernel. */
  int64_t dev_launches[4];
  double dev_ms[4];
  double dev_bytes[4];
} nys_stats;

void nys_stats_enable(int32_t on);
nys_status nys_stats_read(nys_stats* out);

/* Diagnostic of the device-side wait bound (no counterpart in the paper).  Every
 * device-side wait of the library (TMA stages, tensor-core completions, grid steps) is
 * bounded; when a bound runs out the kernel stops waiting, records NYS_ETIMEOUT and
 * returns, so the host gets a status and the CUDA context stays usable.  This call runs
 * one such wait on a barrier that nothing completes, with a bound of wait_us
 * microseconds (0 < wait_us <= 5e6), and returns NYS_ETIMEOUT when the bound works.
 * NYS_EINVAL for a bound outside that range. */
nys_status nys_check_wait_bound(double wait_us, void* stream);

/* Learned warm start for the x-subproblem (no counterpart in the paper; an
 * AI-systems addition).  A multilayer perceptron n_in -> n_hid -> n_hid -> n_out
 * with erf-GELU hidden units; BF16 weights in the matrix products with FP32
 * accumulation, FP32 master weights, Adam (beta 0.9 / 0.999, eps 1e-8).
 * In NysADMM (opts->warm_model) its input at ADMM iteration k is
 *   f = [U^T r / ||r||, log10(rho), k / 100, ln ||r||]   (rank + 3 values)
 * for the x-subproblem right-hand side r and the Nystrom basis U.  The model
 * predicts the solution's coordinates in range(U) scaled by rho / ||r||, and PCG
 * starts at x_prev + U c with c = model(f) ||r|| / rho - U^T x_prev (the component
 * of x_prev in range(U) replaced by the prediction).  The training target recorded
 * in opts->warm_record is U^T x_new * rho / ||r||.  PCG still runs to the same
 * tolerance.
 * Parameters (flat FP32): [W1 (n_hid x n_in), b1, W2 (n_hid x n_hid), b2,
 * W3 (n_out x n_hid), b3], weights row-major (output x input); init_params (host
 * or device) supplies the initial values, drawn by the caller.  X, T, Y are device
 * row-major batches (B x n_in / B x n_out, FP32).  Loss = mean (Y - T)^2. */
typedef struct nys_mlp_s* nys_mlp;
nys_status nys_mlp_create(int32_t n_in, int32_t n_hid, int32_t n_out, const float* init_params, nys_mlp* out);
nys_status nys_mlp_forward(nys_mlp M, const float* X, int32_t B, float* Y, void* stream);
/* loss (host, may be NULL) and gradient (device, flat, may be NULL) at the current parameters */
nys_status nys_mlp_grad(nys_mlp M, const float* X, const float* T, int32_t B, float* grad_out, float* loss,
                        void* stream);
/* one Adam step on the batch; *loss (host, may be NULL) is the loss before the step */
nys_status nys_mlp_train_step(nys_mlp M, const float* X, const float* T, int32_t B, float lr, float* loss,
                              void* stream);
/* copies the FP32 master parameters to out (host or device; NULL to query *n_params) */
nys_status nys_mlp_get_params(nys_mlp M, float* out, int64_t* n_params, void* stream);
void nys_mlp_destroy(nys_mlp M);

/* Autotuner for the fused pass (no counterpart in the paper): times each supported
 * rows-per-stage choice (1, 2 or 4 rows per TMA stage, as the register and shared
 * memory budgets allow) on A with CUDA events (one warm-up and three timed passes
 * each) and keeps the fastest for every later pass over a matrix of the same
 * storage type and row width in this process.  *rows_out, *ms_out (host, may be
 * NULL): the choice and its time per pass. */
nys_status nys_autotune_apass(const nys_matrix* A, int32_t* rows_out, double* ms_out, void* stream);

void nys_precond_destroy(nys_precond P);
const char* nys_strerror(int32_t status);

#ifdef __cplusplus
}
#endif
#endif /* NYSADMM_H */
