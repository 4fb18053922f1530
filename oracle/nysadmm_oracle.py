"""NysADMM oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 NumPy restatement of the method of "NysADMM: faster
composite convex optimization via low-rank approximation" (Zhao, Frangella,
Udell, ICML 2022).  Only the tests, the smoke check and the benchmark's CPU
baseline leg may import this module; the product path never does.  It shares
no code with the CUDA library: its one shared dependency is the seeded input
generator module, which holds no arithmetic of the method.

Each function names the passage of the paper it restates.  NumPy / SciPy
library routines (matmul, QR, Cholesky, SVD, triangular solve) serve as single
steps; nothing is blocked, fused or reordered beyond the paper's algorithms.

Readings where the paper is silent or ambiguous (the same readings as the CUDA path):
  * shift nu = shift_scale * eps(||Y||_2); eps(t) is the spacing of the working
    precision at t (MATLAB eps); default shift_scale = sqrt(d) (the adaptive
    algorithm's form, App. B), used for the fixed-rank sketch as well.
  * Cholesky failure: nu is multiplied by 10, up to 3 retries.
  * PCG stopping: 'rel' (||w|| <= tol*||r||), 'abs' (||w|| <= tol, Alg.
    Nystrom PCG as printed), or a fixed iteration count.
  * ADMM starts from x = z = u = 0; PCG is warm-started at the previous x.
  * Adaptive rank: stop at the first rank whose empirical condition number
    (lam_s + rho)/rho <= Tol; otherwise double, and when doubling would pass
    s_max, extend to s_max once and stop.
  * PCG schedule 'rnorm_pow' (Sec. 5's ||r^k|| / k^beta): k counts ADMM
    iterations from 1 (k = 0 would divide by zero).  Schedule 'sqrt_rprd'
    (sqrt(r_p r_d) of the previous iteration): the first solve, which has no
    residuals yet, uses pcg_tol as a relative tolerance.
  * Elastic net (Sec. 3.1): H^g = (1 - gamma) I enters the sketched matrix and the
    PCG matrix, not the preconditioner's rho; its duality gap is that of the lasso
    of the stacked data [A; sqrt(1 - gamma) I], [b; 0].
  * Mixed precision form without a correction pass: a low-precision copy A_inner
    (its stored values, given in FP64) builds the sketch and the x-subproblem matrix,
    while A^T b comes from the problem matrix A, so the iteration solves the perturbed
    problem 1/2 x^T A_inner^T A_inner x - (A^T b)^T x + gamma ||x||_1; the sketch shift
    then uses the FP32 eps (mantissa_bits = 23).
  * Test matrix of an FP32-class sketch (mantissa_bits = 23): the orthonormal factor of
    qr(Omega, 0) rounded to BF16 values (FP64 -> FP32 -> BF16, each to nearest, ties to
    even), and that rounded matrix is the Omega of every later step (Y = H Omega, the
    shift, Omega^T Y_nu).  The Nystrom approximation depends on Omega only through its
    range and holds for any full-rank test matrix; the rounded one is orthonormal to
    about 2^-8.

Functions with no independent pin: none (every function here is pinned by a
test in tests/test_oracle_pins.py against closed forms, library solvers,
brute force or the paper's lemmas).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


class NotSPDError(RuntimeError):
    pass


class BreakdownError(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# Scalars
# ---------------------------------------------------------------------------

def eps_of(t: float, mantissa_bits: int = 52) -> float:
    """Spacing of the working precision at |t| (MATLAB eps(t)), used for the
    shift of Alg. Randomized Nystrom Approximation (App. B).

    For t = f * 2^e with 0.5 <= f < 1 this is 2^(e - 1 - mantissa_bits).
    mantissa_bits = 52 for FP64, 23 for FP32."""
    t = abs(float(t))
    if t == 0.0:
        return 2.0 ** (-1074) if mantissa_bits == 52 else 2.0 ** (-149)
    _, e = math.frexp(t)
    return 2.0 ** (e - 1 - mantissa_bits)


def soft_threshold(v: np.ndarray, kappa: float) -> np.ndarray:
    """z-update of ADMM for h = gamma*||.||_1 (Sec. 2.1): sign(v) max(|v|-kappa, 0)."""
    return np.sign(v) * np.maximum(np.abs(v) - kappa, 0.0)


# ---------------------------------------------------------------------------
# Gaussian test matrix drawn by a counter-based generator (App. B draws Omega ~ N(0,1))
# ---------------------------------------------------------------------------

PHILOX_M = (0xD2511F53, 0xCD9E8D57)      # round multipliers of Philox-4x32
PHILOX_W = (0x9E3779B9, 0xBB67AE85)      # Weyl increments of its key schedule


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
    as easy as 1, 2, 3", SC 2011), vectorised over the leading axis.
    ctr: uint64 array (..., 4) of 32-bit words, key: (..., 2).  One round maps
    (c0, c1, c2, c3) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
    the key is bumped by the Weyl increments between rounds."""
    mask = np.uint64(0xFFFFFFFF)
    c = [np.asarray(ctr, dtype=np.uint64)[..., i] & mask for i in range(4)]
    k = [np.asarray(key, dtype=np.uint64)[..., i] & mask for i in range(2)]
    m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
    for _ in range(10):
        p0 = m0 * c[0]                       # < 2^64: exact in uint64
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
        k = [(k[0] + np.uint64(PHILOX_W[0])) & mask, (k[1] + np.uint64(PHILOX_W[1])) & mask]
    return np.stack(c, axis=-1)


def gaussian_test_matrix_philox(seed: int, d: int, s: int) -> np.ndarray:
    """Omega (d x s) with iid N(0,1) entries from Philox-4x32-10 and the Box-Muller
    transform; element e = i + j d (column-major) is member e mod 2 of pair m = e // 2:
      counter (lo32(m), hi32(m), 0, 0), key (lo32(seed), hi32(seed)) -> words w0..w3,
      u1 = ((w0 2^32 + w1) >> 11 + 1) 2^-53  in (0, 1],
      u2 = ((w2 2^32 + w3) >> 11) 2^-53      in [0, 1),
      g_even = sqrt(-2 ln u1) cos(2 pi u2),  g_odd = sqrt(-2 ln u1) sin(2 pi u2).
    The same definition is implemented on the device (nys_gaussian_test_matrix)."""
    n = d * s
    m = np.arange((n + 1) // 2, dtype=np.uint64)
    ctr = np.zeros((m.size, 4), dtype=np.uint64)
    ctr[:, 0] = m & np.uint64(0xFFFFFFFF)
    ctr[:, 1] = m >> np.uint64(32)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)
    w = philox4x32_10(ctr, np.broadcast_to(key, (m.size, 2)))
    a = ((w[:, 0] << np.uint64(32)) | w[:, 1]) >> np.uint64(11)
    b = ((w[:, 2] << np.uint64(32)) | w[:, 3]) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.empty(2 * m.size)
    g[0::2] = r * np.cos(2.0 * np.pi * u2)
    g[1::2] = r * np.sin(2.0 * np.pi * u2)
    return g[:n].reshape(s, d).T.copy()


# ---------------------------------------------------------------------------
# Randomized Nystrom approximation (App. B, Alg. Randomized Nystrom Approximation)
# ---------------------------------------------------------------------------

def thin_qr(Omega: np.ndarray) -> np.ndarray:
    """qr(Omega, 0): orthonormal basis of range(Omega) (Householder, LAPACK)."""
    Q, _ = np.linalg.qr(Omega, mode="reduced")
    return Q


def round_to_bf16(X: np.ndarray) -> np.ndarray:
    """Each entry rounded to the nearest BF16 value through FP32: FP64 -> FP32 to nearest,
    then the FP32 bit pattern rounded to its top 16 bits, to nearest with ties to even
    (returned as FP64).  Used for the test matrix of an FP32-class sketch."""
    f = np.asarray(X, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def sketch_test_matrix(Omega: np.ndarray, mantissa_bits: int = 52) -> np.ndarray:
    """The test matrix the sketch uses: qr(Omega, 0) (Alg. Randomized Nystrom
    Approximation), rounded to BF16 values for an FP32-class sketch (mantissa_bits = 23)."""
    Q = thin_qr(Omega)
    return round_to_bf16(Q) if mantissa_bits == 23 else Q


def nystrom_from_sketch(Y: np.ndarray, Omega: np.ndarray, shift_scale: float = 1.0,
                        mantissa_bits: int = 52, max_retries: int = 3):
    """Steps after Y = H Omega of the randomized Nystrom approximation:

        nu   = shift_scale * eps(||Y||_2)
        Y_nu = Y + nu * Omega
        C    = chol(Omega^T Y_nu)        (upper, C^T C = Omega^T Y_nu)
        B    = Y_nu / C                  (B C = Y_nu)
        [U, Sigma] = svd(B, 0)
        Lam  = max(0, Sigma^2 - nu)

    Returns (U, lam, nu) with lam sorted in descending order.
    """
    sigma_max = np.linalg.norm(Y, 2)
    nu = shift_scale * eps_of(sigma_max, mantissa_bits)
    for _ in range(max_retries + 1):
        Ynu = Y + nu * Omega
        M = Omega.T @ Ynu
        M = 0.5 * (M + M.T)
        try:
            C = np.linalg.cholesky(M).T          # upper triangular, C^T C = M
        except np.linalg.LinAlgError:
            nu *= 10.0
            continue
        if not np.all(np.isfinite(C)):
            nu *= 10.0
            continue
        # B C = Y_nu  <=>  C^T B^T = Y_nu^T
        B = sla.solve_triangular(C, Ynu.T, trans="T", lower=False).T
        U, S, _ = np.linalg.svd(B, full_matrices=False)
        lam = np.maximum(0.0, S * S - nu)
        return U, lam, nu
    raise NotSPDError("Omega^T Y_nu is not numerically SPD after shift retries")


def nystrom(H_apply, Omega: np.ndarray, shift_scale: float = 1.0, mantissa_bits: int = 52):
    """Alg. Randomized Nystrom Approximation: H_apply(X) returns H X.

    Omega is the Gaussian test matrix (d x s); it is orthonormalised here (and rounded
    to BF16 values for an FP32-class sketch, mantissa_bits = 23)."""
    Q = sketch_test_matrix(Omega, mantissa_bits)
    Y = H_apply(Q)
    U, lam, nu = nystrom_from_sketch(Y, Q, shift_scale, mantissa_bits)
    return U, lam, nu, Q, Y


def nystrom_definition(H: np.ndarray, Omega: np.ndarray) -> np.ndarray:
    """Eq. (Nystrom approximation): H<Omega> = (H Omega)(Omega^T H Omega)^+ (H Omega)^T."""
    HO = H @ Omega
    return HO @ np.linalg.pinv(Omega.T @ HO) @ HO.T


# ---------------------------------------------------------------------------
# Nystrom preconditioner (Sec. 2.2, Eq. Nystrom preconditioner)
# ---------------------------------------------------------------------------

def precond_apply(U: np.ndarray, lam: np.ndarray, rho: float, v: np.ndarray) -> np.ndarray:
    """P^{-1} v = (lam_s + rho) U (Lam + rho I)^{-1} U^T v + (I - U U^T) v."""
    lam_s = lam[-1]
    Utv = U.T @ v
    return (lam_s + rho) * (U @ (Utv / (lam + rho)))[..., ] + v - U @ Utv


def precond_dense(U: np.ndarray, lam: np.ndarray, rho: float):
    """Dense P and P^{-1} exactly as printed in Eq. (Nystrom preconditioner)."""
    d = U.shape[0]
    lam_s = lam[-1]
    I = np.eye(d)
    P = (U * (lam + rho)) @ U.T / (lam_s + rho) + (I - U @ U.T)
    Pinv = (lam_s + rho) * (U / (lam + rho)) @ U.T + (I - U @ U.T)
    return P, Pinv


def empirical_condition_number(lam: np.ndarray, rho: float) -> float:
    """Eq. (empirical condition number): (lam_s + rho) / rho."""
    return (lam[-1] + rho) / rho


def effective_dimension(H: np.ndarray, rho: float) -> float:
    """Eq. (effective dimension): tr(H (H + rho I)^{-1})."""
    ev = np.linalg.eigvalsh(H)
    ev = np.maximum(ev, 0.0)
    return float(np.sum(ev / (ev + rho)))


# ---------------------------------------------------------------------------
# Nystrom PCG (App. B, Alg. Nystrom PCG)
# ---------------------------------------------------------------------------

def pcg(H_apply, rho: float, U, lam, r: np.ndarray, x0: np.ndarray, tol: float,
        tol_mode: str = "rel", maxit: int | None = None, fixed_iters: int | None = None,
        wnorms: list | None = None):
    """Solve (H + rho I) x = r by PCG with the Nystrom preconditioner.

    U = None (or an empty basis) gives plain CG (P = I).
    Stopping test at the top of the loop, as printed: ||w||_2 > eps.
      tol_mode 'rel': eps = tol * ||r||;  'abs': eps = tol.
    fixed_iters: run exactly this many iterations (no stopping test).
    wnorms: if a list is given, ||w|| at every loop-top test is appended to it (a record
    only: it shows how far each stop decision lay from its threshold).
    Returns (x, iterations, ||w||)."""
    d = r.shape[0]
    if maxit is None:
        maxit = min(d, 1000)

    def Pinv(v):
        if U is None or U.shape[1] == 0:
            return v.copy()
        return precond_apply(U, lam, rho, v)

    def Hrho(v):
        return H_apply(v) + rho * v

    x = x0.astype(np.float64).copy()
    w = r - Hrho(x)
    y = Pinv(w)
    p = y.copy()
    thresh = tol * np.linalg.norm(r) if tol_mode == "rel" else tol
    it = 0
    while True:
        if wnorms is not None:
            wnorms.append(float(np.linalg.norm(w)))
        if fixed_iters is not None:
            if it >= fixed_iters:
                break
        else:
            if not (np.linalg.norm(w) > thresh) or it >= maxit:
                break
        v = Hrho(p)
        pv = p @ v
        if not (pv > 0.0) or not np.isfinite(pv):
            raise BreakdownError("p^T (H + rho I) p <= 0")
        alpha = (w @ y) / pv
        x = x + alpha * p
        w_new = w - alpha * v
        y_new = Pinv(w_new)
        beta = (w_new @ y_new) / (w @ y)
        p = y_new + beta * p
        w, y = w_new, y_new
        it += 1
    return x, it, float(np.linalg.norm(w))


# ---------------------------------------------------------------------------
# Lasso (Eq. 2) by NysADMM (Alg. NysADMM with Eq. ADMMSubProb, H^l = I, g = 0)
# ---------------------------------------------------------------------------

def lasso_objective(A, b, gamma, x) -> float:
    """Eq. (2): 1/2 ||A x - b||^2 + gamma ||x||_1."""
    res = A @ x - b
    return 0.5 * float(res @ res) + gamma * float(np.sum(np.abs(x)))


def lasso_kkt_eta(A, b, gamma, x) -> float:
    """Eq. (31): ||x - prox_{gamma||.||_1}(x - A^T(Ax - b))|| / (1 + ||x|| + ||Ax - b||)."""
    res = A @ x - b
    g = A.T @ res
    num = np.linalg.norm(x - soft_threshold(x - g, gamma))
    return float(num / (1.0 + np.linalg.norm(x) + np.linalg.norm(res)))


def lasso_dual_gap(A, b, gamma, x) -> float:
    """Primal minus dual objective at the dual-feasible point obtained by
    scaling the residual theta = (b - A x) * min(1, gamma / ||A^T (b - A x)||_inf).
    Dual of Eq. (2): max 1/2||b||^2 - 1/2||b - theta||^2 s.t. ||A^T theta||_inf <= gamma."""
    theta = b - A @ x
    s = np.max(np.abs(A.T @ theta))
    if s > gamma:
        theta = theta * (gamma / s)
    dual = 0.5 * float(b @ b) - 0.5 * float((b - theta) @ (b - theta))
    return lasso_objective(A, b, gamma, x) - dual


def lasso_nysadmm(A: np.ndarray, b: np.ndarray, gamma: float, rho: float, Omega: np.ndarray,
                  admm_iters: int, pcg_tol: float = 1e-8, pcg_tol_mode: str = "rel",
                  shift_scale: float | None = None, pcg_fixed=None, pcg_maxit=None,
                  eps_abs: float | None = None, eps_rel: float | None = None,
                  precond=None, mu: float = 0.0, A_inner: np.ndarray | None = None,
                  mantissa_bits: int = 52):
    """Alg. NysADMM for the lasso, and for any problem whose smooth part adds
    g(x) = mu/2 ||x||^2 (the elastic net of Sec. 3.1 has mu = 1 - gamma).

    A_inner (mixed form without residual correction): the matrix H of the sketch and of
    the x-subproblem is built from A_inner (the stored low-precision values, given in
    FP64), while q = A^T b keeps the problem matrix A.  This is the reading of the mixed
    precision form in which the low-precision copy serves only the sketch and PCG and no
    correction pass is made; its fixed point solves the perturbed problem
        min 1/2 x^T (A_inner^T A_inner + mu I) x - (A^T b)^T x + gamma ||x||_1.
    mantissa_bits: precision whose eps enters the sketch shift nu (52 for an FP64
    sketch, 23 for the FP32-class sketch of a low-precision copy).

    Sketch once (App. B) with H = A^T A + H^g, H^g = mu I, then for k = 0, 1, ...:
        r^k     = rho z - rho u + A^T b            (Eq. ADMMSubProb with l = 1/2||.-b||^2;
                                                    the H^g x and grad g terms cancel)
        x^{k+1} = PCG solve of (A^T A + mu I + rho I) x = r^k, warm-started at x^k
        z^{k+1} = S_{gamma/rho}(x^{k+1} + u^k)
        u^{k+1} = u^k + x^{k+1} - z^{k+1}
        r_p     = ||x^{k+1} - z^{k+1}||,  r_d = rho ||z^k - z^{k+1}||   (Sec. 2.1)
    pcg_tol_mode 'rnorm_pow': the decaying schedule of Sec. 5, ||w|| <= ||r^k|| / k^beta with
    beta = pcg_tol and k = 1, 2, ... (k = 0 would divide by zero), i.e. a relative test.
    pcg_tol_mode 'sqrt_rprd': the schedule of Sec. 5's experiments, ||w|| <= sqrt(r_p r_d) of
    the previous ADMM iteration (absolute), pcg_tol relative for the first solve.
    pcg_fixed: None, an int, or a per-iteration sequence of PCG iteration counts.
    Stops after admm_iters, or earlier when eps_abs/eps_rel are given and the
    residual test of Sec. 2.1 holds.
    Returns dict with x, z, u, U, lam, nu, and per-iteration traces."""
    n, d = A.shape
    if shift_scale is None:
        shift_scale = math.sqrt(d)
    Ah = A if A_inner is None else A_inner
    H_apply = lambda X: Ah.T @ (Ah @ X) + mu * X
    if precond is None:
        U, lam, nu, Q, _ = nystrom(H_apply, Omega, shift_scale, mantissa_bits)
    else:
        U, lam, nu = precond
    x = np.zeros(d)
    z = np.zeros(d)
    u = np.zeros(d)
    q = A.T @ b
    trace = {"pcg_iters": [], "r_p": [], "r_d": [], "z": [], "pcg_res": [], "r_norm": [],
             "pcg_thresh": [], "pcg_wnorms": []}
    for k in range(admm_iters):
        r = rho * z - rho * u + q
        fixed = None
        if pcg_fixed is not None:
            fixed = pcg_fixed if isinstance(pcg_fixed, int) else int(pcg_fixed[k])
        if pcg_tol_mode == "rnorm_pow":
            tol_k, mode_k = (k + 1.0) ** (-pcg_tol), "rel"
        elif pcg_tol_mode == "sqrt_rprd":
            # Sec. 5's experiments: eps^{k+1} = sqrt(r_p^k r_d^k), absolute; the first
            # solve has no residuals yet and uses pcg_tol relative
            if k == 0:
                tol_k, mode_k = pcg_tol, "rel"
            else:
                tol_k, mode_k = math.sqrt(trace["r_p"][-1] * trace["r_d"][-1]), "abs"
        else:
            tol_k, mode_k = pcg_tol, pcg_tol_mode
        wn = []
        x, it, res = pcg(H_apply, rho, U, lam, r, x, tol_k, mode_k,
                         maxit=pcg_maxit, fixed_iters=fixed, wnorms=wn)
        trace["pcg_thresh"].append(tol_k * float(np.linalg.norm(r)) if mode_k == "rel" else tol_k)
        trace["pcg_wnorms"].append(wn)
        z_old = z
        z = soft_threshold(x + u, gamma / rho)
        u = u + x - z
        r_p = float(np.linalg.norm(x - z))
        r_d = float(rho * np.linalg.norm(z_old - z))
        trace["pcg_iters"].append(it)
        trace["pcg_res"].append(res)
        trace["r_norm"].append(float(np.linalg.norm(r)))
        trace["r_p"].append(r_p)
        trace["r_d"].append(r_d)
        trace["z"].append(z.copy())
        if eps_abs is not None and eps_rel is not None:
            if (r_p <= eps_abs + eps_rel * max(np.linalg.norm(x), np.linalg.norm(z)) and
                    r_d <= eps_abs + eps_rel * np.linalg.norm(rho * u)):
                break
    return {"x": x, "z": z, "u": u, "U": U, "lam": lam, "nu": nu, "trace": trace}


def quadratic_l1_kkt_eta(G, q, gamma, x) -> float:
    """Prox-gradient fixed-point residual of min 1/2 x^T G x - q^T x + gamma ||x||_1,
    ||x - S_gamma(x - (G x - q))|| / (1 + ||x||): the analogue of Eq. (31) for the problem
    the mixed form without correction solves (G = A_inner^T A_inner, q = A^T b)."""
    g = G @ x - q
    return float(np.linalg.norm(x - soft_threshold(x - g, gamma)) / (1.0 + np.linalg.norm(x)))


# ---------------------------------------------------------------------------
# Elastic net (Sec. 3.1, Eq. 6)
# ---------------------------------------------------------------------------

def elastic_net_objective(A, b, gamma, x) -> float:
    """Eq. (6): 1/2 ||A x - b||^2 + 1/2 (1 - gamma) ||x||^2 + gamma ||x||_1."""
    res = A @ x - b
    return (0.5 * float(res @ res) + 0.5 * (1.0 - gamma) * float(x @ x)
            + gamma * float(np.sum(np.abs(x))))


def elastic_net_kkt_eta(A, b, gamma, x) -> float:
    """Relative prox-gradient fixed-point residual of Eq. (6), the analogue of
    Eq. (31) with the smooth part's gradient A^T(Ax - b) + (1 - gamma) x."""
    res = A @ x - b
    g = A.T @ res + (1.0 - gamma) * x
    num = np.linalg.norm(x - soft_threshold(x - g, gamma))
    return float(num / (1.0 + np.linalg.norm(x) + np.linalg.norm(res)))


def elastic_net_dual_gap(A, b, gamma, x) -> float:
    """Duality gap of Eq. (6) written as the lasso of the stacked data
    [A; sqrt(1 - gamma) I], [b; 0]: primal minus the lasso dual at the scaled
    stacked residual theta = [b - A x; -sqrt(1 - gamma) x] * min(1, gamma / ||stacked A^T theta||_inf)."""
    mu = 1.0 - gamma
    d = A.shape[1]
    At = np.vstack([A, math.sqrt(mu) * np.eye(d)])
    bt = np.concatenate([b, np.zeros(d)])
    theta = bt - At @ x
    s = np.max(np.abs(At.T @ theta))
    if s > gamma:
        theta = theta * (gamma / s)
    dual = 0.5 * float(bt @ bt) - 0.5 * float((bt - theta) @ (bt - theta))
    return elastic_net_objective(A, b, gamma, x) - dual


def elastic_net_nysadmm(A, b, gamma, rho, Omega, admm_iters, **kw):
    """Alg. NysADMM applied to Eq. (6): l = 1/2||. - b||^2, g = 1/2 (1 - gamma)||.||^2,
    h = gamma ||.||_1, so the sketched Hessian is A^T A + (1 - gamma) I (Sec. 3.1)."""
    return lasso_nysadmm(A, b, gamma, rho, Omega, admm_iters, mu=1.0 - gamma, **kw)


# ---------------------------------------------------------------------------
# Adaptive sketch size (App. C, Alg. AdaptiveRandNysAppx)
# ---------------------------------------------------------------------------

def adaptive_nystrom(H_apply, Omega_pool: np.ndarray, s0: int, s_max: int, rho: float,
                     tol: float, shift_scale: float | None = None, mantissa_bits: int = 52):
    """Alg. AdaptiveRandNysAppx.  Gaussian blocks are consecutive column slices
    of Omega_pool (d x s_max), each orthonormalised on its own; the sketch of
    earlier blocks is reused.  Returns (U, lam, nu, ranks_tried)."""
    d = Omega_pool.shape[0]
    if shift_scale is None:
        shift_scale = math.sqrt(d)
    Om = np.zeros((d, 0))
    Y = np.zeros((d, 0))
    m = s0
    used = 0
    ranks = []
    while True:
        Om0 = sketch_test_matrix(Omega_pool[:, used:used + m], mantissa_bits)
        used += m
        Y0 = H_apply(Om0)
        Om = np.hstack([Om, Om0])
        Y = np.hstack([Y, Y0])
        U, lam, nu = nystrom_from_sketch(Y, Om, shift_scale, mantissa_bits)
        ranks.append(Om.shape[1])
        if empirical_condition_number(lam, rho) <= tol:
            break
        m = s0
        s0 = 2 * s0
        if s0 > s_max:
            s0 = s0 - m
            m = s_max - s0
            if m > 0:
                Om0 = sketch_test_matrix(Omega_pool[:, used:used + m], mantissa_bits)
                used += m
                Y0 = H_apply(Om0)
                Om = np.hstack([Om, Om0])
                Y = np.hstack([Y, Y0])
                U, lam, nu = nystrom_from_sketch(Y, Om, shift_scale, mantissa_bits)
                ranks.append(Om.shape[1])
            break
    return U, lam, nu, ranks


# ---------------------------------------------------------------------------
# l1-regularised logistic regression (Sec. 3.2, Eq. 9)
# ---------------------------------------------------------------------------

def logistic_objective(A, b_pm, gamma, x) -> float:
    """Eq. (9) with labels mapped to {0,1} by b01 = (1 + b)/2:
    -sum_i (b01_i t_i - log(1 + exp(t_i))) + gamma ||x||_1,  t = A x."""
    b01 = 0.5 * (1.0 + b_pm)
    t = A @ x
    softplus = np.maximum(t, 0.0) + np.log1p(np.exp(-np.abs(t)))
    return float(np.sum(softplus - b01 * t) + gamma * np.sum(np.abs(x)))


def logistic_weights(t: np.ndarray, b01: np.ndarray):
    """Sec. 3.2: w_i = 1/(2 + e^{-t_i} + e^{t_i}),
    q_i = t_i + (b01_i - 1/(1 + e^{-t_i})) / w_i."""
    with np.errstate(over="ignore"):
        w = 1.0 / (2.0 + np.exp(-t) + np.exp(t))
        sig = 1.0 / (1.0 + np.exp(-t))
    q = t + (b01 - sig) / w
    if not np.all(np.isfinite(q)):
        raise FloatingPointError("logistic weight underflow (|A x| too large for this form)")
    return w, q


def logistic_nysadmm(A, b_pm, gamma, rho, Omega_pool, admm_iters, s0, s_max, ada_tol=2.0,
                     pcg_tol=1e-8, pcg_tol_mode="rel", pcg_fixed=None, resketch_every=1,
                     shift_scale=None):
    """Linearised ADMM for Eq. (9) (Sec. 3.2) with the Nystrom preconditioner
    from Alg. AdaptiveRandNysAppx.  At every outer iteration k:
        t = A x~,  w, q from Sec. 3.2,  H = A^T diag(w) A,
        r = rho z~ - rho u~ + A^T diag(w) q,
        x = PCG solve of (H + rho I) x = r (warm start x~),
        z = S_{gamma/rho}(x + u),  u = u + x - z.
    The rank is chosen adaptively at k = 0; later re-sketches (every
    resketch_every iterations) reuse the settled rank and the same Omega blocks."""
    n, d = A.shape
    b01 = 0.5 * (1.0 + b_pm)
    x = np.zeros(d)
    z = np.zeros(d)
    u = np.zeros(d)
    rank = None
    U = lam = None
    trace = {"pcg_iters": [], "rank": [], "obj": [], "r_p": [], "r_d": []}
    for k in range(admm_iters):
        t = A @ x
        w, q = logistic_weights(t, b01)
        H_apply = lambda X, w=w: A.T @ (w[:, None] * (A @ X)) if X.ndim == 2 else A.T @ (w * (A @ X))
        if k == 0:
            U, lam, nu, ranks = adaptive_nystrom(H_apply, Omega_pool, s0, s_max, rho, ada_tol,
                                                 shift_scale)
            rank = ranks[-1]
        elif resketch_every and k % resketch_every == 0:
            U, lam, nu, _ = adaptive_nystrom(H_apply, Omega_pool, rank, rank, rho, 0.0,
                                             shift_scale)
        r = rho * z - rho * u + A.T @ (w * q)
        fixed = None
        if pcg_fixed is not None:
            fixed = pcg_fixed if isinstance(pcg_fixed, int) else int(pcg_fixed[k])
        x, it, _ = pcg(H_apply, rho, U, lam, r, x, pcg_tol, pcg_tol_mode, fixed_iters=fixed)
        z_old = z
        z = soft_threshold(x + u, gamma / rho)
        u = u + x - z
        trace["pcg_iters"].append(it)
        trace["rank"].append(rank)
        trace["r_p"].append(float(np.linalg.norm(x - z)))
        trace["r_d"].append(float(rho * np.linalg.norm(z_old - z)))
    return {"x": x, "z": z, "u": u, "rank": rank, "trace": trace}


# ---------------------------------------------------------------------------
# Learned warm start: small MLP (two GELU hidden layers), FP64 reference
# ---------------------------------------------------------------------------
# Parameters are one flat vector [W1 (h x i), b1 (h), W2 (h x h), b2 (h), W3 (o x h), b3 (o)],
# weights row-major (output x input).  GELU(z) = z * Phi(z) (erf form).  Loss = mean over
# batch and outputs of (Y - T)^2.  Adam with bias correction.

def mlp_unpack(theta, n_in, n_hid, n_out):
    sizes = [(n_hid, n_in), (n_hid,), (n_hid, n_hid), (n_hid,), (n_out, n_hid), (n_out,)]
    out, off = [], 0
    for sh in sizes:
        cnt = int(np.prod(sh))
        out.append(np.asarray(theta[off:off + cnt], dtype=np.float64).reshape(sh))
        off += cnt
    return out


def mlp_param_count(n_in, n_hid, n_out):
    return n_hid * n_in + n_hid + n_hid * n_hid + n_hid + n_out * n_hid + n_out


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def mlp_forward(theta, X, n_in, n_hid, n_out):
    """Y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3 for each row x of X (B x n_in)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta, n_in, n_hid, n_out)
    Z1 = X @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (Z1, H1, Z2, H2)


def mlp_loss_grad(theta, X, T, n_in, n_hid, n_out):
    """Mean-squared loss and its gradient (backpropagation written out)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta, n_in, n_hid, n_out)
    Y, (Z1, H1, Z2, H2) = mlp_forward(theta, X, n_in, n_hid, n_out)
    B = X.shape[0]
    R = Y - T
    loss = float(np.sum(R * R) / (B * n_out))
    dY = 2.0 * R / (B * n_out)
    dW3 = dY.T @ H2
    db3 = dY.sum(axis=0)
    dZ2 = (dY @ W3) * gelu_grad(Z2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, g


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
