"""Pins for the FP64 oracle: each check ties the oracle to something other than
itself -- closed forms, textbook/library solvers, brute force on tiny inputs,
and the lemmas and propositions of the paper (App. A).  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt
import scipy.sparse.linalg as spla
from scipy.special import expit

import nys_inputs as gen
import oracle.nysadmm_oracle as o


def _spd_decay(d, seed, r=None, decay=1.0, n=None):
    """H = A^T A for a polynomially decaying A (rank r if given)."""
    rng = np.random.default_rng(seed)
    n = n or 3 * d
    if r is None:
        A = rng.standard_normal((n, d)) * gen.column_scales(d, decay)[None, :]
    else:
        A = rng.standard_normal((n, r)) @ rng.standard_normal((r, d))
    return A, A.T @ A


# ---------------------------------------------------------------- scalars

def check_eps():
    for t in [1.0, 0.75, 3.0, 1e-3, 12345.678, 2.0 ** 40, 1e300]:
        assert o.eps_of(t) == np.spacing(t), t
        t32 = np.float32(t) if t < 3e38 else None
        if t32 is not None:
            assert o.eps_of(float(t32), 23) == float(np.spacing(t32)), t
    assert o.eps_of(1.0) == np.finfo(np.float64).eps


def test_eps_matches_numpy_spacing():
    check_eps()


def check_soft_threshold():
    rng = np.random.default_rng(3)
    v = rng.standard_normal(40) * 3
    kap = 0.7
    got = o.soft_threshold(v, kap)
    for vi, gi in zip(v, got):
        res = sopt.minimize_scalar(lambda z: kap * abs(z) + 0.5 * (z - vi) ** 2,
                                   bounds=(-10, 10), method="bounded",
                                   options={"xatol": 1e-12})
        assert abs(res.x - gi) < 1e-7


def test_soft_threshold_is_prox_of_l1():
    check_soft_threshold()


# ---------------------------------------------------------------- Nystrom

def check_nystrom_definition(seed=0, d=60, s=12):
    _, H = _spd_decay(d, seed)
    Om = gen.gaussian_test_matrix(d, s, seed + 100)
    U, lam, nu, Q, Y = o.nystrom(lambda X: H @ X, Om, shift_scale=1.0)
    Hhat = (U * lam) @ U.T
    Hdef = o.nystrom_definition(H, Om)          # Eq. (Nystrom approximation), pinv form
    scale = np.linalg.norm(H, 2)
    assert np.linalg.norm(Hhat - Hdef, 2) <= 1e-10 * scale
    # B B^T = Y_nu (Omega^T Y_nu)^{-1} Y_nu^T, i.e. U diag(Sigma^2) U^T with Sigma^2 = lam + nu
    Ynu = Y + nu * Q
    BBt = Ynu @ np.linalg.inv(Q.T @ Ynu) @ Ynu.T
    assert np.linalg.norm((U * (lam + nu)) @ U.T - BBt, 2) <= 1e-10 * scale
    # descending order, orthonormal U
    assert np.all(np.diff(lam) <= 0)
    assert np.linalg.norm(U.T @ U - np.eye(s)) < 1e-10


def test_nystrom_matches_pinv_definition():
    check_nystrom_definition()


def check_nystrom_lemma_properties(seed=1, d=50, s=10):
    """Lemma (Nystrom properties, App. A): psd, rank <= s, depends only on
    range(Omega), H<Omega> <= H in Loewner order, eigenvalue interlacing."""
    _, H = _spd_decay(d, seed)
    Om = gen.gaussian_test_matrix(d, s, seed + 7)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om, shift_scale=1.0)
    Hhat = (U * lam) @ U.T
    scale = np.linalg.norm(H, 2)
    ev = np.linalg.eigvalsh(Hhat)
    assert ev.min() >= -1e-12 * scale
    assert np.sum(ev > 1e-10 * scale) <= s
    assert np.linalg.eigvalsh(H - Hhat).min() >= -1e-10 * scale
    evH = np.sort(np.linalg.eigvalsh(H))[::-1]
    assert np.all(np.sort(ev)[::-1] <= evH + 1e-10 * scale)
    # range-only: Omega -> Omega R for an invertible R
    R = np.random.default_rng(seed).standard_normal((s, s)) + 3 * np.eye(s)
    U2, lam2, _, _, _ = o.nystrom(lambda X: H @ X, Om @ R, shift_scale=1.0)
    assert np.linalg.norm((U2 * lam2) @ U2.T - Hhat, 2) <= 1e-9 * scale


def test_nystrom_lemma_properties():
    check_nystrom_lemma_properties()


def check_nystrom_exact_low_rank(seed=2, d=40, r=6, s=10):
    """s > rank(H): the Nystrom approximation reproduces H, so the top r
    eigenvalues equal those of H and the rest vanish."""
    A, H = _spd_decay(d, seed, r=r)
    Om = gen.gaussian_test_matrix(d, s, seed)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om, shift_scale=1.0)
    evH = np.sort(np.linalg.eigvalsh(H))[::-1]
    assert np.allclose(lam[:r], evH[:r], rtol=1e-10, atol=0)
    assert np.all(lam[r:] <= 1e-10 * evH[0])
    assert np.linalg.norm((U * lam) @ U.T - H, 2) <= 1e-10 * evH[0]


def test_nystrom_exact_when_rank_exceeds_H():
    check_nystrom_exact_low_rank()


def test_round_to_bf16_matches_torch_cast():
    """The BF16 rounding of the FP32-class test matrix against torch's float32 -> bfloat16
    cast (round to nearest, ties to even), on random values and on exact ties."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(4000), rng.standard_normal(1000) * 1e-30, [0.0, -0.0, 1.0, -3.5]])
    f = x.astype(np.float32)
    # exact ties: low 16 bits 0x8000, upper halves even and odd
    hi = rng.integers(0x3000, 0x4800, size=200).astype(np.uint32)
    ties = ((hi << 16) | 0x8000).view(np.float32)
    f = np.concatenate([f, ties, -ties])
    ref = torch.from_numpy(f).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    got = o.round_to_bf16(f.astype(np.float64))
    assert np.array_equal(got, ref)


def test_nystrom_fp32_class_test_matrix():
    """mantissa_bits = 23: the test matrix is qr(Omega, 0) rounded to BF16 values (within
    2^-8 of each entry, orthonormal to ~2^-7), and the approximation still reproduces an H of rank
    below s (any full-rank test matrix does), up to the FP32-eps shift."""
    A, H = _spd_decay(40, 2, r=6)
    Om = gen.gaussian_test_matrix(40, 10, 2)
    U, lam, nu, Q, _ = o.nystrom(lambda X: H @ X, Om, shift_scale=1.0, mantissa_bits=23)
    Q0 = o.thin_qr(Om)
    bits = Q.astype(np.float32).view(np.uint32)
    assert np.all((bits & 0xFFFF) == 0) and np.array_equal(Q.astype(np.float32).astype(np.float64), Q)
    assert np.all(np.abs(Q - Q0) <= 2.0 ** -8 * np.abs(Q0) * (1 + 1e-6))   # half a BF16 ulp
    assert 0 < np.linalg.norm(Q.T @ Q - np.eye(10), 2) <= 2.0 ** -6
    evH = np.sort(np.linalg.eigvalsh(H))[::-1]
    assert np.linalg.norm((U * lam) @ U.T - H, 2) <= 1e-5 * evH[0]


# ---------------------------------------------------------------- preconditioner

def check_precond_inverse(seed=3, d=45, s=9, rho=0.3):
    _, H = _spd_decay(d, seed)
    Om = gen.gaussian_test_matrix(d, s, seed)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om)
    lam_s = lam[-1]
    # P as printed (first line of Eq. Nystrom preconditioner), inverted by LAPACK
    P = (U * (lam + rho)) @ U.T / (lam_s + rho) + (np.eye(d) - U @ U.T)
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((d, 3))
    for j in range(3):
        got = o.precond_apply(U, lam, rho, V[:, j])
        ref = np.linalg.solve(P, V[:, j])
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_precond_apply_inverts_P():
    check_precond_inverse()


def check_precond_exact(seed=4, d=30, r=5, s=8, rho=0.5):
    """s > rank(H): P^{-1}(H + rho I) = rho I."""
    _, H = _spd_decay(d, seed, r=r)
    Om = gen.gaussian_test_matrix(d, s, seed)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om)
    Hrho = H + rho * np.eye(d)
    M = np.column_stack([o.precond_apply(U, lam, rho, Hrho[:, j]) for j in range(d)])
    assert np.linalg.norm(M - rho * np.eye(d), 2) <= 1e-8 * np.linalg.norm(Hrho, 2)


def test_precond_exact_low_rank():
    check_precond_exact()


def check_condition_bound(seed=5, d=60, s=12, rho=0.05):
    """Proposition (deterministic bound, App. A):
    kappa(P^{-1/2} H_rho P^{-1/2}) <= (lam_s + rho + ||E||)/rho, E = H - Hhat."""
    _, H = _spd_decay(d, seed)
    Om = gen.gaussian_test_matrix(d, s, seed)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om)
    Hrho = H + rho * np.eye(d)
    P = (U * (lam + rho)) @ U.T / (lam[-1] + rho) + (np.eye(d) - U @ U.T)
    ev = sla.eigh(Hrho, P, eigvals_only=True)       # spectrum of P^{-1} H_rho
    kappa = ev.max() / ev.min()
    E = H - (U * lam) @ U.T
    bound = (lam[-1] + rho + np.linalg.norm(E, 2)) / rho
    assert kappa <= bound * (1 + 1e-9)
    assert o.empirical_condition_number(lam, rho) == pytest.approx((lam[-1] + rho) / rho)


def test_deterministic_condition_bound():
    check_condition_bound()


def test_effective_dimension_diagonal():
    lam = np.array([10.0, 3.0, 1.0, 0.1, 0.0])
    rho = 0.5
    assert o.effective_dimension(np.diag(lam), rho) == pytest.approx(
        sum(l / (l + rho) for l in lam), rel=1e-14)


# ---------------------------------------------------------------- PCG

def check_pcg_direct(seed=6, d=80, s=10, rho=0.1):
    _, H = _spd_decay(d, seed)
    Om = gen.gaussian_test_matrix(d, s, seed)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(d)
    x0 = rng.standard_normal(d)
    x, it, _ = o.pcg(lambda v: H @ v, rho, U, lam, r, x0, 1e-13)
    ref = sla.cho_solve(sla.cho_factor(H + rho * np.eye(d)), r)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert it > 0


def test_pcg_matches_cholesky_solve():
    check_pcg_direct()


def check_pcg_iterates_match_scipy(seed=7, d=50, s=6, rho=0.2, k=5):
    """The k-th PCG iterate equals scipy's preconditioned CG k-th iterate (M = P^{-1})."""
    _, H = _spd_decay(d, seed)
    Om = gen.gaussian_test_matrix(d, s, seed)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(d)
    x0 = rng.standard_normal(d)
    for with_p in (False, True):
        iters = []
        M = spla.LinearOperator((d, d), matvec=lambda v: o.precond_apply(U, lam, rho, v)) if with_p else None
        spla.cg(H + rho * np.eye(d), r, x0=x0.copy(), rtol=1e-300, atol=0.0, maxiter=k, M=M,
                callback=lambda xk: iters.append(xk.copy()))
        xk, it, _ = o.pcg(lambda v: H @ v, rho, U if with_p else None, lam, r, x0, 0.0,
                          fixed_iters=k)
        assert it == k
        assert np.linalg.norm(xk - iters[k - 1]) <= 1e-9 * np.linalg.norm(iters[k - 1])


def test_pcg_iterates_match_scipy_cg():
    check_pcg_iterates_match_scipy()


def check_pcg_one_iteration_exact(seed=8, d=40, r=5, s=9, rho=0.7):
    _, H = _spd_decay(d, seed, r=r)
    Om = gen.gaussian_test_matrix(d, s, seed)
    U, lam, _, _, _ = o.nystrom(lambda X: H @ X, Om)
    rhs = np.random.default_rng(seed).standard_normal(d)
    x, it, _ = o.pcg(lambda v: H @ v, rho, U, lam, rhs, np.zeros(d), 1e-9)
    assert it == 1
    ref = np.linalg.solve(H + rho * np.eye(d), rhs)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


def test_pcg_one_iteration_when_exact():
    check_pcg_one_iteration_exact()


def test_pcg_zero_iterations_when_converged():
    d = 10
    H = np.eye(d)
    x_exact = np.arange(d, dtype=float)
    r = (H + 1.0 * np.eye(d)) @ x_exact
    x, it, _ = o.pcg(lambda v: H @ v, 1.0, None, None, r, x_exact, 1e-12)
    assert it == 0 and np.array_equal(x, x_exact)


def test_pcg_breakdown_detected():
    d = 6
    H = -3.0 * np.eye(d)                          # H + rho I indefinite: not a valid input
    with pytest.raises(o.BreakdownError):
        o.pcg(lambda v: H @ v, 1.0, None, None, np.ones(d), np.zeros(d), 1e-12)


# ---------------------------------------------------------------- lasso

def _lasso_run(A, b, gamma, rho=1.0, s=None, iters=300, seed=0):
    d = A.shape[1]
    s = s or min(d, 8)
    Om = gen.gaussian_test_matrix(d, s, seed)
    return o.lasso_nysadmm(A, b, gamma, rho, Om, iters, pcg_tol=1e-13)


def check_lasso_orthonormal(seed=9):
    A = gen.orthonormal_columns(60, 12, seed)
    b = np.random.default_rng(seed).standard_normal(60) * 2
    gamma = 0.4
    out = _lasso_run(A, b, gamma, rho=1.0, s=4, iters=200)
    ref = np.sign(A.T @ b) * np.maximum(np.abs(A.T @ b) - gamma, 0)
    assert np.linalg.norm(out["z"] - ref) <= 1e-9 * max(1.0, np.linalg.norm(ref))


def test_lasso_orthonormal_closed_form():
    check_lasso_orthonormal()


def check_lasso_zero(seed=10):
    p = gen.lasso_problem(80, 20, seed=seed)
    gamma = 1.0001 * np.max(np.abs(p.A.T @ p.b))
    out = _lasso_run(p.A, p.b, gamma, iters=100)
    assert np.max(np.abs(out["z"])) == 0.0


def test_lasso_large_gamma_gives_zero():
    check_lasso_zero()


def check_lasso_least_squares(seed=11):
    p = gen.lasso_problem(90, 15, seed=seed)
    out = _lasso_run(p.A, p.b, 0.0, rho=1.0, s=6, iters=400)
    ref = np.linalg.lstsq(p.A, p.b, rcond=None)[0]
    assert np.linalg.norm(out["x"] - ref) <= 1e-8 * np.linalg.norm(ref)


def test_lasso_gamma_zero_is_least_squares():
    check_lasso_least_squares()


def _lasso_brute_force(A, b, gamma):
    """Enumerate sign patterns s in {-1,0,1}^d; on the support solve the
    stationarity equations A_S^T (A_S x_S - b) + gamma s_S = 0 and keep the
    sign-consistent candidate of least objective."""
    import itertools
    d = A.shape[1]
    best, best_x = np.inf, None
    for pat in itertools.product((-1, 0, 1), repeat=d):
        S = [j for j in range(d) if pat[j] != 0]
        x = np.zeros(d)
        if S:
            As = A[:, S]
            sg = np.array([pat[j] for j in S], float)
            try:
                xs = np.linalg.solve(As.T @ As, As.T @ b - gamma * sg)
            except np.linalg.LinAlgError:
                continue
            if np.any(np.sign(xs) != sg):
                continue
            x[S] = xs
        f = 0.5 * np.sum((A @ x - b) ** 2) + gamma * np.sum(np.abs(x))
        if f < best:
            best, best_x = f, x
    return best_x, best


def check_lasso_brute_force(seed=12):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((25, 5)) * gen.column_scales(5, 0.5)[None, :]
    b = rng.standard_normal(25)
    gamma = 0.3 * np.max(np.abs(A.T @ b))
    ref, fref = _lasso_brute_force(A, b, gamma)
    out = _lasso_run(A, b, gamma, rho=1.0, s=3, iters=2000)
    assert np.linalg.norm(out["z"] - ref) <= 1e-7 * max(1, np.linalg.norm(ref))
    assert o.lasso_objective(A, b, gamma, out["z"]) == pytest.approx(fref, rel=1e-10)


def test_lasso_brute_force_tiny():
    check_lasso_brute_force()


def check_lasso_kkt_and_gap(seed=13):
    p = gen.lasso_problem(300, 60, nnz=6, seed=seed)
    out = _lasso_run(p.A, p.b, p.gamma, rho=10.0, s=20, iters=800)
    z = out["z"]
    assert o.lasso_kkt_eta(p.A, p.b, p.gamma, z) <= 1e-10
    F = o.lasso_objective(p.A, p.b, p.gamma, z)
    gap = o.lasso_dual_gap(p.A, p.b, p.gamma, z)
    assert 0 <= gap <= 1e-10 * F
    # duality gap of a poor point is positive and bounds its suboptimality
    zb = z + 0.01
    assert o.lasso_dual_gap(p.A, p.b, p.gamma, zb) >= o.lasso_objective(p.A, p.b, p.gamma, zb) - F


def test_lasso_kkt_and_duality_gap_at_convergence():
    check_lasso_kkt_and_gap()


# ---------------------------------------------------------------- mixed form without correction
# (BF16 copy of A for the sketch and the x-subproblem, A^T b from the FP64 matrix)

def _bf16_values(A):
    """Values of A rounded to BF16 (round to nearest even), returned in FP64."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(A)).to(torch.bfloat16).to(torch.float64).numpy()


def _quadratic_l1_brute_force(G, q, gamma):
    """min 1/2 x^T G x - q^T x + gamma ||x||_1 by enumerating sign patterns s in {-1,0,1}^d:
    on the support solve G_SS x_S = q_S - gamma s_S, keep the sign-consistent candidate of
    least objective."""
    import itertools
    d = G.shape[0]
    best, best_x = np.inf, None
    for pat in itertools.product((-1, 0, 1), repeat=d):
        S = [j for j in range(d) if pat[j] != 0]
        x = np.zeros(d)
        if S:
            sg = np.array([pat[j] for j in S], float)
            xs = np.linalg.solve(G[np.ix_(S, S)], q[S] - gamma * sg)
            if np.any(np.sign(xs) != sg):
                continue
            x[S] = xs
        f = 0.5 * x @ G @ x - q @ x + gamma * np.sum(np.abs(x))
        if f < best:
            best, best_x = f, x
    return best_x, best


def check_mixed_form_inner_equal_to_A_is_plain(seed=30):
    p = gen.lasso_problem(200, 30, nnz=5, seed=seed)
    Om = gen.gaussian_test_matrix(30, 8, seed)
    a = o.lasso_nysadmm(p.A, p.b, p.gamma, 1.0, Om, 40, pcg_tol=1e-10)
    b = o.lasso_nysadmm(p.A, p.b, p.gamma, 1.0, Om, 40, pcg_tol=1e-10, A_inner=p.A)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["z"], b["z"])


def test_mixed_form_with_inner_equal_to_A_is_the_plain_method():
    check_mixed_form_inner_equal_to_A_is_plain()


def check_mixed_form_fixed_point(seed=31):
    """The mixed form without correction converges to the minimiser of the perturbed
    problem 1/2 x^T (Aq^T Aq) x - (A^T b)^T x + gamma ||x||_1 (Aq = BF16 values of A):
    brute force over sign patterns and its prox-gradient residual.  The perturbation is
    visible: the lasso minimiser of A, and the problem with q = Aq^T b, differ from it."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((40, 5)) * gen.column_scales(5, 0.5)[None, :]
    b = rng.standard_normal(40)
    gamma = 0.2 * np.max(np.abs(A.T @ b))
    Aq = _bf16_values(A)
    Om = gen.gaussian_test_matrix(5, 3, seed)
    out = o.lasso_nysadmm(A, b, gamma, 1.0, Om, 3000, pcg_tol=1e-13, A_inner=Aq, mantissa_bits=23)
    G, q = Aq.T @ Aq, A.T @ b
    ref, _ = _quadratic_l1_brute_force(G, q, gamma)
    z = out["z"]
    assert np.linalg.norm(z - ref) <= 1e-8 * max(1.0, np.linalg.norm(ref))
    assert o.quadratic_l1_kkt_eta(G, q, gamma, z) <= 1e-10
    plain, _ = _lasso_brute_force(A, b, gamma)
    other_q, _ = _quadratic_l1_brute_force(G, Aq.T @ b, gamma)
    assert np.linalg.norm(ref - plain) >= 1e-5 * np.linalg.norm(ref)
    assert np.linalg.norm(ref - other_q) >= 1e-5 * np.linalg.norm(ref)


def test_mixed_form_fixed_point_solves_the_perturbed_problem():
    check_mixed_form_fixed_point()


def test_quadratic_l1_eta_is_the_lasso_eta_numerator():
    """With G = A^T A and q = A^T b the quadratic problem is the lasso: both residuals
    share the numerator ||x - S_gamma(x - grad)|| (Eq. 31) and differ in the scaling."""
    p = gen.lasso_problem(60, 12, seed=32)
    x = np.random.default_rng(32).standard_normal(12)
    res = p.A @ x - p.b
    num_q = o.quadratic_l1_kkt_eta(p.A.T @ p.A, p.A.T @ p.b, p.gamma, x) * (1 + np.linalg.norm(x))
    num_l = o.lasso_kkt_eta(p.A, p.b, p.gamma, x) * (1 + np.linalg.norm(x) + np.linalg.norm(res))
    assert num_q == pytest.approx(num_l, rel=1e-12)
    xs, _ = _quadratic_l1_brute_force(p.A[:, :5].T @ p.A[:, :5], p.A[:, :5].T @ p.b, p.gamma)
    assert o.quadratic_l1_kkt_eta(p.A[:, :5].T @ p.A[:, :5], p.A[:, :5].T @ p.b, p.gamma, xs) <= 1e-12


def test_lasso_residuals_decrease_and_record():
    p = gen.lasso_small(0)
    Om = gen.gaussian_test_matrix(500, 50, 0)
    out = o.lasso_nysadmm(p.A, p.b, p.gamma, p.rho, Om, 40)
    tr = out["trace"]
    assert len(tr["pcg_iters"]) == 40
    assert tr["r_p"][-1] < tr["r_p"][0]
    assert max(tr["pcg_iters"][1:]) <= 30


def check_rnorm_pow_schedule(seed=14, beta=1.5):
    """Sec. 5's decaying schedule: every x-step stops at the first PCG iterate with
    ||w|| <= ||r^k|| / k^beta (k = 1, 2, ...), and the summable tolerances reach the
    lasso solution (KKT eta)."""
    p = gen.lasso_problem(300, 60, nnz=6, seed=seed)
    Om = gen.gaussian_test_matrix(60, 20, seed)
    out = o.lasso_nysadmm(p.A, p.b, p.gamma, 10.0, Om, 300, pcg_tol=beta, pcg_tol_mode="rnorm_pow")
    tr = out["trace"]
    for k in range(300):
        assert tr["pcg_res"][k] <= tr["r_norm"][k] / (k + 1.0) ** beta
    # minimality at a few iterations: one PCG iteration fewer misses the threshold
    U, lam = out["U"], out["lam"]
    H = lambda X: p.A.T @ (p.A @ X)
    x = np.zeros(60); z = np.zeros(60); u = np.zeros(60); q = p.A.T @ p.b
    checked = 0
    for k in range(40):
        r = 10.0 * (z - u) + q
        it = tr["pcg_iters"][k]
        if it > 0 and checked < 5:
            _, _, res_short = o.pcg(H, 10.0, U, lam, r, x, 0.0, "abs", fixed_iters=it - 1)
            assert res_short > np.linalg.norm(r) / (k + 1.0) ** beta
            checked += 1
        x, _, _ = o.pcg(H, 10.0, U, lam, r, x, 0.0, "abs", fixed_iters=it)
        zn = o.soft_threshold(x + u, p.gamma / 10.0)
        u = u + x - zn
        z = zn
    assert checked == 5
    # summable tolerances (beta > 1): the iterates approach the solution, at a rate that
    # follows the schedule (the error of an inexact step is O(k^-beta))
    e300 = o.lasso_kkt_eta(p.A, p.b, p.gamma, out["z"])
    out2 = o.lasso_nysadmm(p.A, p.b, p.gamma, 10.0, Om, 800, pcg_tol=2.0, pcg_tol_mode="rnorm_pow")
    e800 = o.lasso_kkt_eta(p.A, p.b, p.gamma, out2["z"])
    assert e800 < e300 and e800 <= 3e-6


def test_rnorm_pow_schedule_threshold_minimal_and_converges():
    check_rnorm_pow_schedule()


def check_sqrt_rprd_schedule(seed=15):
    """Sec. 5's experiment schedule: the x-step of iteration k >= 1 stops at the first PCG
    iterate with ||w|| <= sqrt(r_p r_d) of iteration k - 1 (one iteration fewer misses it),
    the first at pcg_tol relative; the iterates reach the lasso solution."""
    p = gen.lasso_problem(300, 60, nnz=6, seed=seed)
    Om = gen.gaussian_test_matrix(60, 20, seed)
    out = o.lasso_nysadmm(p.A, p.b, p.gamma, 10.0, Om, 200, pcg_tol=1e-3, pcg_tol_mode="sqrt_rprd")
    tr = out["trace"]
    assert tr["pcg_res"][0] <= 1e-3 * tr["r_norm"][0]
    for k in range(1, 200):
        assert tr["pcg_res"][k] <= math.sqrt(tr["r_p"][k - 1] * tr["r_d"][k - 1])
    U, lam = out["U"], out["lam"]
    H = lambda X: p.A.T @ (p.A @ X)
    x = np.zeros(60); z = np.zeros(60); u = np.zeros(60); q = p.A.T @ p.b
    checked = 0
    for k in range(30):
        r = 10.0 * (z - u) + q
        it = tr["pcg_iters"][k]
        if k > 0 and it > 0 and checked < 5:
            _, _, res_short = o.pcg(H, 10.0, U, lam, r, x, 0.0, "abs", fixed_iters=it - 1)
            assert res_short > math.sqrt(tr["r_p"][k - 1] * tr["r_d"][k - 1])
            checked += 1
        x, _, _ = o.pcg(H, 10.0, U, lam, r, x, 0.0, "abs", fixed_iters=it)
        zn = o.soft_threshold(x + u, p.gamma / 10.0)
        u = u + x - zn
        z = zn
    assert checked == 5
    assert o.lasso_kkt_eta(p.A, p.b, p.gamma, out["z"]) <= 1e-9


def test_sqrt_rprd_schedule_threshold_minimal_and_converges():
    check_sqrt_rprd_schedule()


def test_rnorm_pow_beta_zero_takes_no_first_step():
    # beta = 0: the first threshold is ||r^0|| itself, met by x0 = 0 before any iteration
    p = gen.lasso_small(0)
    Om = gen.gaussian_test_matrix(500, 50, 0)
    out = o.lasso_nysadmm(p.A, p.b, p.gamma, p.rho, Om, 3, pcg_tol=0.0, pcg_tol_mode="rnorm_pow")
    assert out["trace"]["pcg_iters"][0] == 0


# ---------------------------------------------------------------- elastic net

def _enet_run(A, b, gamma, rho=1.0, s=None, iters=300, seed=0):
    d = A.shape[1]
    s = s or min(d, 8)
    Om = gen.gaussian_test_matrix(d, s, seed)
    return o.elastic_net_nysadmm(A, b, gamma, rho, Om, iters, pcg_tol=1e-13)


def check_elastic_net_orthonormal(seed=21):
    # A^T A = I: the minimiser of Eq. (6) is S_gamma(A^T b) / (2 - gamma)
    A = gen.orthonormal_columns(60, 12, seed)
    b = np.random.default_rng(seed).standard_normal(60) * 2
    gamma = 0.6
    out = _enet_run(A, b, gamma, rho=1.0, s=4, iters=200)
    ref = np.sign(A.T @ b) * np.maximum(np.abs(A.T @ b) - gamma, 0) / (2.0 - gamma)
    assert np.linalg.norm(out["z"] - ref) <= 1e-9 * max(1.0, np.linalg.norm(ref))


def test_elastic_net_orthonormal_closed_form():
    check_elastic_net_orthonormal()


def check_elastic_net_augmented_brute_force(seed=22):
    # Eq. (6) is the lasso of the stacked data [A; sqrt(1-gamma) I], [b; 0]:
    # its sign-pattern enumeration is independent of the ADMM iteration
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((20, 5)) * gen.column_scales(5, 0.5)[None, :]
    b = rng.standard_normal(20)
    gamma = 0.3
    At = np.vstack([A, math.sqrt(1.0 - gamma) * np.eye(5)])
    bt = np.concatenate([b, np.zeros(5)])
    ref, fref = _lasso_brute_force(At, bt, gamma)
    out = _enet_run(A, b, gamma, rho=1.0, s=3, iters=1500)
    assert np.linalg.norm(out["z"] - ref) <= 1e-7 * max(1, np.linalg.norm(ref))
    assert o.elastic_net_objective(A, b, gamma, out["z"]) == pytest.approx(fref, rel=1e-10)


def test_elastic_net_augmented_lasso_brute_force():
    check_elastic_net_augmented_brute_force()


def check_elastic_net_kkt(seed=23):
    p = gen.lasso_problem(300, 60, nnz=6, seed=seed)
    gamma = 0.5 * np.max(np.abs(p.A.T @ p.b)) / (1 + np.max(np.abs(p.A.T @ p.b)))
    out = _enet_run(p.A, p.b, gamma, rho=10.0, s=20, iters=600)
    z = out["z"]
    assert o.elastic_net_kkt_eta(p.A, p.b, gamma, z) <= 1e-10
    F = o.elastic_net_objective(p.A, p.b, gamma, z)
    assert 0 <= o.elastic_net_dual_gap(p.A, p.b, gamma, z) <= 1e-10 * F
    zb = z + 0.01      # the gap bounds the suboptimality of any point
    assert o.elastic_net_dual_gap(p.A, p.b, gamma, zb) >= o.elastic_net_objective(p.A, p.b, gamma, zb) - F > 0
    # the minimiser of the lasso part alone is worse for Eq. (6)
    lz = _lasso_run(p.A, p.b, gamma, rho=10.0, s=20, iters=600)["z"]
    assert o.elastic_net_objective(p.A, p.b, gamma, out["z"]) < o.elastic_net_objective(p.A, p.b, gamma, lz)


def test_elastic_net_kkt_at_convergence():
    check_elastic_net_kkt()


def check_elastic_net_small_gamma_is_ridge(seed=24):
    # gamma -> 0: Eq. (6) tends to ridge regression with weight 1,
    # x = (A^T A + I)^{-1} A^T b; the l1 term moves the minimiser by O(gamma)
    p = gen.lasso_problem(200, 40, nnz=5, seed=seed)
    gamma = 1e-9
    out = _enet_run(p.A, p.b, gamma, rho=1.0, s=10, iters=300)
    ref = np.linalg.solve(p.A.T @ p.A + np.eye(40), p.A.T @ p.b)
    assert np.linalg.norm(out["x"] - ref) <= 1e-7 * np.linalg.norm(ref)


def test_elastic_net_small_gamma_is_ridge():
    check_elastic_net_small_gamma_is_ridge()


def test_elastic_net_gamma_one_is_the_lasso():
    p = gen.lasso_small(0)
    Om = gen.gaussian_test_matrix(500, 50, 0)
    a = o.elastic_net_nysadmm(p.A, p.b, 1.0, p.rho, Om, 5, pcg_fixed=4)
    c = o.lasso_nysadmm(p.A, p.b, 1.0, p.rho, Om, 5, pcg_fixed=4)
    assert np.array_equal(a["z"], c["z"])


# ---------------------------------------------------------------- logistic

def test_logistic_weights_identities():
    rng = np.random.default_rng(14)
    t = rng.standard_normal(50) * 4
    b01 = (rng.random(50) > 0.5).astype(float)
    w, q = o.logistic_weights(t, b01)
    assert np.allclose(w, expit(t) * expit(-t), rtol=1e-13)
    assert np.allclose(w * q, w * t + b01 - expit(t), rtol=1e-11, atol=1e-14)


def test_logistic_objective_vs_logaddexp():
    p = gen.logistic_problem(100, 12, seed=15)
    x = np.random.default_rng(15).standard_normal(12)
    t = p.A @ x
    b01 = 0.5 * (1 + p.b)
    ref = np.sum(np.logaddexp(0.0, -p.b * t)) + p.gamma * np.abs(x).sum()
    assert o.logistic_objective(p.A, p.b, p.gamma, x) == pytest.approx(ref, rel=1e-12)
    assert np.sum(np.logaddexp(0, t) - b01 * t) == pytest.approx(np.sum(np.logaddexp(0.0, -p.b * t)), rel=1e-12)


def _logistic_scipy(A, b_pm, gamma):
    """Reference minimiser of Eq. (9) by L-BFGS-B on the split x = xp - xm >= 0."""
    d = A.shape[1]
    b01 = 0.5 * (1 + b_pm)

    def f(v):
        x = v[:d] - v[d:]
        t = A @ x
        val = np.sum(np.logaddexp(0, t) - b01 * t) + gamma * v.sum()
        g = A.T @ (expit(t) - b01)
        return val, np.concatenate([g + gamma, -g + gamma])
    res = sopt.minimize(f, np.zeros(2 * d), jac=True, method="L-BFGS-B",
                        bounds=[(0, None)] * (2 * d), options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    return res.x[:d] - res.x[d:]


def check_logistic_vs_scipy(seed=16):
    p = gen.logistic_problem(400, 8, decay=0.5, nnz=3, xstd=2.0, seed=seed)
    gamma = 0.05 * np.max(np.abs(p.A.T @ (0.5 - 0.5 * (1 + p.b))))
    Om = gen.gaussian_test_matrix(8, 8, seed)
    out = o.logistic_nysadmm(p.A, p.b, gamma, 1.0, Om, 300, s0=2, s_max=8, ada_tol=1.5,
                             pcg_tol=1e-12)
    ref = _logistic_scipy(p.A, p.b, gamma)
    F = o.logistic_objective(p.A, p.b, gamma, out["z"])
    Fref = o.logistic_objective(p.A, p.b, gamma, ref)
    assert F <= Fref + 1e-9 * abs(Fref)
    assert np.linalg.norm(out["z"] - ref) <= 1e-4 * max(1, np.linalg.norm(ref))
    # KKT of Eq. (9): |A^T(sigma(Ax) - b01)|_j <= gamma, equality with sign on the support
    b01 = 0.5 * (1 + p.b)
    g = p.A.T @ (expit(p.A @ out["z"]) - b01)
    assert np.all(np.abs(g) <= gamma * (1 + 1e-6))
    S = np.abs(out["z"]) > 1e-8
    assert np.allclose(g[S], -gamma * np.sign(out["z"][S]), rtol=1e-6, atol=1e-8)


def test_logistic_matches_lbfgsb_and_kkt():
    check_logistic_vs_scipy()


def test_logistic_zero_threshold():
    p = gen.logistic_problem(200, 10, seed=17)
    b01 = 0.5 * (1 + p.b)
    gmax = np.max(np.abs(p.A.T @ (0.5 - b01)))
    Om = gen.gaussian_test_matrix(10, 10, 17)
    out = o.logistic_nysadmm(p.A, p.b, 1.0001 * gmax, 1.0, Om, 50, s0=2, s_max=4)
    assert np.max(np.abs(out["z"])) == 0.0


# ---------------------------------------------------------------- adaptive rank

def test_adaptive_rank_sequence_and_stop():
    A, H = _spd_decay(64, 18, decay=0.5)
    pool = gen.gaussian_test_matrix(64, 40, 18)
    # an unreachable tolerance walks 5 -> 10 -> 20 -> 40 (s_max)
    _, lam, _, ranks = o.adaptive_nystrom(lambda X: H @ X, pool, 5, 40, rho=1e-6, tol=1.0)
    assert ranks == [5, 10, 20, 40]
    # s_max not a power-of-two multiple: 5 -> 10 -> 20 -> 30
    _, _, _, ranks = o.adaptive_nystrom(lambda X: H @ X, pool[:, :30], 5, 30, rho=1e-6, tol=1.0)
    assert ranks == [5, 10, 20, 30]
    # a loose tolerance stops at the first rank
    _, lam, _, ranks = o.adaptive_nystrom(lambda X: H @ X, pool, 5, 40, rho=1e6, tol=2.0)
    assert ranks == [5]
    # the adaptive result equals the fixed-rank approximation of the concatenated blocks
    U, lam, nu, ranks = o.adaptive_nystrom(lambda X: H @ X, pool, 5, 40, rho=1e-6, tol=1.0)
    blocks = [o.thin_qr(pool[:, a:b]) for a, b in [(0, 5), (5, 10), (10, 20), (20, 40)]]
    Om = np.hstack(blocks)
    Hdef = o.nystrom_definition(H, Om)
    assert np.linalg.norm((U * lam) @ U.T - Hdef, 2) <= 1e-9 * np.linalg.norm(H, 2)


# ---------------------------------------------------------------- MLP (learned warm start)

def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(60)
    ni, nh, no = 7, 9, 5
    theta = rng.standard_normal(o.mlp_param_count(ni, nh, no)) * 0.4
    X = rng.standard_normal((6, ni))
    T = rng.standard_normal((6, no))
    _, g = o.mlp_loss_grad(theta, X, T, ni, nh, no)
    h = 1e-6
    for idx in rng.choice(theta.size, 40, replace=False):
        e = np.zeros_like(theta)
        e[idx] = h
        lp, _ = o.mlp_loss_grad(theta + e, X, T, ni, nh, no)
        lm, _ = o.mlp_loss_grad(theta - e, X, T, ni, nh, no)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_gelu_values_and_derivative():
    from scipy.stats import norm
    z = np.linspace(-4, 4, 41)
    assert np.allclose(o.gelu(z), z * norm.cdf(z), rtol=1e-14, atol=1e-15)
    h = 1e-6
    assert np.allclose(o.gelu_grad(z), (o.gelu(z + h) - o.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = o.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(th, -0.01 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)


# ---------------------------------------------------------------- counter-based Gaussian test matrix

def _kat_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        ctr, key, out = (part.split() for part in line.split("|"))
        rows.append(([int(v, 16) for v in ctr], [int(v, 16) for v in key], [int(v, 16) for v in out]))
    return rows


def test_philox_known_answer_vectors():
    """Philox-4x32-10 against the generator's published known-answer vectors."""
    rows = _kat_rows()
    assert len(rows) == 3
    ctr = np.array([r[0] for r in rows], dtype=np.uint64)
    key = np.array([r[1] for r in rows], dtype=np.uint64)
    out = o.philox4x32_10(ctr, key)
    assert out.tolist() == [r[2] for r in rows]


def test_philox_gaussian_moments_and_layout():
    """N(0,1) moments of 2 x 10^6 draws (mean, variance, skewness, excess kurtosis within
    ~5 standard errors; Kolmogorov-Smirnov against the normal CDF), determinism, seeds,
    and the column-major element numbering (a d x s draw is the first d s values of a
    (d s) x 1 draw)."""
    from scipy import stats
    G = o.gaussian_test_matrix_philox(7, 2000, 1000)
    g = G.ravel()
    n = g.size
    assert abs(g.mean()) <= 5 / np.sqrt(n)
    assert abs(g.var() - 1.0) <= 5 * np.sqrt(2.0 / n)
    assert abs(stats.skew(g)) <= 5 * np.sqrt(6.0 / n)
    assert abs(stats.kurtosis(g)) <= 5 * np.sqrt(24.0 / n)
    assert stats.kstest(g[:200000], "norm").pvalue > 1e-3
    assert np.array_equal(G, o.gaussian_test_matrix_philox(7, 2000, 1000))
    assert not np.array_equal(G[:, 0], o.gaussian_test_matrix_philox(8, 2000, 1)[:, 0])
    H = o.gaussian_test_matrix_philox(7, 2000 * 1000, 1)
    assert np.array_equal(G.ravel(order="F"), H[:, 0])
    # odd element count: the last pair contributes its even member only
    K = o.gaussian_test_matrix_philox(7, 7, 3)
    assert np.array_equal(K.ravel(order="F"), H[:21, 0])
