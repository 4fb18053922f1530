"""Planted mistakes in the oracle (on the CPU) must each fail a pin.

Each mutant replaces one oracle function by a plausible wrong variant (a
dropped term, a wrong sign, a transposed operand, an off-by-one index) and
runs the pins of tests/test_oracle_pins.py that should catch it."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle.nysadmm_oracle as o
import tests.test_oracle_pins as pins

_orig_precond = o.precond_apply
_orig_sketch = o.nystrom_from_sketch
_orig_pcg = o.pcg
_orig_soft = o.soft_threshold
_orig_lasso = o.lasso_nysadmm


def _precond_drop_scale(U, lam, rho, v):          # (lam_s + rho) factor dropped
    Utv = U.T @ v
    return U @ (Utv / (lam + rho)) + v - U @ Utv


def _precond_wrong_index(U, lam, rho, v):         # lam_1 instead of lam_s
    Utv = U.T @ v
    return (lam[0] + rho) * (U @ (Utv / (lam + rho))) + v - U @ Utv


def _sketch_no_inverse(Y, Omega, shift_scale=1.0, mantissa_bits=52, max_retries=3):
    # B = Y_nu C instead of Y_nu C^{-1}
    sigma = np.linalg.norm(Y, 2)
    nu = shift_scale * o.eps_of(sigma, mantissa_bits)
    Ynu = Y + nu * Omega
    M = Omega.T @ Ynu
    C = np.linalg.cholesky(0.5 * (M + M.T)).T
    U, S, _ = np.linalg.svd(Ynu @ C, full_matrices=False)
    return U, np.maximum(0, S * S - nu), nu


def _sketch_lower_factor(Y, Omega, shift_scale=1.0, mantissa_bits=52, max_retries=3):
    # transposed factor: B = Y_nu L^{-1} with L lower
    sigma = np.linalg.norm(Y, 2)
    nu = shift_scale * o.eps_of(sigma, mantissa_bits)
    Ynu = Y + nu * Omega
    M = Omega.T @ Ynu
    L = np.linalg.cholesky(0.5 * (M + M.T))
    B = sla.solve_triangular(L, Ynu.T, trans="T", lower=True).T
    U, S, _ = np.linalg.svd(B, full_matrices=False)
    return U, np.maximum(0, S * S - nu), nu


def _sketch_keep_shift(Y, Omega, shift_scale=1.0, mantissa_bits=52, max_retries=3):
    # shift not removed, and a visible one (nu = 1e-3 ||Y||)
    nu = 1e-3 * np.linalg.norm(Y, 2)
    Ynu = Y + nu * Omega
    M = Omega.T @ Ynu
    C = np.linalg.cholesky(0.5 * (M + M.T)).T
    B = sla.solve_triangular(C, Ynu.T, trans="T", lower=False).T
    U, S, _ = np.linalg.svd(B, full_matrices=False)
    return U, S * S, nu


def _pcg_wrong_beta(H_apply, rho, U, lam, r, x0, tol, tol_mode="rel", maxit=None, fixed_iters=None):
    # beta = (w_new . y_new) / (p . v) (wrong denominator)
    Pinv = (lambda v: v.copy()) if U is None else (lambda v: _orig_precond(U, lam, rho, v))
    x = x0.copy(); w = r - (H_apply(x) + rho * x); y = Pinv(w); p = y.copy(); it = 0
    thresh = tol * np.linalg.norm(r) if tol_mode == "rel" else tol
    while (it < fixed_iters) if fixed_iters is not None else (np.linalg.norm(w) > thresh and it < 1000):
        v = H_apply(p) + rho * p
        alpha = (w @ y) / (p @ v)
        x = x + alpha * p
        w = w - alpha * v
        y_new = Pinv(w)
        beta = (w @ y_new) / (p @ v)
        p = y_new + beta * p
        y = y_new
        it += 1
    return x, it, float(np.linalg.norm(w))


def _pcg_no_rho(H_apply, rho, U, lam, r, x0, tol, tol_mode="rel", maxit=None, fixed_iters=None):
    # the rho I term dropped from the system matrix (solves H x = r)
    return _orig_pcg(lambda v: H_apply(v) - rho * v, rho, U, lam, r, x0, tol, tol_mode, maxit,
                     fixed_iters)


def _enet_no_hessian_of_g(A, b, gamma, rho, Omega, admm_iters, **kw):
    # H^g = (1 - gamma) I dropped from the subproblem and the sketch
    return _orig_lasso(A, b, gamma, rho, Omega, admm_iters, **kw)


def _enet_swapped_weights(A, b, gamma, rho, Omega, admm_iters, **kw):
    # l2 weight gamma and l1 weight 1 - gamma
    return _orig_lasso(A, b, 1.0 - gamma, rho, Omega, admm_iters, mu=gamma, **kw)


def _mixed_q_from_inner(A, b, gamma, rho, Omega, admm_iters, A_inner=None, **kw):
    # mixed form: A^T b taken from the low-precision copy instead of the problem matrix
    return _orig_lasso(A if A_inner is None else A_inner, b, gamma, rho, Omega, admm_iters,
                       A_inner=A_inner, **kw)


def _mixed_inner_ignored(A, b, gamma, rho, Omega, admm_iters, A_inner=None, **kw):
    # mixed form: the low-precision copy dropped (H from the problem matrix)
    return _orig_lasso(A, b, gamma, rho, Omega, admm_iters, **kw)


def _soft_wrong_sign(v, kappa):
    return np.sign(v) * np.maximum(np.abs(v) + kappa, 0.0)


MUTANTS = [
    ("precond_apply", _precond_drop_scale, [pins.check_precond_inverse, pins.check_precond_exact]),
    ("precond_apply", _precond_wrong_index, [pins.check_precond_inverse]),
    ("nystrom_from_sketch", _sketch_no_inverse, [pins.check_nystrom_definition]),
    ("nystrom_from_sketch", _sketch_lower_factor, [pins.check_nystrom_definition]),
    ("nystrom_from_sketch", _sketch_keep_shift, [pins.check_nystrom_exact_low_rank]),
    ("pcg", _pcg_wrong_beta, [pins.check_pcg_iterates_match_scipy]),
    ("pcg", _pcg_no_rho, [pins.check_pcg_direct]),
    ("soft_threshold", _soft_wrong_sign, [pins.check_soft_threshold, pins.check_lasso_orthonormal]),
    ("elastic_net_nysadmm", _enet_no_hessian_of_g, [pins.check_elastic_net_orthonormal,
                                                    pins.check_elastic_net_augmented_brute_force,
                                                    pins.check_elastic_net_small_gamma_is_ridge]),
    ("elastic_net_nysadmm", _enet_swapped_weights, [pins.check_elastic_net_orthonormal,
                                                    pins.check_elastic_net_augmented_brute_force]),
    ("lasso_nysadmm", _mixed_q_from_inner, [pins.check_mixed_form_fixed_point]),
    ("lasso_nysadmm", _mixed_inner_ignored, [pins.check_mixed_form_fixed_point]),
]


@pytest.mark.parametrize("name,mutant,checks", MUTANTS,
                         ids=[f"{m[0]}:{m[1].__name__}" for m in MUTANTS])
def test_planted_mistake_is_caught(monkeypatch, name, mutant, checks):
    monkeypatch.setattr(o, name, mutant)
    for chk in checks:
        with pytest.raises((AssertionError, np.linalg.LinAlgError, o.BreakdownError,
                            FloatingPointError, ValueError)):
            chk()
