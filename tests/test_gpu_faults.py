"""Fault handling through the C ABI, with faults made on the host (no GPU fault, trap or
hang): NaN / infinite data in b, in A, in the PCG right-hand side and in the row weights D
is rejected with NYS_EINVAL; a negative D makes p^T (H + rho I) p < 0 at the first PCG
iteration, reported as NYS_EBREAKDOWN (Alg. Nystrom PCG needs an SPD system); a test matrix
with dependent columns cannot be orthonormalised (NYS_EINVAL).  After every refused call
the same context solves a clean problem correctly."""
import numpy as np
import pytest
import torch

import nys_inputs as gen
import oracle.nysadmm_oracle as o

pytestmark = pytest.mark.gpu

nx = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global nx
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_11599_gb300 import nysadmm
    nx = nysadmm


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _clean_solve_is_right():
    p = gen.lasso_problem(600, 90, nnz=8, seed=22)
    Om = gen.gaussian_test_matrix(90, 15, 22)
    ref = o.lasso_nysadmm(p.A, p.b, p.gamma, 10.0, Om, 40, pcg_tol=1e-10)
    out = nx.nysadmm_solve("lasso", nx.Matrix.padded(_dev(p.A)), _dev(p.b), p.gamma, 10.0, 15, 1e-10, _dev(Om),
                           admm_iters=40, pcg_fixed=ref["trace"]["pcg_iters"])
    x = out["x"].cpu().numpy()
    assert np.linalg.norm(x - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])


def _status(fn):
    with pytest.raises(nx.NysError) as e:
        fn()
    return e.value.status


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("device_loop", [True, False])
def test_nonfinite_b_is_rejected(bad, device_loop):
    p = gen.lasso_problem(700, 120, nnz=8, seed=31)
    b = p.b.copy()
    b[17] = bad
    Om = gen.gaussian_test_matrix(120, 16, 31)
    st = _status(lambda: nx.nysadmm_solve("lasso", nx.Matrix.padded(_dev(p.A)), _dev(b), p.gamma, 3.0, 16, 1e-8,
                                          _dev(Om), admm_iters=20, device_loop=device_loop))
    assert st == nx.NYS_EINVAL
    _clean_solve_is_right()


@pytest.mark.parametrize("dtype", [torch.float64, torch.bfloat16])
def test_nonfinite_A_is_rejected(dtype):
    p = gen.lasso_problem(700, 120, nnz=8, seed=32)
    A = p.A.copy()
    A[5, 7] = np.nan
    Om = gen.gaussian_test_matrix(120, 16, 32)
    M = nx.Matrix.padded(_dev(A), dtype)
    assert _status(lambda: nx.sketch(M, _dev(Om))) == nx.NYS_EINVAL
    assert _status(lambda: nx.nysadmm_solve("lasso", nx.Matrix.padded(_dev(A)), _dev(p.b), p.gamma, 3.0, 16, 1e-8,
                                            _dev(Om), admm_iters=10)) == nx.NYS_EINVAL
    _clean_solve_is_right()


def test_nonfinite_pcg_rhs_and_weights_are_rejected():
    p = gen.lasso_problem(500, 80, nnz=6, seed=33)
    M = nx.Matrix.padded(_dev(p.A))
    r = p.A.T @ p.b
    r[3] = np.nan
    assert _status(lambda: nx.pcg_solve(M, _dev(r), 1.0, None, tol=1e-10)) == nx.NYS_EINVAL
    D = np.ones(500)
    D[11] = np.inf
    Om = gen.gaussian_test_matrix(80, 10, 33)
    assert _status(lambda: nx.sketch(M, _dev(Om), D=_dev(D))) == nx.NYS_EINVAL
    _clean_solve_is_right()


def test_negative_weights_break_down_pcg():
    """H = A^T diag(D) A with D = -1 is negative definite: with rho small, p^T (H + rho I) p < 0
    at the first PCG iteration (Alg. Nystrom PCG assumes H + rho I SPD)."""
    p = gen.lasso_problem(500, 80, nnz=6, seed=34)
    M = nx.Matrix.padded(_dev(p.A))
    D = -np.ones(500)
    r = p.A.T @ p.b
    st = _status(lambda: nx.pcg_solve(M, _dev(r), 1e-3, None, tol=1e-10, D=_dev(D)))
    assert st == nx.NYS_EBREAKDOWN
    _clean_solve_is_right()


def test_dependent_test_matrix_columns_are_rejected():
    p = gen.lasso_problem(500, 80, nnz=6, seed=35)
    Om = gen.gaussian_test_matrix(80, 10, 35)
    Om[:, 4] = Om[:, 2]
    assert _status(lambda: nx.sketch(nx.Matrix.padded(_dev(p.A)), _dev(Om))) == nx.NYS_EINVAL
    _clean_solve_is_right()
