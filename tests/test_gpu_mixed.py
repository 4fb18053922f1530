"""GPU parity of the mixed precision form WITHOUT residual correction -- the form the
benchmark times -- against the oracle's A_inner form (the sketch and the x-subproblem
matrix built from the stored BF16 / FP32 values, A^T b from the FP64 matrix; the
perturbed problem 1/2 x^T Aq^T Aq x - (A^T b)^T x + gamma ||x||_1).

Tolerances (FP32 PCG vectors, FP32 accumulation in every matvec):
  * iterates: 1e-5 relative.  One FP32 H-matvec carries about sqrt(d) 2^-24 relative
    rounding (1.3e-6 at d = 500, 1.7e-6 at d = 777); PCG with the Nystrom
    preconditioner has an empirical condition number of a few, and ADMM is
    non-expansive, so the error stays at that level over the 100 iterations instead of
    accumulating; 1e-5 leaves a factor ~6 of margin.
  * the Nystrom operator U Lam U^T: 5e-5 of lam_1 (an FP32-class sketch of the stored
    matrix, 2^-24 times the sqrt(d)-scaled row sums, amplified by the core's
    (Omega^T Y)^{-1} on the trailing directions); P^{-1} v: 1e-5 of ||v||.
"""
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


def _stored(A, dtype):
    """The values the GPU stores for A in `dtype`, in FP64."""
    return torch.from_numpy(A).to(dtype).to(torch.float64).numpy()


def _case(name):
    """(problem, rho, rank): the 2,000 x 500 lasso of the small configuration (rho 1, rank 50)
    and a ragged 3,001 x 777 lasso (no dimension a multiple of a vector width or tile)."""
    if name == "2000x500":
        return gen.lasso_small(0), 1.0, 50
    return gen.lasso_problem(3001, 777, nnz=30, gamma_frac=0.1, seed=41), 5.0, 40


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("hx_refresh", [0, 7])
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("case", ["2000x500", "3001x777"])
def test_mixed_form_without_correction_replays_oracle(case, dtype, hx_refresh):
    """100 ADMM iterations; the oracle runs PCG to rel-tol 1e-8 on the stored values and
    the GPU replays its per-iteration PCG counts, so both follow one trajectory."""
    p, rho, s = _case(case)
    d = p.A.shape[1]
    Om = gen.gaussian_test_matrix(d, s, 0)
    Aq = _stored(p.A, dtype)
    ref = o.lasso_nysadmm(p.A, p.b, p.gamma, rho, Om, 100, pcg_tol=1e-8, A_inner=Aq, mantissa_bits=23)
    out = nx.nysadmm_solve("lasso", nx.Matrix.padded(_dev(p.A)), _dev(p.b), p.gamma, rho, s, 1e-8, _dev(Om),
                           admm_iters=100, A_inner=nx.Matrix.padded(_dev(p.A), dtype), refine=False,
                           pcg_fixed=ref["trace"]["pcg_iters"], hx_refresh=hx_refresh, z_trace=True)
    assert out["info"]["pcg_iters_total"] == sum(ref["trace"]["pcg_iters"])
    assert _rel(out["x"].cpu().numpy(), ref["x"]) <= 1e-5
    assert _rel(out["z"].cpu().numpy(), ref["z"]) <= 1e-5
    zt = out["z_trace"].cpu().numpy()
    for k in (0, 9, 49, 99):
        assert _rel(zt[k], ref["trace"]["z"][k]) <= 1e-5


@pytest.mark.parametrize("hx_refresh", [0, 7])
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_mixed_form_without_correction_schedule(dtype, hx_refresh):
    """The decaying PCG schedule ||w|| <= ||r^k|| / k^1.5 (Sec. 5) run by both sides on
    their own norms.  The GPU's FP32 residual differs from the oracle's by about
    2^-24 * k^1.5 * (condition number) of the threshold (< 1e-4 here); the test first
    checks on the oracle that every stop decision lies at least 1e-3 away from its
    threshold, then requires the same PCG counts and x within 1e-5."""
    p, rho, s = _case("2000x500")
    Om = gen.gaussian_test_matrix(500, s, 0)
    Aq = _stored(p.A, dtype)
    ref = o.lasso_nysadmm(p.A, p.b, p.gamma, rho, Om, 100, pcg_tol=1.5, pcg_tol_mode="rnorm_pow",
                          A_inner=Aq, mantissa_bits=23)
    # ADMM iteration 0 starts PCG at x = 0, so w = r and the threshold ||r|| / 1^beta equals
    # ||w||: both sides stop there without a step (the same vector on both sides)
    assert ref["trace"]["pcg_iters"][0] == 0
    for wn, th in list(zip(ref["trace"]["pcg_wnorms"], ref["trace"]["pcg_thresh"]))[1:]:
        assert wn[-1] <= th * (1 - 1e-3)
        if len(wn) > 1:
            assert wn[-2] >= th * (1 + 1e-3)
    out = nx.nysadmm_solve("lasso", nx.Matrix.padded(_dev(p.A)), _dev(p.b), p.gamma, rho, s, 1.5, _dev(Om),
                           admm_iters=100, A_inner=nx.Matrix.padded(_dev(p.A), dtype), refine=False,
                           tol_mode="rnorm_pow", hx_refresh=hx_refresh)
    assert out["info"]["pcg_iters_total"] == sum(ref["trace"]["pcg_iters"])
    assert _rel(out["x"].cpu().numpy(), ref["x"]) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("n,d,s", [(2000, 256, 24), (3001, 517, 37), (2500, 600, 260)])
def test_low_precision_sketch_operator_and_preconditioner(n, d, s, dtype):
    """The tensor-core sketch of the stored matrix: the approximation U Lam U^T itself
    (a wrong U with correct eigenvalues -- permuted or mixed columns -- fails here) and
    P^{-1} v in FP64 and in the FP32 form PCG uses, for rho below, at and above lam_s."""
    rng = np.random.default_rng(n + s)
    A = rng.standard_normal((n, d)) * gen.column_scales(d, 1.0)[None, :]
    Om = gen.gaussian_test_matrix(d, s, n + s)
    Aq = _stored(A, dtype)
    U, lam, _, _, _ = o.nystrom(lambda X: Aq.T @ (Aq @ X), Om, shift_scale=np.sqrt(d), mantissa_bits=23)
    P = nx.sketch(nx.Matrix.padded(_dev(A), dtype), _dev(Om))
    Ug = P.U.cpu().numpy()
    lg = P.lam.numpy()
    H_o = (U * lam) @ U.T
    H_g = (Ug * lg) @ Ug.T
    assert np.linalg.norm(H_g - H_o, 2) <= 5e-5 * lam[0]
    v = rng.standard_normal(d)
    for rho in (1e-2 * lam[0], lam[-1], 10 * lam[-1]):
        ref = o.precond_apply(U, lam, rho, v)
        y64 = P.apply(_dev(v), rho).cpu().numpy()
        y32 = P.apply(_dev(v).float(), rho).double().cpu().numpy()
        assert np.linalg.norm(y64 - ref) <= 1e-5 * np.linalg.norm(v)
        assert np.linalg.norm(y32 - ref) <= 1e-5 * np.linalg.norm(v)
