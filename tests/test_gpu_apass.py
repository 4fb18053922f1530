"""GPU parity of the two fused A-pass kernels -- the classic step (every warp meets at two
block barriers per group of rows) and the warp-specialised pass (producer, dot, finisher
and update warps meeting only through per-stage mbarriers) -- against the FP64
definition y = A^T diag(D) A p + rho p (Table 1's T_mv) on the stored values.

NYS_APASS_WS selects the kernel when a pass is planned; both are run on wide and ragged
rows of every storage type, with and without D, and must be bitwise repeatable.  The
row modes other than the H-matvec (the residual of the objective, A^T b of the lasso
right-hand side, the logistic weights and gradient) are covered through nys_objective
and short solves on FP64 rows wide enough for the warp-specialised FP64 pass.
Tolerances as in test_gpu_parity.py: FP64 1e-12 of the |A|^T|A||p| scale, FP32 / BF16 /
FP8 2e-5 (an FP32 accumulation over a row of up to 10^4 terms)."""
import os

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


@pytest.fixture(params=["classic", "warp_specialised"])
def kernel(request, monkeypatch):
    monkeypatch.setenv("NYS_APASS_WS", "1" if request.param == "warp_specialised" else "0")
    return request.param


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [(torch.float64, 3000, 2049), (torch.float64, 700, 10001), (torch.float64, 1500, 4096),
         (torch.float32, 5000, 1025), (torch.float32, 2000, 3001), (torch.bfloat16, 4000, 2049),
         (torch.bfloat16, 3000, 9999), (torch.bfloat16, 151, 4000), (torch.float8_e4m3fn, 3000, 4113)]


@pytest.mark.parametrize("dtype,n,d", CASES)
def test_pass_matches_definition(kernel, dtype, n, d):
    rng = np.random.default_rng(n * 17 + d)
    A = rng.standard_normal((n, d)) * gen.column_scales(d, 0.5)[None, :]
    if dtype == torch.float8_e4m3fn:
        M = nx.Matrix.fp8(_dev(A))
    else:
        M = nx.Matrix.padded(_dev(A), dtype)
    Aq = M.dequantized().cpu().numpy()
    ct = M.compute_dtype
    pq = torch.from_numpy(rng.standard_normal(d)).to(ct).double().numpy()
    Dv = rng.random(n) + 0.1
    for D in (None, Dv):
        Dd = None if D is None else _dev(D)
        y = nx.hmatvec(M, _dev(pq), 0.37, Dd)
        assert torch.equal(y, nx.hmatvec(M, _dev(pq), 0.37, Dd))
        w = np.ones(n) if D is None else D
        ref = Aq.T @ (w * (Aq @ pq)) + 0.37 * pq
        scale = np.abs(Aq).T @ (w * (np.abs(Aq) @ np.abs(pq))) + 0.37 * np.abs(pq)
        tol = 1e-12 if dtype == torch.float64 else 2e-5
        assert np.max(np.abs(y.double().cpu().numpy() - ref) / scale) <= tol


def test_kernels_agree_on_the_headline_shape_sampled(monkeypatch):
    """A 30,000 x 10,000 BF16 pass (the row width of the benchmark) through both kernels:
    the two differ only in the order of FP32 sums."""
    rng = np.random.default_rng(3)
    A = torch.randn(30000, 10000, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    M = nx.Matrix.padded(A, torch.bfloat16)
    p = torch.from_numpy(rng.standard_normal(10000)).float().cuda()
    out = {}
    for ws in ("0", "1"):
        monkeypatch.setenv("NYS_APASS_WS", ws)
        out[ws] = nx.hmatvec(M, p, 0.5).double()
    Aq = M.tensor[:, :10000].double()
    scale = Aq.abs().T @ (Aq.abs() @ p.double().abs())
    assert ((out["0"] - out["1"]).abs() / scale).max().item() <= 2e-5


def test_objective_and_rhs_modes_on_wide_fp64_rows(kernel):
    """Residual mode (objective, KKT and gap of Eq. 2 / Eq. 31) and A^T b (the lasso's
    right-hand side, through a 3-iteration solve with replayed PCG counts) on d = 2,049."""
    p = gen.lasso_problem(3000, 2049, nnz=40, gamma_frac=0.1, seed=51)
    M = nx.Matrix.padded(_dev(p.A))
    x = np.random.default_rng(51).standard_normal(2049) * (np.random.default_rng(52).random(2049) < 0.05)
    F, eta, gap = nx.objective("lasso", M, _dev(p.b), p.gamma, _dev(x))
    assert F == pytest.approx(o.lasso_objective(p.A, p.b, p.gamma, x), rel=1e-12)
    assert eta == pytest.approx(o.lasso_kkt_eta(p.A, p.b, p.gamma, x), rel=1e-9)
    assert gap == pytest.approx(o.lasso_dual_gap(p.A, p.b, p.gamma, x), rel=1e-9)
    Om = gen.gaussian_test_matrix(2049, 20, 51)
    ref = o.lasso_nysadmm(p.A, p.b, p.gamma, 10.0, Om, 3, pcg_tol=1e-10)
    out = nx.nysadmm_solve("lasso", M, _dev(p.b), p.gamma, 10.0, 20, 1e-10, _dev(Om), admm_iters=3,
                           pcg_fixed=ref["trace"]["pcg_iters"])
    xg = out["x"].cpu().numpy()
    assert np.linalg.norm(xg - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])


def test_logistic_modes_on_wide_fp64_rows(kernel):
    """The logistic weights / right-hand side (Sec. 3.2) and the gradient of Eq. 9 on d = 2,049."""
    p = gen.logistic_problem(2500, 2049, decay=0.5, nnz=20, seed=53)
    gamma = 0.05 * np.max(np.abs(p.A.T @ (0.5 - 0.5 * (1 + p.b))))
    pool = gen.gaussian_test_matrix(2049, 20, 53)
    ref = o.logistic_nysadmm(p.A, p.b, gamma, 1.0, pool, 4, s0=20, s_max=20, pcg_tol=1e-10)
    M = nx.Matrix.padded(_dev(p.A))
    out = nx.nysadmm_solve("logistic", M, _dev(p.b), gamma, 1.0, 20, 1e-10, _dev(pool), admm_iters=4,
                           pcg_fixed=ref["trace"]["pcg_iters"], rank_max=20, resketch_every=1)
    x = out["x"].cpu().numpy()
    assert np.linalg.norm(x - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"])
    F, g, _ = nx.objective("logistic", M, _dev(p.b), gamma, out["z"])
    assert F == pytest.approx(o.logistic_objective(p.A, p.b, gamma, out["z"].cpu().numpy()), rel=1e-12)
