"""The device-side ADMM loop's fused kernel for iterations whose x-step needs no PCG
iteration (one cooperative launch with two grid barriers per such iteration, Sec. 5's
decaying tolerance makes them the common case late in a solve) against the general graph
body (NYS_ADMM_NOSTEP=0): same arithmetic in the same order, so the iterates, the z trace,
the PCG counts and the residual stop must agree bit for bit."""
import numpy as np
import pytest
import torch

import nys_inputs as gen

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


def _solve(monkeypatch, fused, M, Mi, p, Om, **kw):
    monkeypatch.setenv("NYS_ADMM_NOSTEP", "1" if fused else "0")
    return nx.nysadmm_solve("lasso", M, torch.from_numpy(p.b).cuda(), p.gamma, kw.pop("rho"), Om.shape[1],
                            kw.pop("tol"), Om, A_inner=Mi, refine=False, z_trace=True, **kw)


@pytest.mark.parametrize("dtype", [torch.float64, torch.bfloat16])
@pytest.mark.parametrize("mode,tol,refresh", [("rnorm_pow", 1.5, 7), ("rnorm_pow", 1.75, 100), ("rel", 1e-3, 5)])
def test_nostep_kernel_is_bitwise_the_general_body(monkeypatch, dtype, mode, tol, refresh):
    p = gen.lasso_problem(3000, 700, nnz=30, gamma_frac=0.05, seed=71)
    M = nx.Matrix.padded(torch.from_numpy(p.A).cuda())
    Mi = None if dtype == torch.float64 else nx.Matrix.padded(torch.from_numpy(p.A).cuda(), dtype)
    Om = torch.from_numpy(gen.gaussian_test_matrix(700, 40, 71)).cuda()
    out = {}
    for fused in (True, False):
        out[fused] = _solve(monkeypatch, fused, M, Mi, p, Om, rho=20.0, tol=tol, admm_iters=300, tol_mode=mode,
                            hx_refresh=refresh)
    a, b = out[True], out[False]
    za, zb = a["z_trace"], b["z_trace"]
    first = next((k for k in range(za.shape[0]) if not torch.equal(za[k], zb[k])), None)
    assert first is None, (f"z traces first differ at iteration {first} of {za.shape[0]}; PCG totals "
                           f"{a['info']['pcg_iters_total']} / {b['info']['pcg_iters_total']}")
    assert torch.equal(a["x"], b["x"]) and torch.equal(a["z"], b["z"])
    assert a["info"]["pcg_iters_total"] == b["info"]["pcg_iters_total"]
    assert a["info"]["r_p"] == b["info"]["r_p"] and a["info"]["r_d"] == b["info"]["r_d"]
    # the fused kernel had work: iterations without a PCG step
    assert a["info"]["pcg_iters_total"] < a["info"]["admm_iters"]


def test_nostep_kernel_residual_stop_and_fixed_counts(monkeypatch):
    """The residual stop of Sec. 2.1 taken inside the fused kernel, and replayed PCG counts
    with zeros (the fused kernel runs exactly the iterations whose count is 0)."""
    p = gen.lasso_problem(2000, 500, nnz=20, gamma_frac=0.1, seed=72)
    M = nx.Matrix.padded(torch.from_numpy(p.A).cuda())
    Om = torch.from_numpy(gen.gaussian_test_matrix(500, 30, 72)).cuda()
    res = {}
    for fused in (True, False):
        res[fused] = _solve(monkeypatch, fused, M, None, p, Om, rho=10.0, tol=1.5, admm_iters=2000,
                            tol_mode="rnorm_pow", hx_refresh=50, eps_abs=0.0, eps_rel=1e-5)
    assert res[True]["info"]["admm_iters"] == res[False]["info"]["admm_iters"] < 2000
    assert torch.equal(res[True]["z"], res[False]["z"])
    fixed = [0 if k % 3 else 2 for k in range(60)]
    fx = {}
    for fused in (True, False):
        fx[fused] = _solve(monkeypatch, fused, M, None, p, Om, rho=10.0, tol=1e-10, admm_iters=60,
                           pcg_fixed=fixed, hx_refresh=4)
    assert torch.equal(fx[True]["z_trace"], fx[False]["z_trace"])
    assert fx[True]["info"]["pcg_iters_total"] == sum(fixed)


@pytest.mark.parametrize("dtype", [torch.float64, torch.bfloat16])
@pytest.mark.parametrize("mode,tol,refresh,nostep", [("rel", 1e-3, 5, "1"), ("rnorm_pow", 1.5, 7, "1"),
                                                     ("rel", 1e-3, 5, "0"), ("rnorm_pow", 1.75, 100, "0")])
def test_post_kernel_is_bitwise_the_separate_kernels(monkeypatch, dtype, mode, tol, refresh, nostep):
    """One PCG iteration's reduce, update, scalar step, P^{-1} apply and direction update as
    one cooperative launch (and, in the fast body, the prox / dual step with it) against the
    four separate kernels (NYS_PCG_POST=0), in both graph bodies."""
    p = gen.lasso_problem(3000, 700, nnz=30, gamma_frac=0.05, seed=73)
    M = nx.Matrix.padded(torch.from_numpy(p.A).cuda())
    Mi = None if dtype == torch.float64 else nx.Matrix.padded(torch.from_numpy(p.A).cuda(), dtype)
    Om = torch.from_numpy(gen.gaussian_test_matrix(700, 40, 73)).cuda()
    monkeypatch.setenv("NYS_ADMM_NOSTEP", nostep)
    out = {}
    for post in ("1", "0"):
        monkeypatch.setenv("NYS_PCG_POST", post)
        out[post] = nx.nysadmm_solve("lasso", M, torch.from_numpy(p.b).cuda(), p.gamma, 20.0, 40, tol, Om, A_inner=Mi,
                                     refine=False, z_trace=True, admm_iters=200, tol_mode=mode, hx_refresh=refresh,
                                     pcg_trace=True)
    a, b = out["1"], out["0"]
    assert a["pcg_trace"] == b["pcg_trace"] and a["info"]["pcg_iters_total"] > 50
    assert torch.equal(a["z_trace"], b["z_trace"]) and torch.equal(a["x"], b["x"])
    assert a["info"]["r_p"] == b["info"]["r_p"] and a["info"]["r_d"] == b["info"]["r_d"]
