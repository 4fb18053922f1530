"""Learned warm start: the MLP kernels against the FP64 oracle, the zero-model
identity, and the measured gain on a family of lasso problems sharing A."""
import numpy as np
import pytest
import torch

import nys_inputs as gen
import oracle.nysadmm_oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_11599_gb300 import nysadmm
    return nysadmm


def _bf16(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _init(ni, nh, no, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for (fo, fi) in [(nh, ni), (nh, None), (nh, nh), (nh, None), (no, nh), (no, None)]:
        if fi is None:
            parts.append(rng.standard_normal(fo) * 0.1)
        else:
            parts.append(rng.uniform(-1, 1, (fo, fi)).ravel() * scale * np.sqrt(6.0 / (fi + fo)))
    return np.concatenate(parts).astype(np.float32)


def _theta_as_used(theta32, ni, nh, no):
    """The kernels multiply with BF16-rounded weights and biases."""
    return _bf16(theta32)


@pytest.mark.parametrize("ni,nh,no,B", [(13, 32, 10, 40), (103, 256, 100, 256), (5, 17, 3, 7)])
def test_mlp_forward_and_gradient_match_oracle(nx, ni, nh, no, B):
    th = _init(ni, nh, no, ni + nh)
    rng = np.random.default_rng(B)
    X = rng.standard_normal((B, ni)).astype(np.float32)
    T = rng.standard_normal((B, no)).astype(np.float32)
    m = nx.MLP(ni, nh, no, th)
    thu = _theta_as_used(th, ni, nh, no)
    Yref, _ = o.mlp_forward(thu, X.astype(np.float64), ni, nh, no)
    Y = m.forward(torch.from_numpy(X).cuda()).double().cpu().numpy()
    assert np.max(np.abs(Y - Yref)) <= 1e-4 * max(1.0, np.max(np.abs(Yref)))
    lref, gref = o.mlp_loss_grad(thu, X.astype(np.float64), T.astype(np.float64), ni, nh, no)
    loss, g = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    g = g.double().cpu().numpy()
    assert loss == pytest.approx(lref, rel=1e-4)
    assert np.max(np.abs(g - gref)) <= 2e-4 * np.max(np.abs(gref))


def test_mlp_adam_step_matches_oracle(nx):
    ni, nh, no, B = 9, 24, 6, 32
    th = _init(ni, nh, no, 3)
    rng = np.random.default_rng(4)
    X = torch.from_numpy(rng.standard_normal((B, ni)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.standard_normal((B, no)).astype(np.float32)).cuda()
    m = nx.MLP(ni, nh, no, th)
    _, g = m.grad(X, T)
    g = g.double().cpu().numpy()
    m.train_step(X, T, lr=1e-2)
    ref, _, _ = o.adam_step(th.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-2)
    got = m.params().double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-6 + 1e-5 * np.max(np.abs(ref))


def _family(n=2000, d=200, count=12, seed=70):
    """Lasso instances sharing A (decay (1+j)^-1), each with a fresh sparse x* and b."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) * gen.column_scales(d, 1.0)[None, :]
    out = []
    for i in range(count):
        x = gen.sparse_vector(rng, d, max(2, d // 100))
        b = A @ x + 1e-3 * rng.standard_normal(n)
        out.append((b, 0.05 * np.max(np.abs(A.T @ b))))
    return A, out


def test_warm_start_model_does_not_change_the_solution(nx):
    """A model that predicts zero coordinates restarts PCG from x_prev with its
    range(U) component removed; PCG runs to the same tolerance, so the ADMM iterates
    agree with the plain warm start up to that tolerance."""
    A, fam = _family(count=1)
    s = 20
    Om = gen.gaussian_test_matrix(A.shape[1], s, 71)
    M = nx.Matrix.padded(torch.from_numpy(A).cuda())
    b, gamma = fam[0]
    zero = nx.MLP(s + 3, 32, s, np.zeros(o.mlp_param_count(s + 3, 32, s), np.float32))
    kw = dict(admm_iters=40)
    a = nx.nysadmm_solve("lasso", M, torch.from_numpy(b).cuda(), gamma, 10.0, s, 1e-12,
                         torch.from_numpy(Om).cuda(), warm_model=zero, **kw)
    c = nx.nysadmm_solve("lasso", M, torch.from_numpy(b).cuda(), gamma, 10.0, s, 1e-12,
                         torch.from_numpy(Om).cuda(), **kw)
    za, zc = a["z"].cpu().numpy(), c["z"].cpu().numpy()
    assert np.linalg.norm(za - zc) <= 1e-8 * max(1.0, np.linalg.norm(zc))


def test_learned_warm_start_trains_on_nysadmm_pairs(nx):
    """Train on (features, target) pairs recorded by NysADMM on 8 instances, evaluate
    on 4 others: the solutions are those of the plain warm start (same PCG
    tolerance), and the PCG iteration counts of both starts are reported.  (Measured
    on GB300: the plain x_prev start needs fewer iterations at rel-tol 1e-10 -- once
    ADMM settles, x_prev is far more accurate than the learned coordinates.)"""
    A, fam = _family()
    s, K, tol, rho = 20, 40, 1e-10, 10.0
    Om = torch.from_numpy(gen.gaussian_test_matrix(A.shape[1], s, 72)).cuda()
    M = nx.Matrix.padded(torch.from_numpy(A).cuda())
    rows = []
    for b, gamma in fam[:8]:
        out = nx.nysadmm_solve("lasso", M, torch.from_numpy(b).cuda(), gamma, rho, s, tol, Om, admm_iters=K,
                               warm_record=True)
        rows.append(out["warm_record"])
    R = torch.cat(rows)
    X, T = R[:, : s + 3].contiguous(), R[:, s + 3:].contiguous()
    assert torch.isfinite(R).all() and T.abs().max() > 0
    model = nx.MLP(s + 3, 64, s, _init(s + 3, 64, s, 73, scale=0.5))
    first = model.train_step(X, T, lr=1e-3)
    for _ in range(1500):
        last = model.train_step(X, T, lr=1e-3)
    assert last < 0.1 * first
    base, learned = 0, 0
    for b, gamma in fam[8:]:
        bt = torch.from_numpy(b).cuda()
        p = nx.nysadmm_solve("lasso", M, bt, gamma, rho, s, tol, Om, admm_iters=K)
        q = nx.nysadmm_solve("lasso", M, bt, gamma, rho, s, tol, Om, admm_iters=K, warm_model=model)
        base += p["info"]["pcg_iters_total"]
        learned += q["info"]["pcg_iters_total"]
        zp, zq = p["z"].cpu().numpy(), q["z"].cpu().numpy()
        assert np.linalg.norm(zq - zp) <= 1e-7 * max(1.0, np.linalg.norm(zp))
    print(f"PCG iterations over 4 held-out instances: plain warm start {base}, learned {learned}")
