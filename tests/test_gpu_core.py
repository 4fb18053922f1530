"""The FP64 Nystrom core's eigensolve (App. B: the thin SVD of B through eig(B^T B)) in its
two launch forms -- one cooperative grid with barriers between rounds, one launch per
round -- runs the same rotations in the same order, so lam and U must agree bit for bit;
and the core against the oracle on even and odd ranks, tile-aligned and ragged."""
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


FORMS = {"grid": {}, "rounds": {"NYS_JACOBI_PERSISTENT": "0"}}


@pytest.mark.parametrize("n,d,s", [(3000, 700, 200), (1500, 400, 33), (2000, 600, 96), (1200, 900, 300)])
def test_jacobi_forms_bitwise_and_oracle(monkeypatch, n, d, s):
    A = gen.lasso_problem(n, d, nnz=10, seed=s).A
    Om = gen.gaussian_test_matrix(d, s, s)
    M = nx.Matrix.padded(torch.from_numpy(A).cuda())
    out = {}
    for name, env in FORMS.items():
        monkeypatch.delenv("NYS_JACOBI_PERSISTENT", raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        P = nx.sketch(M, torch.from_numpy(Om).cuda())
        out[name] = (P.lam, P.U.cpu())
    assert torch.equal(out["rounds"][0], out["grid"][0])
    assert torch.equal(out["rounds"][1], out["grid"][1])
    U, lam, _, _, _ = o.nystrom(lambda X: A.T @ (A @ X), Om, shift_scale=np.sqrt(d))
    lg = out["grid"][0].numpy()
    assert np.max(np.abs(lg - lam)) <= 1e-10 * lam[0]
    Ug = out["grid"][1].numpy()
    top = lam > 1e-8 * lam[0]
    Ag = (Ug[:, top] * lg[top]) @ Ug[:, top].T
    Ao = (U[:, top] * lam[top]) @ U[:, top].T
    assert np.max(np.abs(Ag - Ao)) <= 1e-10 * lam[0]
