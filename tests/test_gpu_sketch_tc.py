"""The tensor-core sketch (App. B: Y = A^T D A Omega) in its two staging forms -- TMA tiled
copies (the default) and cp.async -- issues the same MMAs in the same order, so Lam and U
agree bit for bit; both agree with the oracle on the stored matrix.  Ragged rows, a K tail,
N padding, two column panels (s > 256), row weights D, BF16 and FP32 storage."""
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


def _quantised(A, dtype):
    return torch.from_numpy(A).to(dtype).to(torch.float64).numpy()


@pytest.mark.parametrize("n,d,s,dtype,weighted", [
    (3001, 517, 37, torch.bfloat16, False),
    (2500, 600, 260, torch.bfloat16, True),
    (130, 40, 3, torch.bfloat16, False),
    (1000, 256, 64, torch.float32, True),
    (777, 333, 17, torch.float32, False),
])
def test_tma_and_cp_async_staging_bitwise(monkeypatch, n, d, s, dtype, weighted):
    rng = np.random.default_rng(n + s)
    A = rng.standard_normal((n, d)) * gen.column_scales(d, 1.0)[None, :]
    Om = gen.gaussian_test_matrix(d, s, n)
    D = rng.random(n) + 0.1 if weighted else None
    M = nx.Matrix.padded(torch.from_numpy(A).cuda(), dtype)
    out = {}
    for form, env in (("tma", "1"), ("cp", "0")):
        monkeypatch.setenv("NYS_TC_TMA", env)
        P = nx.sketch(M, torch.from_numpy(Om).cuda(), D=None if D is None else torch.from_numpy(D).cuda())
        out[form] = (P.lam.clone(), P.U.cpu().clone())
    assert torch.equal(out["tma"][0], out["cp"][0])
    assert torch.equal(out["tma"][1], out["cp"][1])
    Aq = _quantised(A, dtype)
    w = np.ones(n) if D is None else D
    U, lam, _, _, _ = o.nystrom(lambda X: Aq.T @ (w[:, None] * (Aq @ X)), Om, shift_scale=np.sqrt(d),
                                mantissa_bits=23)
    assert np.max(np.abs(out["tma"][0].numpy() - lam)) <= 2e-5 * lam[0]
