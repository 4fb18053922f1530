"""The test matrix drawn in the library (Omega == NULL): Philox-4x32-10 + Box-Muller on the
device against the oracle's implementation of the same published generator (pinned by
the generator's known-answer vectors), and solves that draw Omega themselves against
solves given the same panel.

Tolerance of the draw: the 32-bit words and the 53-bit uniforms are integers and agree
exactly; the Gaussians go through log, sqrt and sin/cos of the two math libraries, which
differ by a few units in the last place: 1e-13 absolute (|g| < 9)."""
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


@pytest.mark.parametrize("seed,d,s", [(0, 999, 37), (2**40 + 12345, 500, 1), (7, 2000, 1000)])
def test_device_draw_matches_oracle_generator(seed, d, s):
    Om = nx.gaussian_test_matrix(seed, d, s).cpu().numpy()
    ref = o.gaussian_test_matrix_philox(seed, d, s)
    assert Om.shape == (d, s)
    assert np.max(np.abs(Om - ref)) <= 1e-13
    assert torch.equal(nx.gaussian_test_matrix(seed, d, s), nx.gaussian_test_matrix(seed, d, s))


def test_sketch_and_solve_draw_omega_in_library():
    p = gen.lasso_problem(900, 150, nnz=10, seed=61)
    M = nx.Matrix.padded(torch.from_numpy(p.A).cuda())
    b = torch.from_numpy(p.b).cuda()
    Om = nx.gaussian_test_matrix(99, 150, 20)
    P1 = nx.sketch(M, None, s=20, seed=99)
    P2 = nx.sketch(M, Om)
    assert torch.equal(P1.lam, P2.lam)
    # against the oracle on the oracle's own draw of the same generator
    U, lam, _, _, _ = o.nystrom(lambda X: p.A.T @ (p.A @ X), o.gaussian_test_matrix_philox(99, 150, 20),
                                shift_scale=np.sqrt(150))
    assert np.max(np.abs(P1.lam.numpy() - lam)) <= 1e-10 * lam[0]
    a = nx.nysadmm_solve("lasso", M, b, p.gamma, 10.0, 20, 1e-10, None, admm_iters=30, seed=99)
    c = nx.nysadmm_solve("lasso", M, b, p.gamma, 10.0, 20, 1e-10, Om, admm_iters=30)
    assert torch.equal(a["z"], c["z"])
    d = nx.nysadmm_solve("lasso", M, b, p.gamma, 10.0, 20, 1e-10, None, admm_iters=30, seed=100)
    assert not torch.equal(a["x"], d["x"])
