"""Row-sharded solves through the C ABI: two processes share the one GPU, each holding a
contiguous block of rows (row_block), and complete every row sum -- the sketch's
A^T D A Omega, A^T b, each PCG matvec, the refined step's residual -- with a host-staged
gloo all-reduce (nys_opts.allreduce).  No kernel of one process waits on the other: the
reductions go through the host between launches.  Against the FP64 oracle on the unsharded
matrix: the sketch's eigenvalues (1e-10 of lam_1), pcg_solve (1e-10) and the lasso
trajectory with replayed PCG counts (x at 1e-10).  The mixed BF16 form with the FP64
correction against the unsharded GPU solve of the same form (FP32 PCG: the two differ only
in the order of the row sums, 1e-5).  The ranks' replicated iterates must agree bit for
bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import nys_inputs as gen
import oracle.nysadmm_oracle as o

pytestmark = pytest.mark.gpu


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    p = gen.lasso_problem(2003, 300, nnz=20, gamma_frac=0.1, seed=91)
    Om = gen.gaussian_test_matrix(300, 30, 91)
    return p, Om


def _worker(rank, world, port, fixed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_2202_11599_gb300 import nysadmm as nx
        ar = nx.host_staged_allreduce(dist)
        p, Om = _problem()
        r0, r1 = nx.row_block(p.A.shape[0], world, rank)
        Ag = torch.from_numpy(np.ascontiguousarray(p.A[r0:r1])).cuda()
        bg = torch.from_numpy(np.ascontiguousarray(p.b[r0:r1])).cuda()
        M = nx.Matrix.padded(Ag)
        Omd = torch.from_numpy(Om).cuda()
        P = nx.sketch(M, Omd, allreduce=ar)
        q = torch.from_numpy(p.A.T @ p.b).cuda()
        xs, it, _ = nx.pcg_solve(M, q, 2.0, P, tol=1e-12, allreduce=ar)
        sol = nx.nysadmm_solve("lasso", M, bg, p.gamma, 10.0, 30, 1e-10, Omd, admm_iters=60, pcg_fixed=fixed,
                               allreduce=ar)
        Mi = nx.Matrix.padded(Ag, torch.bfloat16)
        mixed = nx.nysadmm_solve("lasso", M, bg, p.gamma, 10.0, 30, 1e-6, Omd, admm_iters=400, A_inner=Mi,
                                 refine=True, allreduce=ar)
        torch.cuda.synchronize()
        out[rank] = (P.lam.numpy(), xs.cpu().numpy(), it, sol["x"].cpu().numpy(), sol["info"]["pcg_iters_total"],
                     mixed["z"].cpu().numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_row_sharded_solves_two_processes_one_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    p, Om = _problem()
    ref = o.lasso_nysadmm(p.A, p.b, p.gamma, 10.0, Om, 60, pcg_tol=1e-10)
    fixed = [int(v) for v in ref["trace"]["pcg_iters"]]
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, fixed, out), nprocs=world, join=True)
    H = lambda X: p.A.T @ (p.A @ X)
    U, lam, _, _, _ = o.nystrom(H, Om, shift_scale=np.sqrt(300))
    xs_ref, _, _ = o.pcg(H, 2.0, U, lam, p.A.T @ p.b, np.zeros(300), 1e-12)
    from paper_2202_11599_gb300 import nysadmm as nx
    Md = nx.Matrix.padded(torch.from_numpy(p.A).cuda())
    zmix_ref = nx.nysadmm_solve("lasso", Md, torch.from_numpy(p.b).cuda(), p.gamma, 10.0, 30, 1e-6,
                                torch.from_numpy(Om).cuda(), admm_iters=400,
                                A_inner=nx.Matrix.padded(torch.from_numpy(p.A).cuda(), torch.bfloat16),
                                refine=True, device_loop=False)["z"].cpu().numpy()
    for r in range(world):
        lam_g, xs, it, x, pcg_total, zmix = out[r]
        assert np.max(np.abs(lam_g - lam)) <= 1e-10 * lam[0]
        assert np.linalg.norm(xs - xs_ref) <= 1e-10 * np.linalg.norm(xs_ref)
        assert np.linalg.norm(x - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])
        assert pcg_total == sum(fixed)
        assert np.linalg.norm(zmix - zmix_ref) <= 1e-5 * np.linalg.norm(zmix_ref)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
