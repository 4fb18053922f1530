"""Row-sharded NysADMM on the CPU with two gloo ranks (world size 2).

The x-subproblem matrix is a sum over row blocks, A^T D A = sum_g A_g^T D_g A_g (Table 1's
T_mv), so a row-sharded solve needs one d x s reduction for the sketch and one d-vector
reduction per PCG matvec; everything in d-space is replicated.  Each rank takes its block
from the binding's row partition (row_block) and runs the oracle's sketch and PCG with an
H-apply whose row sum is completed by a gloo all-reduce; both ranks must reproduce the
unsharded oracle (1e-12), and the partition must cover every row exactly once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import nys_inputs as gen
import oracle.nysadmm_oracle as o
from paper_2202_11599_gb300.nysadmm import row_block


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_row_blocks_cover_rows_once():
    for n, world in [(10, 1), (10, 3), (100001, 8), (7, 7)]:
        rows = []
        for r in range(world):
            r0, r1 = row_block(n, world, r)
            assert r1 - r0 in (n // world, n // world + 1)
            rows.extend(range(r0, r1))
        assert rows == list(range(n))
    with pytest.raises(ValueError):
        row_block(3, 4, 0)


def _problem():
    p = gen.lasso_problem(1201, 150, nnz=10, seed=81)
    Om = gen.gaussian_test_matrix(150, 20, 81)
    D = np.random.default_rng(81).random(1201) + 0.1
    return p, Om, D


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, Om, D = _problem()
        r0, r1 = row_block(p.A.shape[0], world, rank)
        Ag, Dg, bg = p.A[r0:r1], D[r0:r1], p.b[r0:r1]

        def allreduce(a):
            t = torch.from_numpy(np.ascontiguousarray(a))
            dist.all_reduce(t)
            return t.numpy()

        def H_sharded(X):                      # one reduction per matvec (d x k)
            return allreduce(Ag.T @ (Dg[:, None] * (Ag @ X)) if X.ndim == 2 else Ag.T @ (Dg * (Ag @ X)))

        U, lam, nu, _, _ = o.nystrom(H_sharded, Om, shift_scale=np.sqrt(150))
        q = allreduce(Ag.T @ bg)
        x, it, res = o.pcg(H_sharded, 0.5, U, lam, q, np.zeros(150), 1e-12)
        out[rank] = (lam, x, it)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_sketch_and_pcg_match_the_unsharded_oracle():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    p, Om, D = _problem()
    H = lambda X: p.A.T @ (D[:, None] * (p.A @ X)) if X.ndim == 2 else p.A.T @ (D * (p.A @ X))
    U, lam, nu, _, _ = o.nystrom(H, Om, shift_scale=np.sqrt(150))
    x, it, _ = o.pcg(H, 0.5, U, lam, p.A.T @ p.b, np.zeros(150), 1e-12)
    for r in range(world):
        lam_r, x_r, it_r = out[r]
        assert np.max(np.abs(lam_r - lam)) <= 1e-12 * lam[0]
        assert np.linalg.norm(x_r - x) <= 1e-12 * np.linalg.norm(x)
        assert it_r == it
    assert np.array_equal(out[0][1], out[1][1])     # replicated state stays identical on the ranks
