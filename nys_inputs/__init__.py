"""Seeded synthetic workloads for NysADMM (lasso, l1-logistic, test matrices).

This module produces problem DATA only: feature matrices A, responses b,
planted solutions x*, the Gaussian test matrix Omega and the scalar
parameters (gamma, rho, rank).  It holds none of the method's arithmetic and
is the one module shared by the oracle and the CUDA path, so that both sides
see bit-identical inputs.

Shapes and structure follow the workloads of the paper's experiments
(Sec. 5, dataset table): dense n x d feature matrices with polynomial spectral
decay (Sec. 2.2 notes that feature matrices usually show polynomial or
exponential decay).  The paper's datasets (STL-10, CIFAR-10-rf, ...) are not
available offline; these generators stand in for them.

Column index j runs 0..d-1, so the first column has scale (1+0)^-p = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class LassoProblem:
    A: np.ndarray          # (n, d) float64, C-contiguous
    b: np.ndarray          # (n,) float64
    x_true: np.ndarray     # (d,) float64 planted sparse vector
    gamma: float
    rho: float
    rank: int
    seed: int


@dataclasses.dataclass
class LogisticProblem:
    A: np.ndarray          # (n, d) float64
    b: np.ndarray          # (n,) labels in {-1, +1}
    x_true: np.ndarray
    gamma: float
    rho: float
    rank: int
    seed: int


def column_scales(d: int, power: float) -> np.ndarray:
    """scale_j = (1 + j)^(-power), j = 0..d-1."""
    return (1.0 + np.arange(d, dtype=np.float64)) ** (-power)


def sparse_vector(rng: np.random.Generator, d: int, nnz: int, std: float = 1.0) -> np.ndarray:
    x = np.zeros(d)
    idx = rng.choice(d, size=nnz, replace=False)
    x[idx] = std * rng.standard_normal(nnz)
    return x


def lasso_problem(n: int, d: int, *, decay: float = 1.0, nnz: int | None = None,
                  noise: float = 0.01, gamma_frac: float = 0.1, rho: float = 1.0,
                  rank: int = 50, rotate: bool = False, seed: int = 0) -> LassoProblem:
    """Dense lasso instance: A = G diag((1+j)^-decay) [Q^T], b = A x* + noise*N(0,1).

    gamma = gamma_frac * ||A^T b||_inf (the lasso solution is nonzero for gamma_frac < 1).
    With rotate=True the columns are mixed by a random orthogonal Q (QR of a
    Gaussian), so that the singular values are exactly the column scales of G's
    expectation but the decay is not axis-aligned.
    """
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, d))
    A = G * column_scales(d, decay)[None, :]
    if rotate:
        Q, R = np.linalg.qr(rng.standard_normal((d, d)))
        Q = Q * np.sign(np.diag(R))[None, :]
        A = A @ Q.T
    A = np.ascontiguousarray(A)
    if nnz is None:
        nnz = max(1, d // 20)
    x_true = sparse_vector(rng, d, nnz)
    b = A @ x_true + noise * rng.standard_normal(n)
    gamma = gamma_frac * float(np.max(np.abs(A.T @ b)))
    return LassoProblem(A, b, x_true, gamma, rho, rank, seed)


def lasso_small(seed: int = 0) -> LassoProblem:
    """The 2,000 x 500 FP64 lasso: A = G diag((1+j)^-1), 25 nonzeros N(0,1),
    b = A x* + 0.01 N(0,1), gamma = 0.1 ||A^T b||_inf, rho = 1, rank 50."""
    return lasso_problem(2000, 500, decay=1.0, nnz=25, noise=0.01, gamma_frac=0.1,
                         rho=1.0, rank=50, seed=seed)


def logistic_problem(n: int, d: int, *, decay: float = 0.5, nnz: int | None = None,
                     xstd: float = 2.0, gamma_per_row: float = 1e-3, rho: float = 1.0,
                     rank: int = 100, seed: int = 2) -> LogisticProblem:
    """l1-logistic instance: A = N(0, 1/d) diag((1+j)^-decay), labels
    b = sign(A x* + Logistic(0,1)) in {-1,+1}, x* sparse N(0, xstd^2),
    gamma = gamma_per_row * n."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) / math.sqrt(d)
    A = np.ascontiguousarray(A * column_scales(d, decay)[None, :])
    if nnz is None:
        nnz = max(1, d // 50)
    x_true = sparse_vector(rng, d, nnz, std=xstd)
    b = np.sign(A @ x_true + rng.logistic(0.0, 1.0, n))
    b[b == 0] = 1.0
    return LogisticProblem(A, b, x_true, gamma_per_row * n, rho, rank, seed)


def gaussian_test_matrix(d: int, s: int, seed: int) -> np.ndarray:
    """Omega ~ N(0,1)^{d x s}, column-major storage (Fortran order), float64.

    The method draws this matrix; it is passed to both the oracle and the GPU
    path as an input so that the two see the same random numbers."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((d, s)))


def orthonormal_columns(n: int, d: int, seed: int) -> np.ndarray:
    """A with A^T A = I (thin QR of a Gaussian)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, d)))
    return np.ascontiguousarray(Q)


def low_rank_matrix(n: int, d: int, r: int, seed: int) -> np.ndarray:
    """A = G F with G n x r, F r x d Gaussian, so rank(A^T A) = r."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, r)) @ rng.standard_normal((r, d)))


# ---------------------------------------------------------------------------
# Large workloads generated on the GPU with torch (data only).
# ---------------------------------------------------------------------------

def _preload_torch_linalg():
    """torch loads its CUDA linear-algebra library lazily by name; under a profiler
    that changes the library search path this fails, so load it by full path."""
    import ctypes
    import os

    import torch
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        try:
            ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def lasso_large_torch(n: int, d: int, *, nnz_frac: float = 0.01, noise: float = 1e-3,
                      gamma_frac: float = 0.05, seed: int = 1, rotate: bool = True,
                      device: str = "cuda"):
    """The large rotated lasso: A = G diag((1+j)^-1) Q^T with G ~ N(0,1)^{n x d},
    Q from the QR of a d x d Gaussian; x* has nnz_frac*d nonzeros N(0,1);
    b = A x* + noise N(0,1); gamma = gamma_frac ||A^T b||_inf.

    A is formed in FP32 (TF32 off) and returned as FP32; its FP64 widening is
    the problem's exact matrix, and BF16 rounding gives the low-precision copy.
    Returns dict with A32 (n,d) fp32, b (n,) fp64, x_true (d,) fp64, gamma.
    """
    import torch
    _preload_torch_linalg()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        scales = (1.0 + torch.arange(d, device=device, dtype=torch.float64)) ** -1.0
        if rotate:
            M = torch.randn(d, d, generator=g, device=device, dtype=torch.float64)
            Q, R = torch.linalg.qr(M)
            Q = Q * torch.sign(torch.diagonal(R))[None, :]
            S = (scales[:, None] * Q.T).float().contiguous()     # diag(sigma) Q^T  (d x d)
            del M, Q, R
        A32 = torch.empty(n, d, device=device, dtype=torch.float32)
        chunk = max(1, (1 << 28) // d)
        for r0 in range(0, n, chunk):
            r1 = min(n, r0 + chunk)
            Gc = torch.randn(r1 - r0, d, generator=g, device=device, dtype=torch.float32)
            A32[r0:r1] = Gc @ S if rotate else Gc * scales.float()[None, :]
            del Gc
        nnz = max(1, int(round(nnz_frac * d)))
        idx = torch.randperm(d, generator=g, device=device)[:nnz]
        x_true = torch.zeros(d, device=device, dtype=torch.float64)
        x_true[idx] = torch.randn(nnz, generator=g, device=device, dtype=torch.float64)
        b = torch.zeros(n, device=device, dtype=torch.float64)
        for r0 in range(0, n, chunk):
            r1 = min(n, r0 + chunk)
            b[r0:r1] = A32[r0:r1].double() @ x_true
        b += noise * torch.randn(n, generator=g, device=device, dtype=torch.float64)
        Atb = torch.zeros(d, device=device, dtype=torch.float64)
        for r0 in range(0, n, chunk):
            r1 = min(n, r0 + chunk)
            Atb += A32[r0:r1].double().T @ b[r0:r1]
        gamma = gamma_frac * float(Atb.abs().max())
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return {"A32": A32, "b": b, "x_true": x_true, "gamma": gamma}
