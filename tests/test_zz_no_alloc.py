"""The allocation-free H-matvec entry point (nys_hmatvec_noalloc).

Some callers cannot allocate device memory on the request path -- their device
memory belongs to another allocator, or a cudaMalloc/cudaFree pair (cudaFree
synchronises the device) is too costly there.  nys_hmatvec_noalloc serves them
with a fixed scratch array compiled into the library.  This file checks, through
the C ABI, that it returns what nys_hmatvec returns, on two calls in a row (the
shared scratch keeps the previous call's contents), and that a request needing
more scratch than the fixed maximum is refused.  It is named so that pytest
collects it last."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_11599_gb300 import nysadmm
    return nysadmm


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16, torch.float8_e4m3fn])
def test_noalloc_matches_allocating_entry_point(nx, dtype):
    # Both entry points run the same pass plan, kernels and fixed-order partial sums, so the
    # results must be bitwise equal.  d = 777 is not a multiple of any vector width, so the
    # padded partial stride (778 / 780 / 784 / 784 values) differs from d and a stride or
    # offset mistake in the scratch layout would show in the last columns.
    rng = np.random.default_rng(77)
    n, d = 3000, 777
    G = torch.from_numpy(rng.standard_normal((n, d))).cuda()
    A = nx.Matrix.fp8(G) if dtype == torch.float8_e4m3fn else nx.Matrix.padded(G, dtype)
    ct = A.compute_dtype
    D = torch.from_numpy(rng.random(n) + 0.2).cuda()
    for call in range(2):                       # two calls in a row share the scratch
        p = torch.from_numpy(rng.standard_normal(d)).cuda().to(ct)
        y_ref = nx.hmatvec(A, p, 0.25, D if call else None)
        y = nx.hmatvec_noalloc(A, p, 0.25, D if call else None)
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref)


def test_noalloc_refuses_oversized_scratch(nx):
    # 200 rows x 50000 BF16 columns: a valid pass plan whose partial sums
    # (up to 152 blocks x 50000 x 4 B = 30 MB) exceed the 16 MiB scratch.  The allocating
    # entry point accepts the same call, so the scratch limit is the only reason for the refusal.
    A = nx.Matrix(torch.zeros(200, 50000, dtype=torch.bfloat16, device="cuda"))
    p = torch.zeros(50000, dtype=torch.float32, device="cuda")
    y = torch.empty_like(p)
    st = nx.lib().nys_hmatvec_noalloc(ctypes.byref(A.c), None, 0.0, ctypes.c_void_p(p.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(0))
    assert st == nx.NYS_EINVAL
    y_ref = nx.hmatvec(A, p, 0.0)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y_ref).item() == 0
