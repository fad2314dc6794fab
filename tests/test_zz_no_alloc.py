"""The allocation-free FP64 Gram, called through the C ABI, against the workspace entry point.

Some callers cannot call cudaMalloc (a memory-pool or allocator callback, a plugin that is
barred from the device allocator, code that runs while another component captures a CUDA
graph); dopinf_gram_fp64_noalloc serves them with a fixed device array instead of a
workspace.  This file is collected last so that a run stopping at its first failure has run
every other test; it passes alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2504_14338_gb300 import dopinf
    f = dopinf.lib.dopinf_gram_fp64_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return dopinf


def _noalloc(dp, Q, D, accumulate=0):
    n, k = Q.shape
    code = dp.F64 if Q.dtype == torch.float64 else dp.F32
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return dp.lib.dopinf_gram_fp64_noalloc(ctypes.c_void_p(Q.data_ptr()), code, n, k, Q.stride(1), accumulate,
                                           ctypes.c_void_p(D.data_ptr()), D.stride(0), st)


@pytest.mark.parametrize("n,k,dtype", [(1_200_000, 600, torch.float64), (50_001, 130, torch.float32),
                                       (4096, 2816, torch.float64)])
def test_noalloc_gram_matches_workspace_gram_twice(dp, n, k, dtype):
    g = torch.Generator(device="cuda")
    g.manual_seed(n + k)
    Q = torch.randn(k, n, generator=g, device="cuda", dtype=torch.float64).to(dtype).t()
    ref = dp.dopinf_gram(Q)
    diag = torch.diagonal(ref).abs()
    # the FP64 Gram tolerance of the parity tests: 4 sqrt(n) eps sqrt(D_aa D_bb)
    bound = 4 * np.sqrt(n) * EPS * torch.sqrt(torch.outer(diag, diag))
    for _ in range(2):  # the shared array keeps the previous call's contents
        D = torch.full((k, k), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(dp, Q, D) == dp.OK
        torch.cuda.synchronize()
        assert bool(torch.all(torch.abs(D - ref) <= bound))
        assert bool(torch.equal(D, D.t()))


def test_noalloc_accumulate_adds_row_blocks_twice(dp):
    """accumulate = 1 adds Q^T Q of each row block to D, like the workspace entry point does."""
    n, k = 30_000, 200
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    Q = torch.randn(k, n, generator=g, device="cuda", dtype=torch.float64).t()
    ref = dp.dopinf_gram(Q)
    diag = torch.diagonal(ref).abs()
    bound = 8 * np.sqrt(n) * EPS * torch.sqrt(torch.outer(diag, diag))
    for _ in range(2):
        D = torch.zeros(k, k, dtype=torch.float64, device="cuda")
        for a, b in [(0, 10_000), (10_000, 20_000), (20_000, n)]:
            assert _noalloc(dp, Q[a:b], D, accumulate=1) == dp.OK
        torch.cuda.synchronize()
        assert bool(torch.all(torch.abs(D - ref) <= bound))


def test_noalloc_rejects_k_beyond_the_fixed_scratch(dp):
    Q = torch.zeros(2900, 64, dtype=torch.float64, device="cuda").t()   # n = 64, k = 2900
    D = torch.zeros(2900, 2900, dtype=torch.float64, device="cuda")
    assert _noalloc(dp, Q, D) == dp.E_UNSUPPORTED
    assert dp.lib.dopinf_gram_noalloc_scratch_bytes() == 32 << 20
