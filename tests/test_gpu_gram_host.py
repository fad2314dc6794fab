"""Out-of-core Gram: a snapshot matrix in pinned host memory streamed in row blocks through
dopinf_gram_host, against the FP64 oracle (the same tolerances as the device Gram tests)."""
import numpy as np
import pytest
import torch

from oracle import dopinf_oracle as O

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2504_14338_gb300 import dopinf
    return dopinf


def _host(Qn, pad=0):
    n, k = Qn.shape
    dt = torch.float32 if Qn.dtype == np.float32 else torch.float64
    buf = torch.empty(k, n + pad, dtype=dt, pin_memory=True)
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(Qn.T))
    return buf[:, :n].t()


@pytest.mark.parametrize("mode_name,dtype,pad", [("fp64", "f64", 0), ("fp64", "f32", 3), ("ozaki", "f64", 7),
                                                 ("bf16x4", "f32", 0)])
def test_host_streamed_gram_vs_oracle(dp, mode_name, dtype, pad):
    mode = {"fp64": dp.GRAM_FP64, "ozaki": dp.GRAM_OZAKI_FP64, "bf16x4": dp.GRAM_BF16X4}[mode_name]
    rng = np.random.default_rng(17)
    n, k = 100_003, 257
    Qn = rng.standard_normal((n, k)) * np.exp(rng.uniform(-2, 2, k))
    if dtype == "f32":
        Qn = Qn.astype(np.float32)
    Qh = _host(Qn, pad)
    D = dp.dopinf_gram_host(Qh, 30_000, mode=mode).cpu().numpy()     # 4 blocks, the last ragged
    ref = O.gram(Qn)
    sc = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    tol = 2e-6 * sc if mode_name == "bf16x4" else 8 * np.sqrt(n) * EPS * sc
    assert np.all(np.abs(D - ref) <= tol)
    assert np.array_equal(D, D.T)


def test_host_streamed_gram_accumulates_and_single_block(dp):
    """accumulate = 1 adds to D; a block as large as the matrix is one device Gram."""
    rng = np.random.default_rng(18)
    Qn = rng.standard_normal((20_000, 64))
    Qh = _host(Qn)
    ref = O.gram(Qn)
    D = dp.dopinf_gram_host(Qh, 7_000)
    D = dp.dopinf_gram_host(Qh, 7_000, D=D, accumulate=True).cpu().numpy()
    sc = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(D - 2 * ref) <= 16 * np.sqrt(20_000) * EPS * sc)
    one = dp.dopinf_gram_host(Qh, 50_000)
    dev = dp.dopinf_gram(torch.from_numpy(np.ascontiguousarray(Qn.T)).cuda().t())
    assert torch.equal(one, dev)
