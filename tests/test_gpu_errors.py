"""Error paths on the GPU, without a fault: NaN/Inf input to the tensor-core Grams, and bounded
device waits driven to expiry by withholding their signal from the host (the test knob
dopinf_test_expire_waits), after which the context must still work."""
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


def _qmat(n, k, dtype, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randn(k, n, generator=g, device="cuda", dtype=torch.float64).to(dtype).t()


@pytest.mark.parametrize("mode_name", ["bf16x4", "ozaki"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_tensor_gram_reports_nonfinite(dp, mode_name, dtype, bad):
    mode = dp.GRAM_BF16X4 if mode_name == "bf16x4" else dp.GRAM_OZAKI_FP64
    Q = _qmat(3000, 70, dtype, 1)
    Q[1234, 17] = bad
    with pytest.raises(dp.DopinfError) as ei:
        dp.dopinf_gram(Q, mode=mode)
    assert ei.value.status == dp.E_NONFINITE
    D = torch.zeros(70, 70, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    dp.dopinf_gram_async(Q, D, flags, mode=mode)
    torch.cuda.synchronize()
    assert int(flags.item()) & dp.FLAG_NONFINITE and not int(flags.item()) & dp.FLAG_TIMEOUT
    # the same matrix made finite again: a normal result, no flag
    Q[1234, 17] = 0.5
    flags.zero_()
    dp.dopinf_gram_async(Q, D, flags, mode=mode)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    ref = O.gram(Q.cpu().numpy())
    sc = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(D.cpu().numpy() - ref) <= 2e-6 * sc)


@pytest.mark.parametrize("mode_name", ["bf16x4", "ozaki"])
def test_tensor_gram_wait_expires_and_context_survives(dp, mode_name):
    """The MMA issuer never releases a pipeline stage: the TMA producer's and the MMA issuer's
    bounded waits expire, the kernel winds down, the call reports the timeout; then, with the
    knob off, the same call on the same context gives the right D."""
    mode = dp.GRAM_BF16X4 if mode_name == "bf16x4" else dp.GRAM_OZAKI_FP64
    Q = _qmat(20_000, 200, torch.float64, 2)
    prev = dp.dopinf_test_expire_waits(dp.TEST_TENSOR_GRAM)
    try:
        with pytest.raises(dp.DopinfError) as ei:
            dp.dopinf_gram(Q, mode=mode)
        assert ei.value.status == dp.E_TIMEOUT
        D = torch.zeros(200, 200, dtype=torch.float64, device="cuda")
        flags = torch.zeros(1, dtype=torch.int32, device="cuda")
        dp.dopinf_gram_async(Q, D, flags, mode=mode)
        torch.cuda.synchronize()
        assert int(flags.item()) & dp.FLAG_TIMEOUT
    finally:
        dp.dopinf_test_expire_waits(prev)
    D = dp.dopinf_gram(Q, mode=mode).cpu().numpy()
    ref = O.gram(Q.cpu().numpy())
    sc = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(D - ref) <= 2e-6 * sc)


def test_reduce_grid_barrier_wait_expires_and_context_survives(dp):
    """The cooperative tridiagonalisation's grid barrier never releases: every CTA's bounded
    wait expires, dopinf_reduce returns DOPINF_E_TIMEOUT (the asynchronous form flags it); with
    the knob off the same call gives the oracle's eigenvalues."""
    k = 300
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2 * k, k)) @ np.diag(1.1 ** -np.arange(k))
    D = X.T @ X
    Dd = torch.from_numpy(D).cuda()
    prev_coop = dp.dopinf_tune_reduce_coop(1)
    prev = dp.dopinf_test_expire_waits(dp.TEST_GRID_BARRIER)
    try:
        with pytest.raises(dp.DopinfError) as ei:
            dp.dopinf_reduce(Dd, r_cap=8, r_fixed=8)
        assert ei.value.status == dp.E_TIMEOUT
        out = dict(eigvals=torch.empty(8, dtype=torch.float64, device="cuda"),
                   Tr=torch.empty(8, k, dtype=torch.float64, device="cuda").t(),
                   Qhat=torch.empty(k, 8, dtype=torch.float64, device="cuda").t(),
                   r=torch.zeros(1, dtype=torch.int32, device="cuda"),
                   trace=torch.zeros(1, dtype=torch.float64, device="cuda"),
                   flags=torch.zeros(1, dtype=torch.int32, device="cuda"))
        dp.dopinf_reduce_async(Dd, 8, out, r_fixed=8)
        torch.cuda.synchronize()
        assert int(out["flags"].item()) & dp.FLAG_TIMEOUT
    finally:
        dp.dopinf_test_expire_waits(prev)
        dp.dopinf_tune_reduce_coop(prev_coop)
    res = dp.dopinf_reduce(Dd, r_cap=8, r_fixed=8)
    lam_ref = np.linalg.eigvalsh(D)[::-1][:8]
    assert np.all(np.abs(res["eigvals"].cpu().numpy() - lam_ref) <= 1e-10 * lam_ref)
