"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on seeded inputs.

Tolerances (each derived from the arithmetic, see the comments at each assert):
  transform            bit-exact (same operations, same rounding, fixed summation order)
  Gram (FP64)          |dD| <= 4 sqrt(n) eps max|D|-scale per entry (different summation order)
  eigenvalues          1e-10 relative where lambda_i >= 1e-3 lambda_1, else 8 k eps lambda_1
  Qhat (FP64)          1e-10 relative where eps lambda_1 / gap <= 1e-12, else Davis-Kahan
  learn / rollouts     1e-8 relative on well-conditioned candidates (see test)
"""
import numpy as np
import pytest
import torch

from oracle import dopinf_oracle as O
from paper_2504_14338_gb300 import synth

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


def to_dev(dp, Qn, ld_pad=0):
    n, k = Qn.shape
    dt = torch.float32 if Qn.dtype == np.float32 else torch.float64
    buf = torch.empty(k, n + ld_pad, dtype=dt, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(Qn.T))
    return buf[:, :n].t()


# ------------------------------------------------------------------------------ Step II
@pytest.mark.parametrize("n_vars,n_per,k,pad", [(2, 2048, 200, 0), (3, 333, 37, 5), (1, 7, 1, 0), (4, 1, 9, 3),
                                                (2, 50_001, 13, 0)])
def test_transform_bit_exact_f64(dp, n_vars, n_per, k, pad):
    rng = np.random.default_rng(n_vars * 1000 + k)
    Qn = rng.standard_normal((n_vars * n_per, k)) * rng.uniform(1e-3, 1e3, (n_vars * n_per, 1)) + 3.0
    offs = np.arange(n_vars + 1) * n_per
    Q = to_dev(dp, Qn, pad)
    mean, scale, flags = dp.dopinf_transform(Q, offs)
    ref, rmean, rscale, rflags = O.transform(Qn, offs)
    assert np.array_equal(mean.cpu().numpy(), rmean)
    assert np.array_equal(scale.cpu().numpy(), rscale)
    assert np.array_equal(Q.cpu().numpy(), ref)
    assert int(flags.item()) == rflags


@pytest.mark.parametrize("flags", [1, 2])
def test_transform_flags_center_or_scale_only(dp, flags):
    rng = np.random.default_rng(3)
    Qn = rng.standard_normal((500, 21)) + 2.0
    offs = [0, 200, 500]
    Q = to_dev(dp, Qn)
    dp.dopinf_transform(Q, offs, flags=flags)
    ref, _, _, _ = O.transform(Qn, offs, center=bool(flags & 1), scale=bool(flags & 2))
    assert np.array_equal(Q.cpu().numpy(), ref)


def test_transform_bit_exact_f32(dp):
    rng = np.random.default_rng(11)
    Qn = (rng.standard_normal((3000, 57)) * 7.0 + 1.5).astype(np.float32)
    offs = [0, 1000, 2500, 3000]
    Q = to_dev(dp, Qn)
    mean, scale, flags = dp.dopinf_transform(Q, offs)
    ref, rmean, rscale, rflags = O.transform(Qn, offs)
    assert np.array_equal(mean.cpu().numpy(), rmean)
    assert np.array_equal(scale.cpu().numpy(), rscale)
    assert np.array_equal(Q.cpu().numpy(), ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_transform_std_scaling_vs_oracle(dp, dtype):
    """Standard-deviation scaling: the centring is bit-exact as before; the scale is an FP64
    sum in another order than the oracle's (1e-13 relative; FP32 data then round it to FP32,
    which may move it by one FP32 ulp); and given the GPU's scale the scaled values are the
    oracle's steps bit for bit."""
    rng = np.random.default_rng(31)
    Qn = rng.standard_normal((3000, 41)) * np.repeat([1e-3, 1.0, 5e3], 1000)[:, None] + 2.0
    if dtype == "f32":
        Qn = Qn.astype(np.float32)
    offs = [0, 1000, 2000, 3000]
    Q = to_dev(dp, Qn)
    mean, scale, flags = dp.dopinf_transform(Q, offs, flags=dp.CENTER | dp.SCALE_STD)
    _, rmean, rscale, rflags = O.transform(Qn, offs, scaling="std")
    assert np.array_equal(mean.cpu().numpy(), rmean)
    sc = scale.cpu().numpy()
    assert np.allclose(sc, rscale, rtol=1e-13 if dtype == "f64" else 1.2e-7, atol=0)
    assert int(flags.item()) == rflags == 0
    centred, _, _, _ = O.transform(Qn, offs, scale=False)
    var = np.repeat(np.arange(3), 1000)
    if dtype == "f64":
        expect = centred / sc[var][:, None]
    else:
        expect = centred / sc[var][:, None].astype(np.float32)
    assert np.array_equal(Q.cpu().numpy(), expect)


def test_transform_bit_exact_at_the_ends_of_the_exponent_range(dp):
    """Centred values around 2^+-900 (where the division switches between Markstein's correction
    and the IEEE division), subnormals and mixed magnitudes: still the oracle's bits."""
    rng = np.random.default_rng(900)
    k = 23
    big = np.ldexp(rng.uniform(1, 2, (40, k)) * rng.choice([-1, 1], (40, k)), rng.integers(880, 921, (40, 1)))
    tiny = np.ldexp(rng.uniform(1, 2, (40, k)) * rng.choice([-1, 1], (40, k)), rng.integers(-930, -869, (40, 1)))
    sub = rng.standard_normal((40, k)) * 1e-310
    sub[:, ::3] = rng.standard_normal((40, (k + 2) // 3))
    # rows of a unit-scale variable whose centred values sit around 2^-900
    low = rng.standard_normal((40, k))
    low[20:] = np.ldexp(rng.uniform(1, 2, (20, k)) * rng.choice([-1, 1], (20, k)), rng.integers(-905, -894, (20, 1)))
    Qn = np.vstack([big, tiny, sub, low])
    offs = [0, 40, 80, 120, 160]
    Q = to_dev(dp, Qn)
    mean, scale, _ = dp.dopinf_transform(Q, offs)
    ref, rmean, rscale, _ = O.transform(Qn, offs)
    assert np.array_equal(scale.cpu().numpy(), rscale)
    assert np.array_equal(Q.cpu().numpy(), ref)


def test_transform_zero_scale_and_nonfinite(dp):
    Qn = np.ones((64, 5))
    Qn[32:] = np.arange(5.0)
    Q = to_dev(dp, Qn)
    _, scale, flags = dp.dopinf_transform(Q, [0, 32, 64])
    assert int(flags.item()) & dp.FLAG_ZERO_SCALE
    assert scale.cpu().tolist()[0] == 1.0
    Qn[3, 2] = np.nan
    Q = to_dev(dp, Qn)
    _, _, flags = dp.dopinf_transform(Q, [0, 32, 64])
    assert int(flags.item()) & dp.FLAG_NONFINITE


# ------------------------------------------------------------------------------ Step III Gram
@pytest.mark.parametrize("n,k,dtype", [(4096, 200, "f64"), (20_011, 67, "f64"), (3000, 130, "f32"), (17, 3, "f64"),
                                       (1, 1, "f64")])
def test_gram_fp64_vs_oracle(dp, n, k, dtype):
    rng = np.random.default_rng(n + k)
    Qn = rng.standard_normal((n, k))
    if dtype == "f32":
        Qn = Qn.astype(np.float32)
    Q = to_dev(dp, Qn)
    D = dp.dopinf_gram(Q).cpu().numpy()
    ref = O.gram(Qn)
    # different summation order: |error| <= c * sqrt(n) * eps * sum_i |q_ia q_ib| <= c sqrt(n) eps sqrt(D_aa D_bb)
    bound = 4 * np.sqrt(n) * EPS * np.sqrt(np.outer(np.diag(ref), np.diag(ref))) + 1e-300
    assert np.all(np.abs(D - ref) <= bound)
    assert np.array_equal(D, D.T)
    D2 = dp.dopinf_gram(Q).cpu().numpy()
    assert np.array_equal(D, D2)  # fixed reduction order: run-to-run identical


def test_gram_row_partition_accumulates(dp):
    # the paper's partitioned sum D = sum_i Q_i^T Q_i over row blocks (eq. mos_partitioned)
    rng = np.random.default_rng(21)
    Qn = rng.standard_normal((10_000, 50))
    ref = O.gram(Qn)
    D = None
    for a, b in [(0, 3333), (3333, 6666), (6666, 10_000)]:
        D = dp.dopinf_gram(to_dev(dp, Qn[a:b]), D=D, accumulate=D is not None)
    bound = 8 * np.sqrt(10_000) * EPS * np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(D.cpu().numpy() - ref) <= bound)


@pytest.mark.parametrize("n,k,dtype", [(100_003, 300, "f32"), (40_000, 257, "f64"), (5000, 64, "f32"), (70, 17, "f64")])
def test_gram_bf16x4_vs_oracle(dp, n, k, dtype):
    # two BF16 slices per value leave |e| <= 2^-17 |x| out, with signs varying from row to
    # row.  The H^T H columns of a 128-row chunk receive the 8 MMAs of H^T H products only,
    # each rounding toward zero by at most one ulp of the running chunk sum: <= 8 * 2^-23 of
    # the chunk's sum of |terms|, about 1e-6 (the small products have columns of their own);
    # the chunks are then summed with TwoSum (error ~2^-44).  Allowed: 2e-6.
    rng = np.random.default_rng(n + 7 * k)
    Qn = rng.standard_normal((n, k)) * np.exp(rng.uniform(-3, 3, k))
    if dtype == "f32":
        Qn = Qn.astype(np.float32)
    Q = to_dev(dp, Qn)
    D = dp.dopinf_gram(Q, mode=dp.GRAM_BF16X4).cpu().numpy()
    ref = O.gram(Qn)
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    rel = np.abs(D - ref) / scale
    diag = (np.diag(D) - np.diag(ref)) / np.diag(ref)
    print("bf16x4 max rel", rel.max(), "median", np.median(rel), "diag bias", diag.mean())
    assert rel.max() <= 2e-6
    assert np.array_equal(D, D.T)
    assert np.array_equal(D, dp.dopinf_gram(Q, mode=dp.GRAM_BF16X4).cpu().numpy())  # reproducible


def test_gram_bf16x4_eigenvalues_within_target(dp):
    # a lifted spectrum lambda_i ~ i^-3 (the detonation-shaped case): the split Gram's
    # leading eigenvalues match the FP64 oracle within 1e-6 lambda_1
    w = synth.Workload("t", 4, 25_000, 400, 60, decay=3.0, noise_rel=1e-6, dtype="f32", seed=77)
    Qn, _ = synth.snapshots_numpy(w)
    Qt, _, _, _ = O.transform(Qn, w.var_row_offsets())
    ref = O.gram(Qt)
    D = dp.dopinf_gram(to_dev(dp, Qt), mode=dp.GRAM_BF16X4).cpu().numpy()
    lam_ref = np.linalg.eigvalsh(ref)[::-1]
    lam = np.linalg.eigvalsh(D)[::-1]
    err = np.max(np.abs(lam[:50] - lam_ref[:50])) / lam_ref[0]
    print("top-50 eigenvalue error / lambda_1", err)
    assert err <= 1e-6


@pytest.mark.parametrize("n,k,dtype", [(100_003, 300, "f64"), (4096, 200, "f64"), (20_011, 129, "f32"), (70, 17, "f64")])
def test_gram_ozaki_fp64_vs_oracle(dp, n, k, dtype):
    # exact digit products: the only errors are the digit truncation (2^-57 of the column's
    # scale 2^s_a, plus dropped products below 2^-55 of it) and the FP64 sums of the partials,
    # far inside the FP64 path's bound
    rng = np.random.default_rng(n + 3 * k)
    Qn = rng.standard_normal((n, k)) * np.exp(rng.uniform(-3, 3, k)) * np.exp(rng.uniform(-2, 2, (n, 1)))
    if dtype == "f32":
        Qn = Qn.astype(np.float32)
    Q = to_dev(dp, Qn)
    D = dp.dopinf_gram(Q, mode=dp.GRAM_OZAKI_FP64).cpu().numpy()
    ref = O.gram(Qn)
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    rel = np.abs(D - ref) / scale
    print("ozaki max rel", rel.max())
    assert np.all(np.abs(D - ref) <= 4 * np.sqrt(n) * EPS * scale)
    assert np.array_equal(D, D.T)


def test_gram_ozaki_exact_on_integers(dp):
    # small integers have exact digits and exact FP64 sums: D must equal Q^T Q exactly
    rng = np.random.default_rng(9)
    Qn = rng.integers(-1000, 1001, (30_000, 96)).astype(np.float64)
    D = dp.dopinf_gram(to_dev(dp, Qn), mode=dp.GRAM_OZAKI_FP64).cpu().numpy()
    assert np.array_equal(D, O.gram(Qn))


# ------------------------------------------------------------------------------ Step III reduce
def _pipeline_D(seed=1234, n_vars=2, n_per=2048, k=200, r_true=6, scales=()):
    w = synth.Workload("t", n_vars, n_per, k, r_true, var_scales=scales, seed=seed)
    Qn, _ = synth.snapshots_numpy(w)
    Qt, _, _, _ = O.transform(Qn, w.var_row_offsets())
    return O.gram(Qt), Qt


def _align_signs(U_ref, U):
    s = np.sign(np.sum(U_ref * U, axis=0))
    s[s == 0] = 1
    return U * s


def assert_eigen_qhat(lam, lam_ref, Qh, Qh_ref, k, r):
    """The FP64 tolerance of the reduce step (1e-10 relative) where the problem allows it.

    Eigenvalues: 1e-10 relative where lambda_i >= 1e-3 lambda_1; below that the eigenvalue
    is magnitude-limited (any backward-stable solver moves it by about k eps lambda_1, Weyl),
    and the bound 8 k eps lambda_1 is asserted instead.  Qhat rows: 1e-10 relative where the
    perturbation estimate eps lambda_1 / gap_i is at most 1e-12 (100 times the rounding of a
    backward-stable eigensolver); the others are gap-limited and get the Davis-Kahan bound
    1e3 k eps lambda_1 / gap_i + 1e-10.  Returns the names of the limited modes."""
    lam_all = np.asarray(lam_ref)
    lam_ref = lam_all[:r]
    strict = lam_ref >= 1e-3 * lam_ref[0]
    rel = np.abs(lam - lam_ref) / np.abs(lam_ref)
    assert np.all(rel[strict] <= 1e-10), rel[strict].max()
    assert np.all(np.abs(lam - lam_ref)[~strict] <= 8 * k * EPS * lam_ref[0])
    limited = {"magnitude_limited_eigenvalues": np.nonzero(~strict)[0].tolist(), "gap_limited_qhat_rows": []}
    worst = 0.0
    if Qh_ref is not None:
        for j in range(r):
            gap = min(abs(lam_all[j - 1] - lam_all[j]) if j else np.inf,
                      abs(lam_all[j] - lam_all[j + 1]) if j + 1 < len(lam_all) else np.inf)
            err = np.linalg.norm(Qh[j] - Qh_ref[j]) / np.linalg.norm(Qh_ref[j])
            dk = k * EPS * lam_ref[0] / gap
            if EPS * lam_ref[0] / gap <= 1e-12:
                assert err <= 1e-10, (j, err)
                worst = max(worst, err)
            else:
                limited["gap_limited_qhat_rows"].append(j)
                assert err <= 1e3 * dk + 1e-10, (j, err)
    print("eigenvalue max rel (strict modes) %.2e, Qhat max rel (strict rows) %.2e, limited %s"
          % (rel[strict].max(), worst, limited))
    return limited


@pytest.mark.parametrize("k,r_cap", [(200, 12), (61, 61), (3, 2), (1, 1), (130, 40)])
def test_reduce_vs_oracle(dp, k, r_cap):
    rng = np.random.default_rng(k)
    X = rng.standard_normal((max(3 * k, 10), k)) @ np.diag(1.2 ** -np.arange(k))
    D = X.T @ X
    Dd = torch.from_numpy(D).cuda()
    res = dp.dopinf_reduce(Dd, r_cap=r_cap, r_fixed=r_cap)
    lam_ref, U_ref = O.eig_desc(D)
    lam = res["eigvals"].cpu().numpy()
    Qh = res["Qhat"].cpu().numpy()
    Qh_ref = O.projection(D, U_ref, lam_ref, r_cap)[1] if lam_ref[r_cap - 1] > 0 else None
    # with k = r_cap the next eigenvalue is absent: its gap is the distance to the end
    lam_full = np.concatenate([lam_ref, [0.0]]) if r_cap == k else lam_ref
    assert_eigen_qhat(lam, lam_full, Qh, Qh_ref, k, r_cap)
    # eigenvectors (T_r scaled back): the same gap rule
    gaps = np.abs(np.diff(lam_full))
    Tr = res["Tr"].cpu().numpy()
    U = Tr * np.sqrt(np.maximum(lam, 1e-300))
    for j in range(r_cap):
        gap = min(gaps[j - 1] if j > 0 else np.inf, gaps[j] if j < len(gaps) else np.inf)
        dk = k * EPS * lam_ref[0] / gap
        bound = 1e-10 if EPS * lam_ref[0] / gap <= 1e-12 else 1e3 * dk + 1e-12
        assert np.linalg.norm(U[:, j] - U_ref[:, j]) <= bound, j


@pytest.mark.parametrize("s", [-300, 300])
def test_reduce_exact_under_power_of_two_scaling(dp, s):
    """D and 2^s D (s even): every step scales exactly (norms, reflectors, the bisection on the
    normalised tridiagonal, inverse iteration), so the eigenvalues scale by 2^s and T_r^T, Qhat by
    2^(-s/2), 2^(s/2) bit for bit; far from 1 the Sturm recurrence rescales its minors."""
    k, r_cap = 301, 10
    rng = np.random.default_rng(77)
    X = rng.standard_normal((2 * k, k)) @ np.diag(1.15 ** -np.arange(k))
    D = X.T @ X
    a = dp.dopinf_reduce(torch.from_numpy(D).cuda(), r_cap=r_cap, r_fixed=r_cap)
    b = dp.dopinf_reduce(torch.from_numpy(np.ldexp(D, s)).cuda(), r_cap=r_cap, r_fixed=r_cap)
    def host(t):
        return t.cpu().numpy()
    # np.ldexp scales exactly (a device pow(2, s) need not be exact)
    assert np.array_equal(np.ldexp(host(a["eigvals"]), s), host(b["eigvals"]))
    assert np.array_equal(np.ldexp(host(a["Tr"]), -s // 2), host(b["Tr"]))
    assert np.array_equal(np.ldexp(host(a["Qhat"]), s // 2), host(b["Qhat"]))


def test_reduce_large_k_vectors_outside_shared_memory(dp):
    """k above the shared-memory size of inverse iteration (4000): eigenvalues against LAPACK's,
    eigenvector residuals ||D u - lambda u|| against the FP64 bound."""
    k, r_cap = 4001, 6
    rng = np.random.default_rng(4001)
    X = rng.standard_normal((k + 100, k)) @ np.diag(1.002 ** -np.arange(k))
    D = X.T @ X
    res = dp.dopinf_reduce(torch.from_numpy(D).cuda(), r_cap=r_cap, r_fixed=r_cap)
    lam_ref = np.linalg.eigvalsh(D)[::-1][:r_cap]
    lam = res["eigvals"].cpu().numpy()
    assert np.all(np.abs(lam - lam_ref) <= 1e-10 * lam_ref + 8 * k * EPS * lam_ref[0])
    U = res["Tr"].cpu().numpy() * np.sqrt(lam)
    for j in range(r_cap):
        u = U[:, j]
        assert abs(np.linalg.norm(u) - 1.0) <= 1e-12
        assert np.linalg.norm(D @ u - lam[j] * u) <= 1e3 * k * EPS * lam_ref[0]


@pytest.mark.parametrize("k", [3, 4, 9, 200, 601])
def test_reduce_cooperative_matches_per_column_launches(dp, k):
    """The one-launch tridiagonalisation (grid barrier per column) gives the same bits as
    three launches per column."""
    rng = np.random.default_rng(100 + k)
    X = rng.standard_normal((2 * k, k)) @ np.diag(1.1 ** -np.arange(k))
    Dd = torch.from_numpy(X.T @ X).cuda()
    r_cap = min(k, 8)
    prev = dp.dopinf_tune_reduce_coop(1)
    try:
        a = dp.dopinf_reduce(Dd, r_cap=r_cap, r_fixed=r_cap)
        dp.dopinf_tune_reduce_coop(0)
        b = dp.dopinf_reduce(Dd, r_cap=r_cap, r_fixed=r_cap)
    finally:
        dp.dopinf_tune_reduce_coop(prev)
    for key in ("eigvals", "Tr", "Qhat"):
        assert torch.equal(a[key], b[key]), key


def test_reduce_energy_rank_and_pipeline_qhat(dp):
    D, _ = _pipeline_D()
    ref = O.reduce(D, tau=0.9996, r_cap=None)
    res = dp.dopinf_reduce(torch.from_numpy(D).cuda(), r_cap=20, energy_target=0.9996)
    assert 1 <= ref["r"] <= 20
    assert res["r"] == ref["r"]
    assert abs(res["trace"] - np.trace(D)) <= 1e-13 * abs(np.trace(D))
    r = ref["r"]
    Qh = res["Qhat"].cpu().numpy()[:r]
    Qh_ref = O.reduce(D, r_fixed=r)["Qhat"]
    rel = np.linalg.norm(Qh - Qh_ref, axis=1) / np.linalg.norm(Qh_ref, axis=1)
    print("Qhat row rel err", rel)
    assert np.all(rel < 1e-10)
    assert_eigen_qhat(res["eigvals"].cpu().numpy()[:r], ref["lam"], Qh, Qh_ref, D.shape[0], r)
    # the target is out of reach of r_cap = 1 eigenpairs: the energy rule reports it
    with pytest.raises(dp.DopinfError) as ei:
        dp.dopinf_reduce(torch.from_numpy(D).cuda(), r_cap=1, energy_target=0.9996)
    assert ei.value.status == dp.E_RANK


# ------------------------------------------------------------------------------ Step IV
def _reduced(r_fixed=6, seed=1234, **kw):
    D, _ = _pipeline_D(seed=seed, **kw)
    return O.reduce(D, r_fixed=r_fixed)["Qhat"]


@pytest.fixture(params=["dw", "fp64"])
def arith(request, dp):
    """The learn rollouts in double-word FP32 (the default) and in FP64."""
    code = dp.ROLLOUT_DW if request.param == "dw" else dp.ROLLOUT_FP64
    prev = dp.dopinf_tune_rollout_arith(code)
    yield request.param
    dp.dopinf_tune_rollout_arith(prev)


def _oracle_rollout_metrics(Op, r, Qh, n_steps, mode, dt, max_growth=1.2):
    """The oracle's rollout of a given operator with Step IV's metrics: status (0 valid,
    2 non-finite, 3 growth), the state index where a rollout that stops early stops (the first
    state that is non-finite or brings the growth to max_growth), training error, growth, and
    how far (relative) the deciding growth value lies from the threshold."""
    Qr = np.asarray(Qh, dtype=np.float64)[:r].T
    k = Qr.shape[0]
    traj = O.rollout(Op, r, Qr[0], n_steps, mode=mode, dt=dt)
    mu = Qr.mean(axis=0)
    mdt = np.max(np.abs(Qr - mu), axis=0)
    denom = np.max(mdt)
    fin = np.all(np.isfinite(traj), axis=1)
    with np.errstate(invalid="ignore"):
        dev = np.where(fin, np.max(np.abs(traj - mu), axis=1), 0.0)
    g = np.maximum.accumulate(dev) / denom
    bad = (~fin) | (g >= max_growth)
    if bad.any():
        t = int(np.argmax(bad))
        st = 2 if not fin[t] else 3
        margin = abs(g[t] / max_growth - 1.0) if fin[t] else np.inf
        if t > 0 and fin[t]:
            margin = min(margin, abs(g[t - 1] / max_growth - 1.0))
        return dict(status=st, steps=t, err=np.inf, growth=g[t] if fin[t] else np.inf, margin=margin)
    return dict(status=0, steps=n_steps - 1, err=O.train_error(Qr[:k], traj[:k]),
                growth=O.growth_ratio(traj, mu, mdt), margin=abs(g[-1] / max_growth - 1.0))


def _learn_parity(dp, Qh, r_list, b1, b2, n_steps, mode, dt, rollout_tol=1e-8):
    """dopinf_learn against the oracle on every candidate:
    (a) operators: each candidate's O against the oracle's Cholesky solve, normwise, within
        4 d eps cond(G + reg) (two backward-stable solves of the same system; cond is bounded
        above by (lambda_max(G) + max beta) / (lambda_min(G) + min beta), G positive semi-definite);
    (b) rollouts: status and stop step of every candidate, training error and growth of every
        valid one, against the oracle's rollout of the GPU's own operator (1e-8 relative, the
        rollout tolerance), except where the deciding growth lies within 1e-8 of the threshold;
    (c) selection: the GPU's pick is the lowest-index minimum over its valid candidates, and the
        oracle's pick is valid on the GPU with an error within the tolerances of the minimum."""
    mcode = dp.DISCRETE if mode == "discrete" else dp.CONTINUOUS_RK4
    Qd = torch.from_numpy(np.ascontiguousarray(Qh.T)).cuda().t()
    res = dp.dopinf_learn(Qd, r_list, b1, b2, n_steps, mode=mcode, dt=dt, operators=True)
    st = res["status"].cpu().numpy()
    err = res["train_err"].cpu().numpy()
    gro = res["growth"].cpu().numpy()
    steps = res["steps"].cpu().numpy()
    nb = len(b1) * len(b2)
    checked = dict(ops=0, roll=0, skipped_edge=0)
    for ir, r in enumerate(r_list):
        Dh, Y = O.learning_data(Qh, r, mode, dt)
        G, B = O.normal_equations(Dh, Y)
        lam = np.linalg.eigvalsh(G)
        d = G.shape[0]
        for p in range(nb):
            c = ir * nb + p
            bb1, bb2 = b1[p // len(b2)], b2[p % len(b2)]
            Oref, ok = O.solve_cholesky(G, B, O.regulariser(r, bb1, bb2))
            cond = (lam[-1] + max(bb1, bb2)) / (max(lam[0], 0.0) + min(bb1, bb2))
            if not ok:
                assert st[c] == 1 or cond * EPS > 1e-3, (c, st[c])
                continue
            if st[c] == 1:
                assert cond * EPS > 1e-3, (c, cond)   # breakdown only where the system is near singular
                continue
            Og = res["operators"][c].cpu().numpy()
            tol = 4 * d * EPS * cond
            rel = np.linalg.norm(Og - Oref) / np.linalg.norm(Oref)
            assert rel <= max(tol, 1e-14), (r, bb1, bb2, rel, tol)
            checked["ops"] += 1
            m = _oracle_rollout_metrics(Og, r, Qh, n_steps, mode, dt)
            if m["margin"] < 1e-8:
                checked["skipped_edge"] += 1
                continue
            assert st[c] == m["status"], (c, r, bb1, bb2, st[c], m)
            assert steps[c] == m["steps"], (c, steps[c], m["steps"])
            if m["status"] == 0:
                # the training error compares two nearly equal trajectories when it is small: a
                # relative trajectory difference delta moves it by at most delta (1 + err), so
                # an absolute 1e-10 (far above the FP64 and double-word rounding) is allowed too
                assert abs(err[c] - m["err"]) <= rollout_tol * m["err"] + 1e-10, (c, err[c], m["err"])
                assert abs(gro[c] - m["growth"]) <= rollout_tol * m["growth"], (c, gro[c], m["growth"])
            elif m["status"] == 3:
                # the growth of a stopped rollout is read where it diverges, which amplifies the
                # rounding differences of the two arithmetics: both must be past the threshold
                assert gro[c] >= 1.2, (c, gro[c], m)
            checked["roll"] += 1
    valid = np.nonzero(st == 0)[0]
    if valid.size:
        emin = err[valid].min()
        assert res["best"] == int(valid[np.argmax(err[valid] == emin)])
    else:
        assert res["best"] == -1
    return res, checked


@pytest.mark.parametrize("mode", ["discrete", "continuous"])
def test_learn_vs_oracle(dp, mode, arith):
    Qh = _reduced(r_fixed=6)
    b1 = synth.logspace(-8, 2, 4)
    b2 = synth.logspace(-8, 2, 4)
    dt = synth.WORKLOADS["small"].snap_dt
    res, checked = _learn_parity(dp, Qh, [4, 6], b1, b2, 400, mode, dt)
    print(checked)
    assert checked["ops"] >= 24 and checked["roll"] >= 24
    ref = O.learn(Qh, [4, 6], b1, b2, 400, mode=mode, dt=dt)
    best = res["best"]
    assert best >= 0 and ref["best"] >= 0
    # the chosen candidate is (within rounding) a minimiser of the oracle's training error
    assert ref["valid"][best]
    assert ref["train_err"][best] <= ref["train_err"][ref["best"]] * (1 + 1e-6) + 1e-12


@pytest.mark.parametrize("mode", ["discrete", "continuous"])
def test_learn_qr_solver_vs_oracle(dp, mode):
    """The QR route of the regularised problems (no normal equations): every candidate's
    operators against the oracle at the conditioning tolerance, statuses and metrics against the
    oracle's rollouts; and, where the problem is well conditioned, the operators against the
    oracle's own QR solve to 1e-10."""
    Qh = _reduced(r_fixed=6)
    b1 = synth.logspace(-8, 2, 4)
    b2 = synth.logspace(-8, 2, 4)
    dt = synth.WORKLOADS["small"].snap_dt
    prev = dp.dopinf_tune_learn_solver(dp.SOLVE_QR)
    try:
        res, checked = _learn_parity(dp, Qh, [4, 6], b1, b2, 400, mode, dt)
    finally:
        dp.dopinf_tune_learn_solver(prev)
    assert checked["ops"] >= 24 and checked["roll"] >= 24
    for c in range(len(res["operators"])):
        r = [4, 6][c // 16]
        bb1, bb2 = b1[(c % 16) // 4], b2[c % 4]
        if min(bb1, bb2) < 1e-2:
            continue
        Dh, Y = O.learning_data(Qh, r, mode, dt)
        Oq, ok = O.solve_qr(Dh, Y, O.regulariser(r, bb1, bb2))
        Og = res["operators"][c].cpu().numpy()
        assert ok and np.linalg.norm(Og - Oq) <= 1e-10 * np.linalg.norm(Oq), c


_LARGE = {}


def _reduced_large(r_fixed):
    """Reduced data with up to 80 modes from a step-flow-style system (r_true = 40, two
    variables x 3000 rows, k = 400): the modes past 40 carry the noise, as in the batched
    learn workloads that fit r up to 80 on such data."""
    if "Qh" not in _LARGE:
        w = synth.Workload("large-r", 2, 3000, 400, 40, seed=4040)
        Qn, _ = synth.snapshots_numpy(w)
        Qt, _, _, _ = O.transform(Qn, w.var_row_offsets())
        _LARGE["Qh"] = O.reduce(O.gram(Qt), r_fixed=80)["Qhat"]
    return _LARGE["Qh"][:r_fixed]


@pytest.mark.parametrize("r", [33, 48, 64])
@pytest.mark.parametrize("mode", ["discrete", "continuous"])
def test_learn_large_r_vs_oracle(dp, r, mode, arith):
    """r above 32 (operator rows in shared memory, block-Schur solves with quadratic blocks of
    s = 561 .. 2080): operators, statuses, stop steps and metrics of every candidate."""
    Qh = _reduced_large(r)
    b1 = synth.logspace(-6, 0, 3)
    b2 = synth.logspace(-2, 4, 3)
    res, checked = _learn_parity(dp, Qh, [r], b1, b2, 400, mode, 1e-2)
    print(r, mode, checked, res["status"].cpu().numpy())
    assert checked["ops"] >= 6 and checked["roll"] >= 6


def test_learn_r80_vs_oracle(dp, arith):
    """The largest r of the batched-learn workloads (d = 3321 > the 399 data rows): short RK4
    horizon, every candidate against the oracle."""
    Qh = _reduced_large(80)
    b1 = synth.logspace(-4, 0, 2)
    b2 = synth.logspace(0, 4, 2)
    res, checked = _learn_parity(dp, Qh, [80], b1, b2, 400, "continuous", 1e-2)
    print(checked, res["status"].cpu().numpy())
    assert checked["ops"] >= 3 and checked["roll"] >= 3


def _learn_outputs(res):
    return [res["train_err"], res["growth"], res["status"], res["O_best"]]


def test_learn_double_word_matches_fp64(dp):
    """Double-word and FP64 rollouts of the same grid: the same statuses and step counts;
    training errors and growths of the valid candidates within 1e-10 relative (rounding of the
    two arithmetics).  An invalid candidate's growth is read at the step its rollout diverged,
    where the divergence has amplified the rounding differences by an amount that depends on
    the rollout: there both must be at or above the threshold."""
    Qh = _reduced(r_fixed=12)
    Qd = torch.from_numpy(Qh.T.copy()).cuda().t()
    b1 = synth.logspace(-8, 2, 5)
    b2 = synth.logspace(-8, 2, 5)
    dt = synth.WORKLOADS["small"].snap_dt
    prev = dp.dopinf_tune_rollout_arith(0)
    try:
        out = {}
        for a in (dp.ROLLOUT_FP64, dp.ROLLOUT_DW):
            dp.dopinf_tune_rollout_arith(a)
            out[a] = dp.dopinf_learn(Qd, [4, 8, 12], b1, b2, 600, mode=dp.CONTINUOUS_RK4, dt=dt)
    finally:
        dp.dopinf_tune_rollout_arith(prev)
    f, w = out[dp.ROLLOUT_FP64], out[dp.ROLLOUT_DW]
    st = f["status"].cpu().numpy()
    assert (st == 0).sum() >= 3
    assert np.array_equal(st, w["status"].cpu().numpy())
    assert np.array_equal(f["steps"].cpu().numpy(), w["steps"].cpu().numpy())
    assert f["best"] == w["best"]
    for key in ("train_err", "growth"):
        a, b = f[key].cpu().numpy(), w[key].cpu().numpy()
        fin = np.isfinite(a)
        assert np.array_equal(fin, np.isfinite(b)), key
        ok = fin & (st == 0)
        rel = np.abs(a[ok] - b[ok]) / np.abs(a[ok])
        assert rel.max() <= 1e-10, (key, rel.max())
    gro = st == 3
    assert np.all(f["growth"].cpu().numpy()[gro] >= 1.2) and np.all(w["growth"].cpu().numpy()[gro] >= 1.2)


@pytest.mark.parametrize("edge", [1.0 + 1e-13, 1.0 - 1e-13, 1.0 + 1e-9])
def test_learn_double_word_growth_threshold_edge(dp, edge):
    """max_growth set right at a valid candidate's FP64 growth (just above, just below): the
    double-word rollouts must not decide a growth that close to the threshold themselves, so
    statuses, step counts and the selection are those of the FP64 arithmetic."""
    Qh = _reduced(r_fixed=12)
    Qd = torch.from_numpy(Qh.T.copy()).cuda().t()
    b1 = synth.logspace(-8, 2, 5)
    b2 = synth.logspace(-8, 2, 5)
    dt = synth.WORKLOADS["small"].snap_dt
    prev = dp.dopinf_tune_rollout_arith(0)
    try:
        dp.dopinf_tune_rollout_arith(dp.ROLLOUT_FP64)
        base = dp.dopinf_learn(Qd, [4, 8, 12], b1, b2, 600, mode=dp.CONTINUOUS_RK4, dt=dt)
        st = base["status"].cpu().numpy()
        gro = base["growth"].cpu().numpy()
        valid = np.nonzero(st == 0)[0]
        assert valid.size >= 2
        c = valid[np.argmax(gro[valid])]          # the valid candidate closest to the threshold
        mg = float(gro[c]) * edge
        out = {}
        for a in (dp.ROLLOUT_FP64, dp.ROLLOUT_DW):
            dp.dopinf_tune_rollout_arith(a)
            out[a] = dp.dopinf_learn(Qd, [4, 8, 12], b1, b2, 600, mode=dp.CONTINUOUS_RK4, dt=dt, max_growth=mg)
    finally:
        dp.dopinf_tune_rollout_arith(prev)
    f, w = out[dp.ROLLOUT_FP64], out[dp.ROLLOUT_DW]
    assert (int(f["status"][c].item()) == 0) == (edge > 1.0)
    assert torch.equal(f["status"], w["status"])
    assert torch.equal(f["steps"], w["steps"])
    assert f["best"] == w["best"]


def test_learn_double_word_out_of_range_runs_fp64(dp):
    """Reduced data far outside the double-word range (2^70 scale): every candidate is handed to
    the FP64 kernel, so the results are bit for bit those of the FP64 arithmetic."""
    Qh = _reduced(r_fixed=6) * 2.0 ** 70
    Qd = torch.from_numpy(Qh.T.copy()).cuda().t()
    b1 = synth.logspace(-8, 2, 3)
    b2 = synth.logspace(-8, 2, 3)
    prev = dp.dopinf_tune_rollout_arith(0)
    try:
        out = {}
        for a in (dp.ROLLOUT_FP64, dp.ROLLOUT_DW):
            dp.dopinf_tune_rollout_arith(a)
            out[a] = dp.dopinf_learn(Qd, [4, 6], b1, b2, 300, mode=dp.CONTINUOUS_RK4,
                                     dt=synth.WORKLOADS["small"].snap_dt)
    finally:
        dp.dopinf_tune_rollout_arith(prev)
    assert out[dp.ROLLOUT_FP64]["best"] == out[dp.ROLLOUT_DW]["best"]
    for key in ("train_err", "growth", "status", "steps", "O_best"):
        assert torch.equal(out[dp.ROLLOUT_FP64][key], out[dp.ROLLOUT_DW][key]), key


def test_learn_ignores_extra_qhat_rows(dp):
    """Qhat may hold more rows than the largest r of the list (every r uses its leading rows)."""
    Qh = _reduced(r_fixed=12)
    b1 = synth.logspace(-8, 2, 3)
    b2 = synth.logspace(-8, 2, 3)
    full = torch.from_numpy(Qh.T.copy()).cuda().t()
    lead = torch.from_numpy(Qh[:6].T.copy()).cuda().t()
    a = dp.dopinf_learn(full, [4, 6], b1, b2, 300)
    b = dp.dopinf_learn(lead, [4, 6], b1, b2, 300)
    assert a["best"] == b["best"]
    for x, y in zip(_learn_outputs(a)[:3], _learn_outputs(b)[:3]):
        assert torch.equal(x, y)


def test_rollout_vs_oracle(dp):
    Qh = _reduced(r_fixed=5)
    Dh, Y = O.learning_data(Qh, 5)
    G, B = O.normal_equations(Dh, Y)
    Op, ok = O.solve_cholesky(G, B, O.regulariser(5, 1e-2, 1e-1))
    assert ok
    for mode, mc in [("discrete", 0), ("continuous", 1)]:
        ref = O.rollout(Op, 5, Qh[:, 0], 300, mode=mode, dt=1e-3)
        Od = torch.from_numpy(Op.T.copy()).cuda().t()
        Qt, fin = dp.dopinf_rollout(Od, torch.from_numpy(Qh[:, 0].copy()).cuda(), 300, mode=mc, dt=1e-3)
        assert int(fin.item()) == 1
        Qt = Qt.cpu().numpy()
        rel = np.linalg.norm(Qt - ref) / np.linalg.norm(ref)
        assert rel < 1e-8, (mode, rel)


def _stable_operator(r, seed):
    """A seeded quadratic operator [A | H | c] with a contracting linear part."""
    rng = np.random.default_rng(seed)
    d = r + r * (r + 1) // 2 + 1
    Op = np.zeros((r, d))
    Op[:, :r] = -0.5 * np.eye(r) + 0.05 * rng.standard_normal((r, r)) / np.sqrt(r)
    Op[:, r:d - 1] = 0.02 * rng.standard_normal((r, d - r - 1)) / r
    Op[:, d - 1] = 0.01 * rng.standard_normal(r)
    return Op, 0.5 * rng.standard_normal(r)


@pytest.mark.parametrize("r", [1, 2, 7, 16, 30, 32, 33, 36, 47, 64, 80, 92])
def test_rollout_every_width_vs_oracle(dp, r):
    """r <= 32 runs the register kernel (1 to 5 column slots per thread), 32 < r <= 96 the
    shared-memory kernel (3 to 8 rows per CTA, clusters of up to 16 CTAs, r = 92 filling the
    227 KB of shared memory); both against the
    oracle's rollout."""
    Op, q0 = _stable_operator(r, 100 + r)
    Od = torch.from_numpy(Op.T.copy()).cuda().t()
    q0d = torch.from_numpy(q0.copy()).cuda()
    for mode, mc, dt in [("discrete", 0, 1.0), ("continuous", 1, 1e-2)]:
        ref = O.rollout(Op, r, q0, 300, mode=mode, dt=dt)
        Qt, fin = dp.dopinf_rollout(Od, q0d, 300, mode=mc, dt=dt)
        assert int(fin.item()) == 1
        Qt = Qt.cpu().numpy()
        assert np.array_equal(Qt[0], q0)
        rel = np.linalg.norm(Qt - ref) / np.linalg.norm(ref)
        assert rel < 1e-12, (r, mode, rel)


@pytest.mark.parametrize("r", [5, 16, 30])
def test_rollout_same_bits_for_every_rows_setting(dp, r):
    """1, 2 or 4 operator rows per CTA (clusters of up to 16 CTAs) give the same trajectory."""
    Op, q0 = _stable_operator(r, 7 * r)
    Od = torch.from_numpy(Op.T.copy()).cuda().t()
    q0d = torch.from_numpy(q0.copy()).cuda()
    prev = dp.dopinf_tune_rollout_rows(0)
    out = {}
    try:
        for rc in (1, 2, 4):
            dp.dopinf_tune_rollout_rows(rc)
            out[rc] = dp.dopinf_rollout(Od, q0d, 200, mode=1, dt=1e-2)[0]
    finally:
        dp.dopinf_tune_rollout_rows(prev)
    for rc in (2, 4):
        assert torch.equal(out[rc], out[1]), rc


def test_rollout_nonfinite_stops_writing(dp):
    """A rollout that overflows reports finite = 0 and leaves the rows after the first
    non-finite state unwritten, like the oracle's trajectory up to that state."""
    r = 6
    Op, q0 = _stable_operator(r, 5)
    Op[:, r:-1] *= 1e6  # a strongly quadratic map blows up within a few steps
    q0 = q0 * 10
    ref = O.rollout(Op, r, q0, 60, mode="discrete")
    bad = int(np.argmax(~np.all(np.isfinite(ref), axis=1)))
    assert bad > 0
    Od = torch.from_numpy(Op.T.copy()).cuda().t()
    Qt, fin = dp.dopinf_rollout(Od, torch.from_numpy(q0.copy()).cuda(), 60, mode=0)
    assert int(fin.item()) == 0
    Qt = Qt.cpu().numpy()
    good = ref[:bad]
    rel = np.abs(Qt[:bad] - good) / np.maximum(np.abs(good), 1e-300)
    assert np.all(rel[np.isfinite(rel)] < 1e-8)
    assert not np.all(np.isfinite(Qt[bad]))
