"""The proposal network's GPU kernels (features, forward, backward, Adam) against the FP64
oracle.  Tolerances: FP32 accumulation over at most 256 terms with BF16-rounded weights on both
sides, so logits agree to ~1e-5 relative and gradients to ~1e-4 normwise."""
import numpy as np
import pytest
import torch

from oracle import dopinf_oracle as O
from oracle import mlp_oracle as M
from paper_2504_14338_gb300 import synth

pytestmark = pytest.mark.gpu
HEADS = (8, 8, 4)


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2504_14338_gb300 import dopinf
    return dopinf


def _params(seed=0):
    rng = np.random.default_rng(seed)
    n_out = sum(HEADS)
    P = M.param_count(n_out)
    p = np.empty(P)
    off = 0
    for o, i in M.layer_shapes(n_out):
        p[off:off + o * i] = rng.uniform(-1, 1, o * i) / np.sqrt(i)
        off += o * i
        p[off:off + o] = rng.uniform(-0.1, 0.1, o)
        off += o
    return p.astype(np.float32).astype(np.float64)


def test_features_match_oracle(dp):
    w = synth.WORKLOADS["small"]
    Qn, _ = synth.snapshots_numpy(w)
    Qt, _, _, _ = O.transform(Qn, w.var_row_offsets())
    D = O.gram(Qt)
    red = O.reduce(D, r_fixed=20)
    ref = M.features(red["lam"][:40], red["trace"], red["Qhat"], w.k)
    lam = torch.from_numpy(red["lam"][:40].copy()).cuda()
    Qh = torch.from_numpy(red["Qhat"].T.copy()).cuda().t()
    f = dp.dopinf_proposal_features(lam, red["trace"], Qh).cpu().numpy().astype(np.float64)
    assert np.allclose(f, ref, rtol=1e-5, atol=1e-5), np.abs(f - ref).max()


def test_forward_backward_adam_match_oracle(dp):
    rng = np.random.default_rng(3)
    n_out = sum(HEADS)
    p = _params()
    B = 96
    X = rng.standard_normal((B, M.N_IN)).astype(np.float32)
    y = np.stack([rng.integers(0, n, B) for n in HEADS], axis=1).astype(np.int32)
    pd = torch.from_numpy(p.astype(np.float32)).cuda()
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    logits = dp.dopinf_mlp_forward(pd, n_out, Xd).cpu().numpy()
    ref_logits, _ = M.forward(p, X.astype(np.float64), n_out)
    assert np.linalg.norm(logits - ref_logits) <= 1e-5 * np.linalg.norm(ref_logits)
    m = torch.zeros_like(pd)
    v = torch.zeros_like(pd)
    loss, g = dp.dopinf_mlp_train_step(pd, m, v, 1, 0.0, HEADS, Xd, yd, want_grad=True)
    ref_loss, ref_g = M.backward(p, X.astype(np.float64), y, HEADS)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss)
    g = g.cpu().numpy()
    for (o, i), off in zip(M.layer_shapes(n_out), np.cumsum([0] + [o * i + o for o, i in M.layer_shapes(n_out)])):
        sl = slice(off, off + o * i + o)
        assert np.linalg.norm(g[sl] - ref_g[sl]) <= 1e-4 * np.linalg.norm(ref_g[sl])
    # an Adam step with lr > 0 moves the parameters as the oracle's update of the same gradient
    lr = 1e-3
    dp.dopinf_mlp_train_step(pd, m, v, 1, lr, HEADS, Xd, yd)
    p_ref, _, _ = M.adam_step(p, g.astype(np.float64), np.zeros_like(p), np.zeros_like(p), 1, lr)
    assert np.max(np.abs(pd.cpu().numpy() - p_ref)) <= 1e-6


def test_training_fits_a_separable_problem(dp):
    rng = np.random.default_rng(4)
    n_out = sum(HEADS)
    B = 256
    X = rng.standard_normal((B, M.N_IN)).astype(np.float32)
    y = np.stack([(X[:, 0] > 0) * 3 + (X[:, 1] > 0), (X[:, 2] > 0) * 5, (X[:, 3] > 0) * 2], axis=1).astype(np.int32)
    pd = torch.from_numpy(_params(1).astype(np.float32)).cuda()
    m = torch.zeros_like(pd)
    v = torch.zeros_like(pd)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    first = None
    for t in range(1, 201):
        loss, _ = dp.dopinf_mlp_train_step(pd, m, v, t, 3e-3, HEADS, Xd, yd)
        if first is None:
            first = float(loss.item())
    last = float(loss.item())
    assert last < 0.05 * first


def test_feature_stats_standardise_and_ranking_vs_oracle(dp):
    """The library's input statistics and standardisation, and its ranking of the grid candidates
    by joint log-probability, against the oracle's definitions."""
    from oracle import mlp_oracle as M
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((300, 64)) * rng.uniform(0.1, 50, 64) + rng.uniform(-5, 5, 64)).astype(np.float32)
    X[:, 7] = 2.5                                               # a constant feature: floored deviation
    Xd = torch.from_numpy(X).cuda()
    mu, sd = dp.dopinf_mlp_feature_stats(Xd)
    rmu, rsd = M.feature_stats(X)
    assert np.allclose(mu.cpu().numpy(), rmu, rtol=1e-13, atol=0)
    assert np.allclose(sd.cpu().numpy(), rsd, rtol=1e-12, atol=0)
    Xs = dp.dopinf_mlp_standardize(Xd, mu, sd).cpu().numpy()
    ref = M.standardise(X, mu.cpu().numpy(), sd.cpu().numpy())     # the same statistics: the same FP32 bits
    assert np.array_equal(Xs, ref)
    for heads, top in [((8, 8, 5), 5), ((6, 6, 3), 12), ((2, 3, 1), 6), ((1, 1, 1), 3)]:
        L = (rng.standard_normal((40, sum(heads))) * 3).astype(np.float32)
        ranked, score = dp.dopinf_mlp_rank(torch.from_numpy(L).cuda(), heads, top)
        idx, sc = M.rank_candidates(L, heads, min(top, int(np.prod(heads))))
        n = idx.shape[1]
        assert np.array_equal(ranked.cpu().numpy()[:, :n], idx)
        assert np.allclose(score.cpu().numpy()[:, :n], sc, rtol=1e-13, atol=1e-13)
        assert np.all(ranked.cpu().numpy()[:, n:] == -1)
