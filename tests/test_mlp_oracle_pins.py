"""Pins of the proposal-network oracle: library routines (BF16 conversion, erf, logsumexp),
finite differences, closed forms of Adam's first step and of the features on sinusoids."""
import math

import numpy as np
import torch
from scipy.special import logsumexp

from oracle import mlp_oracle as M


def test_bf16_round_matches_library_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.uniform(-5, 5, 1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)
    assert M.bf16_round(1.0 + 2 ** -8) == 1.0            # tie to even (down)
    assert M.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie to even (up)


def test_gelu_and_its_derivative():
    z = np.linspace(-6, 6, 101)
    expect = np.array([0.5 * t * (1.0 + math.erf(t / math.sqrt(2.0))) for t in z])
    assert np.allclose(M.gelu(z), expect, rtol=1e-15, atol=1e-300)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


def test_heads_loss_and_gradient():
    rng = np.random.default_rng(1)
    heads = (3, 4, 2)
    L = rng.standard_normal((5, 9)) * 3
    y = np.stack([rng.integers(0, n, 5) for n in heads], axis=1)
    loss, g = M.heads_loss(L, y, heads)
    ref, off = 0.0, 0
    for h, n in enumerate(heads):
        z = L[:, off:off + n]
        ref += np.sum(logsumexp(z, axis=1) - z[np.arange(5), y[:, h]])
        off += n
    assert np.isclose(loss, ref / 5, rtol=1e-14)
    h = 1e-6
    for (i, j) in [(0, 0), (2, 5), (4, 8), (3, 3)]:
        Lp, Lm = L.copy(), L.copy()
        Lp[i, j] += h
        Lm[i, j] -= h
        fd = (M.heads_loss(Lp, y, heads)[0] - M.heads_loss(Lm, y, heads)[0]) / (2 * h)
        assert abs(fd - g[i, j]) < 1e-8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    heads = (8, 8, 4)
    n_out = sum(heads)
    P = M.param_count(n_out)
    params = rng.standard_normal(P) * 0.05
    X = rng.standard_normal((6, M.N_IN))
    y = np.stack([rng.integers(0, n, 6) for n in heads], axis=1)
    loss, g = M.backward(params, X, y, heads, use_bf16=False)
    h = 1e-6
    for idx in rng.choice(P, 24, replace=False).tolist() + [P - 1, 0, 64 * 256 + 3]:
        pp, pm = params.copy(), params.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (M.backward(pp, X, y, heads, False)[0] - M.backward(pm, X, y, heads, False)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(g[idx])), (idx, fd, g[idx])


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    # after one step m_hat = g and v_hat = g^2: the update is lr * g / (|g| + eps)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_features_closed_forms():
    k = 400
    t = np.arange(k)
    # whole periods of sin(w t): the k - 1 squared first differences sum to
    # 2 k sin^2(w/2) - sin^2(w) (a full period minus the wrap-around term), the mean square is
    # 1/2, and mean(q^4) / mean(q^2)^2 = 3/2, so the kurtosis feature is 0
    ws = [2 * np.pi * m / k for m in (1, 2, 5, 10)]
    Qh = np.stack([np.sin(w * t) for w in ws])
    lam = np.array([8.0, 4.0, 2.0, 1.0])
    f = M.features(lam, 20.0, Qh, k)
    assert np.allclose(f[0:3], np.log10([0.5, 0.25, 0.125]))
    assert np.all(f[3:32] == -30.0)
    assert np.isclose(f[32], math.log10(1 - 15.0 / 20.0))     # r = 5 takes the 4 available
    for j, w in enumerate(ws):
        ms_diff = (2 * k * math.sin(w / 2) ** 2 - math.sin(w) ** 2) / (k - 1)
        assert np.isclose(f[36 + j], math.log10(math.sqrt(ms_diff / 0.5)), atol=1e-12)
        assert abs(f[52 + j]) < 1e-12
    assert np.all(f[36 + 4:52] == 0) and np.all(f[52 + 4:63] == 0)
    assert f[63] == math.log10(k)


def test_feature_stats_and_standardise_by_hand():
    X = np.array([[1.0, 10.0], [3.0, 10.0], [5.0, 10.0]])
    mu, sd = M.feature_stats(X)
    assert mu.tolist() == [3.0, 10.0]
    assert sd.tolist() == [2.0, 1e-6]           # sample std (ddof = 1); a constant feature is floored
    Xs = M.standardise(X, mu, sd)
    assert Xs.dtype == np.float32 and Xs[:, 0].tolist() == [-1.0, 0.0, 1.0] and Xs[:, 1].tolist() == [0.0] * 3


def test_rank_candidates_by_hand():
    """Heads of sizes (2, 2, 1): joint log-probabilities are sums of the per-head log-softmaxes;
    equal joint scores keep the lowest flat index first."""
    logits = np.array([[0.0, np.log(3.0), 0.0, 0.0, 5.0]])   # p1 = (1/4, 3/4), p2 = (1/2, 1/2), p3 = (1)
    idx, sc = M.rank_candidates(logits, (2, 2, 1), 4)
    assert idx[0].tolist() == [[1, 0, 0], [1, 1, 0], [0, 0, 0], [0, 1, 0]]
    assert np.allclose(np.exp(sc[0]), [3 / 8, 3 / 8, 1 / 8, 1 / 8], rtol=1e-14)
    # the joint distribution sums to one over every candidate
    idx, sc = M.rank_candidates(np.random.default_rng(0).standard_normal((3, 9)), (3, 4, 2), 24)
    assert np.allclose(np.exp(sc).sum(axis=1), 1.0, rtol=1e-12)
