"""FP64 CPU oracle of the learned (beta1, beta2, r) proposal network.

TEST INFRASTRUCTURE ONLY (same rules as dopinf_oracle): only tests, smoke() and the bench's
CPU-baseline leg use it; it shares no code with the CUDA library.

The paper selects (beta1, beta2) by an exhaustive grid search (Section 3.5) and r by the
retained energy (Section 3.4).  The proposal network predicts those choices from spectral and
temporal statistics of the reduced data; the grid search remains its fallback and its judge.
The paper has no network of its own; the definitions below are this project's.

Network: x (64) -> Linear(64, 256) -> GELU -> Linear(256, 256) -> GELU -> Linear(256, 256) ->
GELU -> Linear(256, H), H = n_b1 + n_b2 + n_r.  The logits split into three heads (beta1 grid
index, beta2 grid index, r candidate index); the loss is the mean over the batch of the sum
of the three softmax cross-entropies.  Weights are kept in FP32 and rounded to BF16
(round-to-nearest-even) where they are used; GELU is the exact erf form.  Parameters are
stored flat: W1 (256 x 64, row-major), b1, W2 (256 x 256), b2, W3, b3, W4 (H x 256), b4.

Features (64), from the descending eigenvalues lambda of the Gram matrix, its trace and the
reduced data Qhat (modes x time):
  f[0:32]   log10(max(lambda_i / lambda_1, 1e-30)), i = 2..33 (-30 where lambda_i is missing)
  f[32:36]  log10(max(1 - sum_{i<=r} lambda_i / trace, 1e-30)) for r = 5, 10, 20, 30
  f[36:52]  log10(rms_t(q_j[t+1] - q_j[t]) / rms_t(q_j[t])) for modes j = 0..15 (0 if missing)
  f[52:63]  mean_t(q_j^4) / mean_t(q_j^2)^2 - 1.5 for modes j = 0..10 (0 if missing)
  f[63]     log10(k)
"""
import math

import numpy as np
from scipy.special import erf

N_IN = 64
HIDDEN = 256


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    x32 = np.asarray(x, dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return rounded.view(np.float32).astype(np.float64)


def layer_shapes(n_out, n_in=N_IN, hidden=HIDDEN):
    return [(hidden, n_in), (hidden, hidden), (hidden, hidden), (n_out, hidden)]


def param_count(n_out, n_in=N_IN, hidden=HIDDEN):
    return sum(o * i + o for o, i in layer_shapes(n_out, n_in, hidden))


def unpack(params, n_out, n_in=N_IN, hidden=HIDDEN):
    """List of (W, b) views into the flat parameter vector."""
    out, off = [], 0
    for o, i in layer_shapes(n_out, n_in, hidden):
        W = params[off:off + o * i].reshape(o, i)
        off += o * i
        b = params[off:off + o]
        off += o
        out.append((W, b))
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X, n_out, use_bf16=True):
    """Returns (logits, cache) for a batch X (B x 64)."""
    layers = unpack(np.asarray(params, dtype=np.float64), n_out)
    a = np.asarray(X, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(layers):
        Wq = bf16_round(W) if use_bf16 else W
        z = a @ Wq.T + b
        cache.append((a, z, Wq))
        a = gelu(z) if li < len(layers) - 1 else z
    return a, cache


def heads_loss(logits, labels, head_sizes):
    """Mean over the batch of the sum of per-head softmax cross-entropies, and d loss/d logits."""
    B = logits.shape[0]
    loss = 0.0
    grad = np.zeros_like(logits)
    off = 0
    for h, n in enumerate(head_sizes):
        z = logits[:, off:off + n]
        zmax = z.max(axis=1, keepdims=True)
        lse = zmax[:, 0] + np.log(np.exp(z - zmax).sum(axis=1))
        y = labels[:, h]
        loss += np.sum(lse - z[np.arange(B), y])
        p = np.exp(z - lse[:, None])
        p[np.arange(B), y] -= 1.0
        grad[:, off:off + n] = p / B
        off += n
    return loss / B, grad


def backward(params, X, labels, head_sizes, use_bf16=True):
    """(loss, flat gradient) of heads_loss(forward(params, X)); the gradient of a BF16-rounded
    weight is applied to its FP32 master copy."""
    n_out = sum(head_sizes)
    logits, cache = forward(params, X, n_out, use_bf16)
    loss, g = heads_loss(logits, labels, head_sizes)
    grads = []
    for li in range(len(cache) - 1, -1, -1):
        a, z, Wq = cache[li]
        if li < len(cache) - 1:
            g = g * gelu_grad(z)
        grads.append((g.T @ a, g.sum(axis=0)))
        g = g @ Wq
    grads.reverse()
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat


def adam_step(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def features(eigvals, trace, Qhat, k):
    """The 64 input features of one reduced system (see the module docstring)."""
    lam = np.asarray(eigvals, dtype=np.float64)
    Qh = np.asarray(Qhat, dtype=np.float64)
    f = np.zeros(N_IN)
    for i in range(32):
        j = i + 1
        f[i] = math.log10(max(lam[j] / lam[0], 1e-30)) if j < len(lam) else -30.0
    for c, r in enumerate((5, 10, 20, 30)):
        cum = float(np.sum(lam[:min(r, len(lam))]))
        f[32 + c] = math.log10(max(1.0 - cum / trace, 1e-30))
    for j in range(16):
        if j < Qh.shape[0]:
            q = Qh[j]
            f[36 + j] = math.log10(math.sqrt(np.mean(np.diff(q) ** 2)) / math.sqrt(np.mean(q * q)))
    for j in range(11):
        if j < Qh.shape[0]:
            q = Qh[j]
            m2 = np.mean(q * q)
            f[52 + j] = np.mean(q ** 4) / (m2 * m2) - 1.5
    f[63] = math.log10(k)
    return f


# --------------------------------------------------------------------------------------
# Input standardisation and the ranking of grid candidates by the network's joint probability.
# --------------------------------------------------------------------------------------
def feature_stats(X, sd_floor=1e-6):
    """Per-feature mean and sample standard deviation (ddof = 1, floored) of a training set."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = np.maximum(X.std(axis=0, ddof=1), sd_floor) if X.shape[0] > 1 else np.full(X.shape[1], sd_floor)
    return mu, sd


def standardise(X, mu, sd):
    """(x - mu) / sd per feature, in FP64, rounded to FP32 (the network's input type)."""
    return ((np.asarray(X, dtype=np.float64) - mu) / sd).astype(np.float32)


def log_softmax(z):
    z = np.asarray(z, dtype=np.float64)
    m = z.max(axis=-1, keepdims=True)
    return z - (m + np.log(np.exp(z - m).sum(axis=-1, keepdims=True)))


def rank_candidates(logits, heads, top):
    """The `top` grid candidates (i1, i2, i3) of each row in decreasing joint log-probability
    log p1(i1) + log p2(i2) + log p3(i3) (the three heads' softmaxes), ties to the lowest flat
    index (i1 h2 + i2) h3 + i3.  Returns (indices (B, top, 3), scores (B, top))."""
    L = np.asarray(logits, dtype=np.float64)
    h1, h2, h3 = heads
    lp1, lp2, lp3 = log_softmax(L[:, :h1]), log_softmax(L[:, h1:h1 + h2]), log_softmax(L[:, h1 + h2:h1 + h2 + h3])
    idx = np.zeros((L.shape[0], top, 3), dtype=np.int64)
    sc = np.zeros((L.shape[0], top))
    for b in range(L.shape[0]):
        joint = (lp1[b][:, None, None] + lp2[b][None, :, None] + lp3[b][None, None, :]).reshape(-1)
        order = sorted(range(joint.size), key=lambda c: (-joint[c], c))[:top]
        for t, c in enumerate(order):
            idx[b, t] = (c // (h2 * h3), (c // h3) % h2, c % h3)
            sc[b, t] = joint[c]
    return idx, sc
