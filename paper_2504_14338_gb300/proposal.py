"""Learned proposal of (beta1, beta2, r), trained on grid-search outcomes of seeded systems.

Each seeded system (a synthetic quadratic system of dimension r_true lifted to n rows) goes
through Steps II-III on the GPU; its 64 features come from the eigenvalues and the reduced
data, its label is the (beta1 index, beta2 index, r index) the full grid search of Step IV
selects.  The network is trained with the library's own forward/backward/Adam kernels.  At
use, the proposal is verified by a single-candidate learn step (one Cholesky solve and one
rollout); if that candidate is not valid the next most probable candidates are tried and, as
the last resort, the full grid search runs.  Every step runs in the CUDA library.
"""
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import dopinf as dp
from . import synth


@dataclass
class ProposalSpec:
    r_list: tuple = (4, 8, 12, 16)
    n_b1: int = 8
    n_b2: int = 8
    beta1_range: tuple = (-10.0, 0.0)
    beta2_range: tuple = (-4.0, 4.0)
    r_true_range: tuple = (5, 30)
    k_range: tuple = (200, 400)
    n_per_var: int = 1000
    steps_factor: int = 2      # rollout length = steps_factor * k
    r_cap: int = 40            # eigenpairs computed (features use lambda_2..lambda_33)
    mode: int = dp.DISCRETE

    @property
    def heads(self):
        return (self.n_b1, self.n_b2, len(self.r_list))

    def beta1s(self):
        return synth.logspace(self.beta1_range[0], self.beta1_range[1], self.n_b1)

    def beta2s(self):
        return synth.logspace(self.beta2_range[0], self.beta2_range[1], self.n_b2)


def system(spec, seed):
    rng = np.random.default_rng(seed)
    r_true = int(rng.integers(spec.r_true_range[0], spec.r_true_range[1] + 1))
    k = int(rng.integers(spec.k_range[0], spec.k_range[1] + 1))
    return synth.Workload("proposal", 2, spec.n_per_var, k, r_true, seed=seed)


def reduced(spec, w, ws, device="cuda"):
    """Steps II-III of one system on the GPU: (eigvals, trace, Qhat)."""
    Qn, _ = synth.snapshots_numpy(w)
    Q = dp.snapshot_matrix(w.n, w.k, device=device)
    Q.copy_(torch.from_numpy(np.asarray(Qn)))
    dp.dopinf_transform(Q, w.var_row_offsets(), ws=ws)
    D = dp.dopinf_gram(Q, ws=ws)
    r_cap = min(spec.r_cap, w.k - 1)
    red = dp.dopinf_reduce(D, r_cap=r_cap, r_fixed=r_cap, ws=ws)
    return red["eigvals"], red["trace"], red["Qhat"]


def grid_search(spec, Qhat, k, ws):
    return dp.dopinf_learn(Qhat, list(spec.r_list), spec.beta1s(), spec.beta2s(), spec.steps_factor * k,
                           mode=spec.mode, dt=1.0, ws=ws)


def dataset(spec, seeds, ws):
    """Features (N x 64, device) and labels (N x 3, device) of the systems with a valid grid optimum."""
    feats, labels, kept = [], [], []
    nb = spec.n_b1 * spec.n_b2
    for s in seeds:
        w = system(spec, s)
        lam, tr, Qh = reduced(spec, w, ws)
        res = grid_search(spec, Qh, w.k, ws)
        if res["best"] < 0:
            continue
        b = res["best"]
        labels.append([(b % nb) // spec.n_b2, b % spec.n_b2, b // nb])
        feats.append(dp.dopinf_proposal_features(lam, tr, Qh))
        kept.append(s)
    X = torch.stack(feats)
    y = torch.tensor(labels, dtype=torch.int32, device=X.device)
    return X, y, kept


def init_params(n_out, seed=0, device="cuda"):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, small biases (seeded, host-drawn)."""
    rng = np.random.default_rng(seed)
    shapes = [(256, 64), (256, 256), (256, 256), (n_out, 256)]
    parts = []
    for o, i in shapes:
        parts.append(rng.uniform(-1, 1, o * i) / np.sqrt(i))
        parts.append(rng.uniform(-0.1, 0.1, o))
    return torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(device)


def _standardise(X, mu, sd):
    """Host-side input scaling of the (small) feature matrix."""
    Xh = X.cpu().numpy().astype(np.float64)
    return torch.from_numpy(((Xh - mu) / sd).astype(np.float32)).to(X.device).contiguous()


def train(spec, X, y, steps=1500, batch=64, lr=1e-3, seed=0):
    """Adam on the GPU (library kernels); inputs standardised with the training statistics."""
    Xh = X.cpu().numpy().astype(np.float64)
    mu = Xh.mean(axis=0)
    sd = np.maximum(Xh.std(axis=0, ddof=1), 1e-6)
    Xs = _standardise(X, mu, sd)
    n_out = sum(spec.heads)
    params = init_params(n_out, seed, X.device)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    N = Xs.shape[0]
    losses = []
    ws = dp.Workspace(X.device)
    for t in range(1, steps + 1):
        idx = torch.randint(0, N, (min(batch, N),), generator=g).to(X.device)
        loss, _ = dp.dopinf_mlp_train_step(params, m, v, t, lr, spec.heads, Xs[idx], y[idx], ws=ws)
        if t % 100 == 0 or t == 1:
            losses.append(float(loss.item()))
    return dict(params=params, mu=mu, sd=sd, losses=losses)


def propose(spec, model, feats, top=3):
    """The `top` most probable (i1, i2, ir) grid candidates for each row of feats."""
    n_out = sum(spec.heads)
    logits = dp.dopinf_mlp_forward(model["params"], n_out, _standardise(feats, model["mu"], model["sd"]))
    L = logits.cpu().numpy().astype(np.float64)   # a few numbers per system: ranked on the host
    h1, h2, h3 = spec.heads

    def logsoftmax(z):
        z = z - z.max(axis=1, keepdims=True)
        return z - np.log(np.exp(z).sum(axis=1, keepdims=True))
    lp1, lp2, lp3 = logsoftmax(L[:, :h1]), logsoftmax(L[:, h1:h1 + h2]), logsoftmax(L[:, h1 + h2:])
    joint = lp1[:, :, None, None] + lp2[:, None, :, None] + lp3[:, None, None, :]
    flat = joint.reshape(joint.shape[0], -1)
    best = np.argsort(-flat, axis=1, kind="stable")[:, :top]
    out = []
    for row in best:
        out.append([(int(c // (h2 * h3)), int((c // h3) % h2), int(c % h3)) for c in row])
    return out


def evaluate(spec, model, seeds, ws, top=3):
    """Proposal-with-fallback against the full grid search on held-out systems."""
    b1, b2 = spec.beta1s(), spec.beta2s()
    rows = []
    for s in seeds:
        w = system(spec, s)
        lam, tr, Qh = reduced(spec, w, ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grid = grid_search(spec, Qh, w.k, ws)
        torch.cuda.synchronize()
        t_grid = time.perf_counter() - t0
        if grid["best"] < 0:
            continue
        t0 = time.perf_counter()
        f = dp.dopinf_proposal_features(lam, tr, Qh)
        cands = propose(spec, model, f[None, :], top)[0]
        chosen, tries, fallback = None, 0, False
        for (i1, i2, ir) in cands:
            tries += 1
            res = dp.dopinf_learn(Qh, [spec.r_list[ir]], [b1[i1]], [b2[i2]], spec.steps_factor * w.k,
                                  mode=spec.mode, dt=1.0, ws=ws)
            if res["best"] >= 0:
                chosen = float(res["train_err"][0].item())
                break
        if chosen is None:
            fallback = True
            chosen = float(grid_search(spec, Qh, w.k, ws)["train_err"][grid["best"]].item())
        torch.cuda.synchronize()
        t_prop = time.perf_counter() - t0
        g_err = float(grid["train_err"][grid["best"]].item())
        n_grid = len(spec.r_list) * spec.n_b1 * spec.n_b2
        rows.append(dict(seed=s, ratio=chosen / g_err, tries=tries, fallback=fallback, t_grid=t_grid,
                         t_prop=t_prop, evals=tries + (n_grid if fallback else 0)))
    ratios = np.array([r["ratio"] for r in rows])
    return dict(n=len(rows), median_error_ratio=float(np.median(ratios)),
                within_1p5=float(np.mean(ratios <= 1.5)), fallback_rate=float(np.mean([r["fallback"] for r in rows])),
                top1_valid=float(np.mean([r["tries"] == 1 and not r["fallback"] for r in rows])),
                speedup=float(np.sum([r["t_grid"] for r in rows]) / np.sum([r["t_prop"] for r in rows])),
                work_ratio=float(len(spec.r_list) * spec.n_b1 * spec.n_b2 / np.mean([r["evals"] for r in rows])),
                rows=rows)
