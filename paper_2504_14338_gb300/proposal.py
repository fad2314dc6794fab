"""Learned proposal of (beta1, beta2, r), trained on grid-search outcomes of seeded systems.

Each seeded system (a synthetic quadratic system of dimension r_true lifted to n rows) goes
through Steps II-III on the GPU on its training window of k snapshots; its 64 features come from
the eigenvalues and the reduced data, its label is the (beta1 index, beta2 index, r index) the
full grid search of Step IV selects.  The network is trained with the library's own
forward/backward/Adam kernels on inputs standardised by the library (the training set's
statistics).  At use, the library ranks the grid candidates by the network's joint probability;
the most probable is verified by a single-candidate learn step (one Cholesky solve and one
rollout); if that candidate is not valid the next ones are tried and, as the last resort, the
full grid search runs.

The judge of a selection is its validation error: the selected ROM is rolled out past the
training window over a held-out continuation of the true trajectory (val_frac * k further
snapshots), lifted to the transformed snapshot coordinates with Step V, and compared with the
held-out snapshots transformed with the training window's mean and scale: the largest relative
2-norm error over the held-out instants.  Every step of the method runs in the CUDA library; the
validation error's final norms are evaluation arithmetic on the lifted states.

Systems are generated by worker processes (spawned: they touch no GPU), so large training sets
do not wait on the host.  `python -m paper_2504_14338_gb300.proposal --train N --eval M` runs the
whole experiment and prints one JSON line.
"""
import argparse
import json
import multiprocessing as mp
import os
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
    steps_factor: int = 2      # grid-search rollout length = steps_factor * k
    val_frac: float = 0.25     # held-out continuation: val_frac * k snapshots after the training window
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
    """(workload with k_train + k_val snapshots, k_train) of one seeded system."""
    rng = np.random.default_rng(seed)
    r_true = int(rng.integers(spec.r_true_range[0], spec.r_true_range[1] + 1))
    k = int(rng.integers(spec.k_range[0], spec.k_range[1] + 1))
    k_val = max(1, int(round(spec.val_frac * k)))
    return synth.Workload("proposal", 2, spec.n_per_var, k + k_val, r_true, seed=seed), k


def _generate(args):
    spec, seed = args
    w, k = system(spec, seed)
    Qn, _ = synth.snapshots_numpy(w)
    return seed, w, k, np.asarray(Qn)


def generated(spec, seeds, workers=None):
    """Yields (seed, workload, k_train, snapshots (n, k_train + k_val)) in seed order, made by a pool
    of spawned worker processes (started before any of them is consumed)."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    seeds = list(seeds)
    if workers == 1 or len(seeds) < 4:
        for s in seeds:
            yield _generate((spec, s))
        return
    with mp.get_context("spawn").Pool(workers) as pool:
        for item in pool.imap(_generate, [(spec, s) for s in seeds], chunksize=2):
            yield item


def reduced(spec, w, k, Qn, ws, device="cuda"):
    """Steps II-III of one system's training window on the GPU.  Returns a dict: eigvals, trace,
    Qhat, Tr, the transformed training snapshots Q and the transform's mean and scale."""
    Q = dp.snapshot_matrix(w.n, k, device=device)
    Q.copy_(torch.from_numpy(np.ascontiguousarray(Qn[:, :k])))
    mean, scale, _ = dp.dopinf_transform(Q, w.var_row_offsets(), ws=ws)
    D = dp.dopinf_gram(Q, ws=ws)
    r_cap = min(max(spec.r_cap, max(spec.r_list)), k - 1)  # the grid's largest r needs its rows of Qhat
    red = dp.dopinf_reduce(D, r_cap=r_cap, r_fixed=r_cap, ws=ws)
    return dict(eigvals=red["eigvals"], trace=red["trace"], Qhat=red["Qhat"], Tr=red["Tr"], Q=Q, mean=mean,
                scale=scale)


def grid_search(spec, Qhat, k, ws):
    return dp.dopinf_learn(Qhat, list(spec.r_list), spec.beta1s(), spec.beta2s(), spec.steps_factor * k,
                           mode=spec.mode, dt=1.0, ws=ws)


def dataset(spec, seeds, ws, workers=None):
    """Features (N x 64, device) and labels (N x 3, device) of the systems with a valid grid optimum."""
    feats, labels, kept = [], [], []
    nb = spec.n_b1 * spec.n_b2
    for s, w, k, Qn in generated(spec, seeds, workers):
        red = reduced(spec, w, k, Qn, ws)
        res = grid_search(spec, red["Qhat"], k, ws)
        if res["best"] < 0:
            continue
        b = res["best"]
        labels.append([(b % nb) // spec.n_b2, b % spec.n_b2, b // nb])
        feats.append(dp.dopinf_proposal_features(red["eigvals"], red["trace"], red["Qhat"]))
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


def train(spec, X, y, steps=1500, batch=64, lr=1e-3, seed=0):
    """Adam on the GPU (library kernels); inputs standardised by the library with the training
    set's statistics."""
    mu, sd = dp.dopinf_mlp_feature_stats(X)
    Xs = dp.dopinf_mlp_standardize(X, mu, sd)
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
    """The `top` most probable (i1, i2, ir) grid candidates for each row of feats (ranked by the
    library)."""
    n_out = sum(spec.heads)
    logits = dp.dopinf_mlp_forward(model["params"], n_out, dp.dopinf_mlp_standardize(feats, model["mu"], model["sd"]))
    ranked, _ = dp.dopinf_mlp_rank(logits, spec.heads, top)
    return [[tuple(int(x) for x in c) for c in row if c[0] >= 0] for row in ranked.cpu().numpy()]


def validation_error(spec, w, k, Qn, red, O, r, ws):
    """Largest relative 2-norm error, over the held-out instants k .. k_total - 1, between the ROM
    (operators O of dimension r) rolled out from the training window's first reduced state and
    lifted with Step V, and the held-out snapshots transformed with the training statistics."""
    k_tot = w.k
    traj, fin = dp.dopinf_rollout(O, red["Qhat"][:r, 0].contiguous(), k_tot, mode=spec.mode, dt=1.0)
    if int(fin.item()) != 1:
        return float("inf")
    X = dp.dopinf_lift(red["Q"], red["Tr"][:, :r], traj[k:].t(), ws=ws)        # n x k_val, transformed
    S = torch.from_numpy(np.ascontiguousarray(Qn[:, k:])).to(X.device)
    var = torch.from_numpy(np.repeat(np.arange(w.n_vars), w.n_per_var)).to(X.device)
    S = (S - red["mean"][:, None]) / red["scale"][var][:, None]
    err = torch.linalg.vector_norm(X - S, dim=0) / torch.linalg.vector_norm(S, dim=0)
    return float(err.max().item())


def _learn_one(spec, Qh, r, b1, b2, k, ws):
    return dp.dopinf_learn(Qh, [r], [b1], [b2], spec.steps_factor * k, mode=spec.mode, dt=1.0, ws=ws)


def evaluate(spec, model, seeds, ws, top=3, workers=None):
    """Proposal-with-fallback against the full grid search on held-out systems: the ratio of the
    validation errors of the two selections, their training-error ratio, and the time and the
    candidate evaluations each needs."""
    b1, b2 = spec.beta1s(), spec.beta2s()
    n_grid = len(spec.r_list) * spec.n_b1 * spec.n_b2
    rows = []
    for s, w, k, Qn in generated(spec, seeds, workers):
        red = reduced(spec, w, k, Qn, ws)
        Qh = red["Qhat"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grid = grid_search(spec, Qh, k, ws)
        torch.cuda.synchronize()
        t_grid = time.perf_counter() - t0
        if grid["best"] < 0:
            continue
        t0 = time.perf_counter()
        f = dp.dopinf_proposal_features(red["eigvals"], red["trace"], Qh)
        cands = propose(spec, model, f[None, :], top)[0]
        chosen, tries, fallback = None, 0, False
        for (i1, i2, ir) in cands:
            tries += 1
            res = _learn_one(spec, Qh, spec.r_list[ir], b1[i1], b2[i2], k, ws)
            if res["best"] >= 0:
                chosen = res
                break
        if chosen is None:
            fallback = True
            chosen = grid_search(spec, Qh, k, ws)
        torch.cuda.synchronize()
        t_prop = time.perf_counter() - t0
        pick = chosen["best"]
        e_prop = float(chosen["train_err"][pick].item())
        e_grid = float(grid["train_err"][grid["best"]].item())
        v_prop = validation_error(spec, w, k, Qn, red, chosen["O"], chosen["r"], ws)
        v_grid = validation_error(spec, w, k, Qn, red, grid["O"], grid["r"], ws)
        rows.append(dict(seed=s, ratio=e_prop / e_grid, val_ratio=v_prop / v_grid, val_prop=v_prop, val_grid=v_grid,
                         tries=tries, fallback=fallback, t_grid=t_grid, t_prop=t_prop,
                         evals=tries + (n_grid if fallback else 0)))
    ratios = np.array([r["ratio"] for r in rows])
    vr = np.array([r["val_ratio"] for r in rows])
    return dict(n=len(rows), median_error_ratio=float(np.median(ratios)),
                median_validation_error_ratio=float(np.median(vr[np.isfinite(vr)])) if np.isfinite(vr).any() else None,
                validation_within_1p5=float(np.mean(vr <= 1.5)),
                within_1p5=float(np.mean(ratios <= 1.5)), fallback_rate=float(np.mean([r["fallback"] for r in rows])),
                top1_valid=float(np.mean([r["tries"] == 1 and not r["fallback"] for r in rows])),
                speedup=float(np.sum([r["t_grid"] for r in rows]) / np.sum([r["t_prop"] for r in rows])),
                work_ratio=float(n_grid / np.mean([r["evals"] for r in rows])),
                rows=rows)


def experiment(spec, n_train, n_eval, steps=1500, workers=None, seed0=0, eval_seed0=1_000_000):
    """Train on n_train seeded systems, evaluate on n_eval held-out ones, against the untrained
    network too; returns a summary dict."""
    ws = dp.Workspace("cuda")
    t0 = time.perf_counter()
    X, y, kept = dataset(spec, range(seed0, seed0 + n_train), ws, workers)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    model = train(spec, X, y, steps=steps)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    seeds = range(eval_seed0, eval_seed0 + n_eval)
    res = evaluate(spec, model, seeds, ws, workers=workers)
    base = evaluate(spec, train(spec, X, y, steps=1, lr=0.0), seeds, ws, workers=workers)
    strip = lambda d: {k: v for k, v in d.items() if k != "rows"}
    return dict(spec=dict(r_list=list(spec.r_list), grid=[spec.n_b1, spec.n_b2], r_true_range=list(spec.r_true_range),
                          k_range=list(spec.k_range), n_per_var=spec.n_per_var, val_frac=spec.val_frac,
                          steps_factor=spec.steps_factor),
                n_train=n_train, n_labelled=int(X.shape[0]), n_eval=n_eval, labelling_s=t_data, training_s=t_train,
                final_loss=model["losses"][-1], trained=strip(res), untrained=strip(base))


def main():
    p = argparse.ArgumentParser(description="learned (beta1, beta2, r) proposal: train and evaluate")
    p.add_argument("--train", type=int, default=1000)
    p.add_argument("--eval", type=int, default=200)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--r-true", default="5,30")
    p.add_argument("--k", default="300,800")
    p.add_argument("--r-list", default="5,10,15,20,30")
    a = p.parse_args()
    lo, hi = (int(x) for x in a.r_true.split(","))
    klo, khi = (int(x) for x in a.k.split(","))
    spec = ProposalSpec(r_list=tuple(int(x) for x in a.r_list.split(",")), r_true_range=(lo, hi), k_range=(klo, khi))
    print(json.dumps(experiment(spec, a.train, a.eval, steps=a.steps)), flush=True)


if __name__ == "__main__":
    main()
