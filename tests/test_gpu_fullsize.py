"""Parity at the benchmark's full size (2D step-flow shape: n = 1.2M rows, k = 600,
r in {10, 20, 30}, 8 x 8 grid, 5000-step RK4), in the launch configuration bench.py times
(FP64-accurate digit-product Gram on the tensor cores, cluster rollouts),
on outputs the FP64 oracle can compute one by one: sampled rows of the transform, sampled
Gram entries, the whole k x k eigenproblem, and a sample of the learn candidates."""
import numpy as np
import pytest
import torch

from oracle import dopinf_oracle as O
from paper_2504_14338_gb300 import synth

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2504_14338_gb300 import dopinf as dp
    w = synth.WORKLOADS["stepflow"]
    QT = synth.snapshots_torch(w, torch.device("cuda"))
    Q = QT.t()
    rng = np.random.default_rng(0)
    npv = w.n_per_var
    rows = np.unique(np.concatenate([rng.choice(w.n, 3000, replace=False),
                                     [0, npv - 1, npv, 2 * npv - 1, 2 * npv, w.n - 1]]))
    raw = Q[torch.from_numpy(rows).cuda()].cpu().numpy()
    ws = dp.Workspace("cuda")
    mean, scale, flags = dp.dopinf_transform(Q, w.var_row_offsets(), ws=ws)
    D = dp.dopinf_gram(Q, mode=dp.GRAM_OZAKI_FP64, ws=ws)   # the Gram mode bench.py times
    red = dp.dopinf_reduce(D, r_cap=max(w.r_list), r_fixed=max(w.r_list), ws=ws)
    b1, b2 = w.beta1s(), w.beta2s()
    res = dp.dopinf_learn(red["Qhat"], list(w.r_list), b1, b2, w.n_steps, mode=dp.CONTINUOUS_RK4,
                          dt=w.snap_dt, ws=ws)
    torch.cuda.synchronize()
    return dict(dp=dp, w=w, Q=Q, rows=rows, raw=raw, mean=mean, scale=scale, flags=flags, D=D, red=red,
                res=res, b1=b1, b2=b2)


def test_transform_sampled_rows_bit_exact(run):
    w, rows, raw = run["w"], run["rows"], run["raw"]
    _, rmean, _, _ = O.transform(raw, [0, len(rows)], scale=False)
    assert np.array_equal(run["mean"].cpu().numpy()[rows], rmean)
    scale = run["scale"].cpu().numpy()
    var = rows // w.n_per_var
    centred, _, _, _ = O.transform(raw, [0, len(rows)], scale=False)
    expect = centred / scale[var][:, None]
    got = run["Q"][torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(got, expect)
    # the scale is the block's max |centred value|: every block then peaks at exactly 1
    Q = run["Q"]
    for j in range(w.n_vars):
        blk = Q[j * w.n_per_var:(j + 1) * w.n_per_var]
        assert float(blk.abs().max()) == 1.0
    assert int(run["flags"].item()) == 0


def test_gram_sampled_entries(run):
    w, Q, D = run["w"], run["Q"], run["D"].cpu().numpy()
    rng = np.random.default_rng(1)
    cols = np.unique(np.concatenate([rng.choice(w.k, 24, replace=False), [0, 63, 64, w.k - 1]]))
    Qc = Q[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    ref = O.gram(Qc)
    got = D[np.ix_(cols, cols)]
    bound = 4 * np.sqrt(w.n) * EPS * np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(got - ref) <= bound)
    assert np.array_equal(D, D.T)


def test_reduce_full_eigenproblem(run):
    """The whole 600 x 600 eigenproblem: 1e-10 relative for the eigenvalues above 1e-3 lambda_1
    and for the Qhat rows whose eigen-gap makes them well determined (eps lambda_1 / gap <=
    1e-12); the magnitude- or gap-limited ones against the FP64 backward-error bounds."""
    from test_gpu_parity import assert_eigen_qhat
    w, D, red = run["w"], run["D"].cpu().numpy(), run["red"]
    r = max(w.r_list)
    ref = O.reduce(D, r_fixed=r)
    limited = assert_eigen_qhat(red["eigvals"].cpu().numpy(), ref["lam"], red["Qhat"].cpu().numpy(), ref["Qhat"],
                                w.k, r)
    assert len(limited["gap_limited_qhat_rows"]) <= r // 2


def test_learn_selected_candidate_and_sample(run):
    w, res, red = run["w"], run["res"], run["red"]
    st = res["status"].cpu().numpy()
    err = res["train_err"].cpu().numpy()
    gro = res["growth"].cpu().numpy()
    nb = len(run["b1"]) * len(run["b2"])
    best = res["best"]
    assert best >= 0 and st[best] == 0
    Qh = red["Qhat"].cpu().numpy()            # the GPU's reduced data: the learn step's input
    r = res["r"]
    Ob = res["O"].cpu().numpy()
    # (a) the selected operators, rolled out by the oracle: train error and growth to 1e-8
    Qr = Qh[:r].T
    traj = O.rollout(Ob, r, Qr[0], w.n_steps, mode="continuous", dt=w.snap_dt)
    mu = Qr.mean(axis=0)
    e_ref = O.train_error(Qr[:w.k], traj[:w.k])
    g_ref = O.growth_ratio(traj, mu, np.max(np.abs(Qr - mu), axis=0))
    assert abs(err[best] - e_ref) <= 1e-8 * e_ref, (err[best], e_ref)
    assert abs(gro[best] - g_ref) <= 1e-8 * g_ref, (gro[best], g_ref)
    # (b) the regularised normal equations are solved backward-stably
    Dh, Y = O.learning_data(Qh, r, mode="continuous", dt=w.snap_dt)
    G, B = O.normal_equations(Dh, Y)
    M = G + np.diag(O.regulariser(r, res["beta1"], res["beta2"]))
    resid = np.linalg.norm(M @ Ob.T - B) / (np.linalg.norm(M) * np.linalg.norm(Ob))
    assert resid <= 50 * M.shape[0] * EPS, resid
    # (c) sampled candidates: the oracle's grid search on the same reduced data; the
    # tolerance follows the conditioning of G + reg (FP64 on both sides)
    rng = np.random.default_rng(2)
    sample = sorted(set(rng.choice(len(st), 5, replace=False).tolist()))
    for c in sample:
        rc = w.r_list[c // nb]
        b1 = run["b1"][(c % nb) // len(run["b2"])]
        b2 = run["b2"][c % len(run["b2"])]
        ref = O.learn(Qh, [rc], [b1], [b2], w.n_steps, mode="continuous", dt=w.snap_dt)
        Dh, Y = O.learning_data(Qh, rc, mode="continuous", dt=w.snap_dt)
        G, _ = O.normal_equations(Dh, Y)
        cond = np.linalg.cond(G + np.diag(O.regulariser(rc, b1, b2)))
        tol = 1e-8 + 100 * cond * EPS
        if tol > 1e-3:
            continue
        assert ref["valid"][0] == (st[c] == 0), (c, st[c], ref["growth"][0])
        if st[c] == 0:
            assert abs(err[c] - ref["train_err"][0]) <= tol * ref["train_err"][0], (c, err[c], ref["train_err"][0])


def test_lift_of_the_selected_rollout_at_sampled_rows(run):
    """Step V at full size: the selected ROM's 5000-step rollout lifted at the 3006 sampled rows
    (the paper lifts at probe rows) against the oracle's lift of the same inputs."""
    from oracle import dopinf_oracle as Or
    dp, w, res, red, Q, rows = run["dp"], run["w"], run["res"], run["red"], run["Q"], run["rows"]
    r = res["r"]
    traj, fin = dp.dopinf_rollout(res["O"], red["Qhat"][:r, 0].contiguous(), w.n_steps, mode=dp.CONTINUOUS_RK4,
                                  dt=w.snap_dt)
    assert int(fin.item()) == 1
    Tr = red["Tr"][:, :r]
    X = dp.dopinf_lift(Q, Tr, traj.t(), rows=torch.from_numpy(rows), row_mean=run["mean"], var_scale=run["scale"],
                       var_row_offsets=w.var_row_offsets()).cpu().numpy()
    Qs = Q[torch.from_numpy(rows).cuda()].cpu().numpy()
    sc = run["scale"].cpu().numpy()[rows // w.n_per_var]
    ref = Or.lift(Qs, Tr.cpu().numpy(), traj.cpu().numpy().T, np.arange(len(rows))) * sc[:, None] \
        + run["mean"].cpu().numpy()[rows][:, None]
    err = np.abs(X - ref).max(axis=1)
    assert np.all(err <= 1e-11 * np.abs(ref).max(axis=1) + 1e-12 * sc), err.max()
