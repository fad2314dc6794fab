"""Step V (lifting the reduced solution at chosen rows, inverse transform) through the C ABI
against the oracle's lift on the same inputs (the GPU's transformed snapshots, T_r and reduced
trajectory).  Both sides are FP64 sums over k snapshots and r modes in different orders:
per row, |dX| <= 4 (k + r) eps (|Q_row| |T_r| |Qtilde| scale), checked normwise as 1e-12
relative to the row's lifted values plus that absolute bound."""
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


def _setup(dp, dtype="f64", n_per=2048, k=200, r=6, seed=1234):
    w = synth.Workload("lift", 2, n_per, k, 6, var_scales=(1e-2, 1e3), dtype=dtype, seed=seed)
    Qn, _ = synth.snapshots_numpy(w)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    Q = torch.from_numpy(np.ascontiguousarray(Qn.T)).to(tdt).cuda().t()
    mean, scale, _ = dp.dopinf_transform(Q, w.var_row_offsets())
    D = dp.dopinf_gram(Q)
    red = dp.dopinf_reduce(D, r_cap=r, r_fixed=r)
    return w, Qn, Q, mean, scale, red


def _check(X, ref, Qh, Tr, Qt, rows, scale_rows):
    k, r = Tr.shape
    bound = 4 * (k + r) * EPS * (np.abs(Qh[rows]).sum(axis=1) * np.abs(Tr).max() * np.abs(Qt).sum(axis=0).max()
                                 * scale_rows)
    err = np.abs(X - ref).max(axis=1)
    assert np.all(err <= 1e-12 * np.abs(ref).max(axis=1) + bound), (err, bound)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_lift_probes_of_a_rollout_vs_oracle(dp, dtype):
    """The paper's use: a rollout of the learned ROM, lifted at three probe rows of each
    variable and returned to the original coordinates."""
    w, Qn, Q, mean, scale, red = _setup(dp, dtype)
    r = 6
    b = synth.logspace(-6, 0, 3)
    res = dp.dopinf_learn(red["Qhat"], [r], b, b, 400)
    assert res["best"] >= 0
    traj, fin = dp.dopinf_rollout(res["O"], red["Qhat"][:, 0].contiguous(), 400)
    assert int(fin.item()) == 1
    rows = torch.tensor([17, 1500, 2047, 2048, 3000, 4095], dtype=torch.int64)
    X = dp.dopinf_lift(Q, red["Tr"], traj.t(), rows=rows, row_mean=mean, var_scale=scale,
                       var_row_offsets=w.var_row_offsets()).cpu().numpy()
    Qh = Q.cpu().numpy().astype(np.float64)
    Tr, Qt = red["Tr"].cpu().numpy(), traj.cpu().numpy().T
    ref = O.lift(Qh, Tr, Qt, rows.numpy(), mean.cpu().numpy(), scale.cpu().numpy(), w.var_row_offsets())
    sc = scale.cpu().numpy()[np.searchsorted(w.var_row_offsets(), rows.numpy(), side="right") - 1]
    _check(X, ref, Qh, Tr, Qt, rows.numpy(), sc)


def test_lift_every_row_recovers_the_snapshots(dp):
    """All rows, the reduced coordinates of the training data themselves, r = every mode with a
    non-negligible eigenvalue: the lift returns the raw snapshots (V_r V_r^T Q = Q on the data's
    range), up to the noise the truncated modes carry."""
    w, Qn, Q, mean, scale, red = _setup(dp, r=6)
    X = dp.dopinf_lift(Q, red["Tr"], red["Qhat"], row_mean=mean, var_scale=scale,
                       var_row_offsets=w.var_row_offsets()).cpu().numpy()
    assert X.shape == Qn.shape
    # the synthetic data are rank 6 plus noise of 1e-4 of the RMS entry: the lift keeps 6 modes
    rel = np.linalg.norm(X - Qn) / np.linalg.norm(Qn)
    assert rel < 5e-4, rel
    # and equals the oracle's lift of the same inputs
    Qh = Q.cpu().numpy()
    ref = O.lift(Qh, red["Tr"].cpu().numpy(), red["Qhat"].cpu().numpy(), np.arange(Qh.shape[0]),
                 mean.cpu().numpy(), scale.cpu().numpy(), w.var_row_offsets())
    assert np.max(np.abs(X - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_lift_without_inverse_transform_and_bad_rows(dp):
    """No mean, no scale: the lifted transformed coordinates; a row index outside [0, n) gives
    a NaN row and touches nothing else."""
    w, Qn, Q, mean, scale, red = _setup(dp)
    rows = torch.tensor([5, -1, 4096, 100], dtype=torch.int64)
    X = dp.dopinf_lift(Q, red["Tr"], red["Qhat"][:, :50], rows=rows).cpu().numpy()
    Qh = Q.cpu().numpy()
    ref = O.lift(Qh, red["Tr"].cpu().numpy(), red["Qhat"].cpu().numpy()[:, :50], [5, 100])
    assert np.all(np.isnan(X[1])) and np.all(np.isnan(X[2]))
    assert np.max(np.abs(X[[0, 3]] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_lift_many_rows_ragged_tiles(dp):
    """Row counts and mode counts that leave partial tiles (rows not a multiple of 128, r not a
    multiple of 8, k not a multiple of 64)."""
    w, Qn, Q, mean, scale, red = _setup(dp, n_per=3001, k=131, r=11, seed=99)
    n = Q.shape[0]
    rng = np.random.default_rng(4)
    rows = torch.from_numpy(rng.choice(n, 777, replace=False).astype(np.int64))
    Qt = torch.from_numpy(rng.standard_normal((37, 11))).cuda().t()   # 11 x 37, column-major
    X = dp.dopinf_lift(Q, red["Tr"], Qt, rows=rows, row_mean=mean, var_scale=scale,
                       var_row_offsets=w.var_row_offsets()).cpu().numpy()
    Qh = Q.cpu().numpy()
    ref = O.lift(Qh, red["Tr"].cpu().numpy(), Qt.cpu().numpy(), rows.numpy(), mean.cpu().numpy(),
                 scale.cpu().numpy(), w.var_row_offsets())
    sc = scale.cpu().numpy()[np.searchsorted(w.var_row_offsets(), rows.numpy(), side="right") - 1]
    _check(X, ref, Qh, red["Tr"].cpu().numpy(), Qt.cpu().numpy(), rows.numpy(), sc)
