"""The knobs the autotuner turns change where the work runs, not the results; the tuner picks
one of them from measurements and leaves it set."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2504_14338_gb300 import dopinf as dp
    from paper_2504_14338_gb300 import synth
    from oracle import dopinf_oracle as O
    w = synth.WORKLOADS["small"]
    Qn, _ = synth.snapshots_numpy(w)
    Q = O.transform(Qn, w.var_row_offsets())[0]
    D = O.gram(Q)
    Qh = O.reduce(D, r_fixed=16)["Qhat"]
    return dp, synth, w, torch.from_numpy(D).cuda(), torch.from_numpy(Qh.T.copy()).cuda().t()


@pytest.mark.parametrize("arith", ["dw", "fp64"])
def test_learn_same_bits_for_every_rows_setting(setup, arith):
    """Column-owned rollouts (r <= 32): 1, 2 or 4 operator rows per CTA, i.e. clusters of up
    to 16 CTAs per candidate, give the same bits in either arithmetic."""
    dp, synth, w, D, Qh = setup
    b1 = synth.logspace(-8, 2, 4)
    b2 = synth.logspace(-8, 2, 4)
    prev = dp.dopinf_tune_rollout_rows(0)
    prev_a = dp.dopinf_tune_rollout_arith(dp.ROLLOUT_DW if arith == "dw" else dp.ROLLOUT_FP64)
    runs = {}
    try:
        for rc in (1, 2, 4):
            dp.dopinf_tune_rollout_rows(rc)
            runs[rc] = dp.dopinf_learn(Qh, [6, 16], b1, b2, 400, mode=dp.CONTINUOUS_RK4, dt=w.snap_dt)
    finally:
        dp.dopinf_tune_rollout_rows(prev)
        dp.dopinf_tune_rollout_arith(prev_a)
    ref = runs[1]
    assert (ref["status"] == 0).sum().item() >= 2
    for rc, res in runs.items():
        assert res["best"] == ref["best"], rc
        for key in ("train_err", "growth", "status", "steps", "O_best"):
            assert torch.equal(res[key], ref[key]), (rc, key)


@pytest.mark.parametrize("arith", ["fp64", "dw"])
def test_learn_same_bits_for_every_large_rows_setting(setup, arith):
    """Rollouts of an r above 32 (operator rows in shared memory): 3 to 8 rows per CTA (clusters
    of 12 down to 5 CTAs at r = 34) give the same bits, in both arithmetics."""
    dp, synth, w, D, Qh = setup
    Qh34 = torch.from_numpy(_reduce34(setup)).cuda().t()
    b1 = synth.logspace(-6, 2, 3)
    b2 = synth.logspace(-6, 2, 3)
    prev = dp.dopinf_tune_rollout_rows_large(0)
    prev_a = dp.dopinf_tune_rollout_arith(dp.ROLLOUT_FP64 if arith == "fp64" else dp.ROLLOUT_DW)
    runs = {}
    try:
        for c in (3, 4, 5, 6, 7, 8):
            dp.dopinf_tune_rollout_rows_large(c)
            runs[c] = dp.dopinf_learn(Qh34, [6, 34], b1, b2, 200, mode=dp.CONTINUOUS_RK4, dt=w.snap_dt)
    finally:
        dp.dopinf_tune_rollout_rows_large(prev)
        dp.dopinf_tune_rollout_arith(prev_a)
    ref = runs[3]
    assert (ref["status"] == 0).sum().item() >= 1
    for c, res in runs.items():
        assert res["best"] == ref["best"], c
        for key in ("train_err", "growth", "status", "steps", "O_best"):
            assert torch.equal(res[key], ref[key]), (c, key)


def _reduce34(setup):
    from oracle import dopinf_oracle as O
    D = setup[3].cpu().numpy()
    return O.reduce(D, r_fixed=34)["Qhat"].T.copy()


def test_tuners_pick_a_measured_setting(setup):
    dp, synth, w, D, Qh = setup
    from paper_2504_14338_gb300 import autotune
    b1 = synth.logspace(-8, 2, 4)
    b2 = synth.logspace(-8, 2, 4)
    prev_c, prev_r = dp.dopinf_tune_rollout_rows(0), dp.dopinf_tune_reduce_coop(-1)
    try:
        t = autotune.tune_learn(Qh, [6, 16], b1, b2, 400, mode=dp.CONTINUOUS_RK4, dt=w.snap_dt)
        assert t["best"] in (1, 2, 4, 8) and len(t["rollout_ms"]) == 4
        assert dp.dopinf_tune_rollout_rows(0) == t["best"]
        assert min(t["rollout_ms"].values()) == t["rollout_ms"][t["best"]] > 0
        r = autotune.tune_reduce(D, 16)
        assert r["best"] in (0, 1) and dp.dopinf_tune_reduce_coop(-1) == r["best"]
    finally:
        dp.dopinf_tune_rollout_rows(prev_c)
        dp.dopinf_tune_reduce_coop(prev_r)
