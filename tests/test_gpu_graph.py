"""The whole hot path captured into a CUDA graph through the asynchronous entry points gives
the same bits as the synchronous calls, and a replay on fresh input gives them again."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2504_14338_gb300 import dopinf
    return dopinf


@pytest.mark.parametrize("gram_mode", ["ozaki", "fp64"])
def test_graph_replay_matches_synchronous_calls(dp, gram_mode):
    from paper_2504_14338_gb300 import synth
    from paper_2504_14338_gb300.graph import PipelineGraph
    w = synth.WORKLOADS["small"]
    Qn, _ = synth.snapshots_numpy(w)
    Q0 = torch.from_numpy(np.asarray(Qn)).cuda()
    Q = dp.snapshot_matrix(w.n, w.k)
    gm = dp.GRAM_OZAKI_FP64 if gram_mode == "ozaki" else dp.GRAM_FP64
    r_list, r_cap, n_steps = [4, 6], 6, 400
    b1 = synth.logspace(-8, 2, 4)
    b2 = synth.logspace(-8, 2, 4)
    mode, dt = dp.CONTINUOUS_RK4, w.snap_dt
    # synchronous calls
    Q.copy_(Q0)
    dp.dopinf_transform(Q, w.var_row_offsets())
    D = dp.dopinf_gram(Q, mode=gm)
    red = dp.dopinf_reduce(D, r_cap=r_cap, r_fixed=r_cap)
    ref = dp.dopinf_learn(red["Qhat"], r_list, b1, b2, n_steps, mode=mode, dt=dt)
    # captured graph
    Q.copy_(Q0)
    pg = PipelineGraph(Q, w.var_row_offsets(), r_cap, r_list, b1, b2, n_steps, mode=mode, dt=dt, gram_mode=gm)
    pg.capture()
    for _ in range(2):  # each replay starts from the same input
        Q.copy_(Q0)
        pg.replay()
        torch.cuda.synchronize()
        assert pg.flags_value() == 0
        assert torch.equal(pg.D, D)
        assert torch.equal(pg.red["eigvals"], red["eigvals"])
        assert torch.equal(pg.red["Qhat"], red["Qhat"])
        assert int(pg.red["r"].item()) == red["r"]
        for key in ("train_err", "growth", "status", "steps"):
            assert torch.equal(pg.res[key], ref[key]), key
        assert int(pg.res["best"].item()) == ref["best"]
        assert torch.equal(pg.res["O_best"], ref["O_best"])


def test_overlapped_pipeline_matches_synchronous_calls(dp):
    """Consecutive pipelines with the front of each step beside the previous step's learn step
    (two streams, two snapshot copies) give every step the bits of the synchronous calls on its
    own input."""
    import dataclasses
    from paper_2504_14338_gb300 import synth
    from paper_2504_14338_gb300.graph import OverlappedPipeline
    base = synth.WORKLOADS["small"]
    r_list, r_cap, n_steps = [4, 6], 6, 300
    b1 = synth.logspace(-8, 2, 3)
    b2 = synth.logspace(-8, 2, 3)
    inputs, refs = [], []
    for seed in (11, 12):
        w = dataclasses.replace(base, seed=seed)
        Qn, _ = synth.snapshots_numpy(w)
        Q0 = torch.from_numpy(np.asarray(Qn)).cuda()
        Q = dp.snapshot_matrix(w.n, w.k)
        Q.copy_(Q0)
        dp.dopinf_transform(Q, w.var_row_offsets())
        red = dp.dopinf_reduce(dp.dopinf_gram(Q, mode=dp.GRAM_OZAKI_FP64), r_cap=r_cap, r_fixed=r_cap)
        refs.append(dp.dopinf_learn(red["Qhat"], r_list, b1, b2, n_steps, mode=dp.CONTINUOUS_RK4, dt=w.snap_dt))
        assert refs[-1]["best"] >= 0
        inputs.append(Q0)
    copies = [dp.snapshot_matrix(w.n, w.k) for _ in range(2)]
    for c, q in zip(copies, inputs):
        c.copy_(q)
    op = OverlappedPipeline(copies, w.var_row_offsets(), r_cap, r_list, b1, b2, n_steps, mode=dp.CONTINUOUS_RK4,
                            dt=w.snap_dt, gram_mode=dp.GRAM_OZAKI_FP64)
    for i in range(5):  # inputs alternate with the copies; no synchronisation between steps
        op.submit(refill=lambda Q, src=inputs[i % 2]: Q.copy_(src, non_blocking=True))
        if i >= 3:
            out = op.results(i)
            ref = refs[i % 2]
            assert out["flags"] == 0
            assert int(out["res"]["best"].item()) == ref["best"]
            for key in ("train_err", "growth", "status", "steps", "O_best"):
                assert torch.equal(out["res"][key], ref[key]), (i, key)


def test_batched_learn_graph_matches_each_problem(dp):
    """Several problems of uneven r (the batched-learn configuration at test scale: r drawn
    from a range, a 6 x 6 grid each) in one captured graph, each equal to its own learn call."""
    from paper_2504_14338_gb300 import synth
    from paper_2504_14338_gb300.graph import BatchedLearnGraph
    from oracle import dopinf_oracle as O
    rng = np.random.default_rng(7)
    problems = []
    for p in range(4):
        w = synth.Workload("batch%d" % p, 2, 512, int(rng.integers(160, 220)), int(rng.integers(6, 14)), seed=100 + p)
        Qn, _ = synth.snapshots_numpy(w)
        Q = O.transform(Qn, w.var_row_offsets())[0]
        r = int(rng.integers(4, 9))
        Qh = O.reduce(O.gram(Q), r_fixed=r)["Qhat"]
        problems.append(dict(Qhat=torch.from_numpy(Qh.T.copy()).cuda().t(), r_list=[r - 2, r],
                             beta1=synth.logspace(-8, 0, 6), beta2=synth.logspace(-4, 2, 6)))
    bg = BatchedLearnGraph(problems, 300, mode=dp.DISCRETE).capture()
    bg.replay()
    torch.cuda.synchronize()
    for pr, out in zip(problems, bg.out):
        ref = dp.dopinf_learn(pr["Qhat"], pr["r_list"], pr["beta1"], pr["beta2"], 300)
        assert int(out["best"].item()) == ref["best"]
        for key in ("train_err", "growth", "status", "steps", "O_best"):
            assert torch.equal(out[key], ref[key]), key


def test_streaming_pipeline_matches_synchronous_calls(dp):
    """Matrices streamed from pinned host memory through the double-buffered pipeline (uploads
    and each step's transform and Gram overlapping the previous step): each step's host results
    equal the synchronous calls on that matrix, and a result slot is only reused two steps
    later."""
    import dataclasses
    from paper_2504_14338_gb300 import synth
    from paper_2504_14338_gb300.graph import StreamingPipeline
    base = synth.WORKLOADS["small"]
    r_list, r_cap, n_steps = [4, 6], 6, 300
    b1 = synth.logspace(-8, 2, 3)
    b2 = synth.logspace(-8, 2, 3)
    mode, dt = dp.CONTINUOUS_RK4, base.snap_dt
    mats, refs = [], []
    for seed in (11, 12, 13):
        w = dataclasses.replace(base, seed=seed)
        Qn, _ = synth.snapshots_numpy(w)
        host = torch.empty((w.k, w.n), dtype=torch.float64, pin_memory=True)
        host.copy_(torch.from_numpy(np.ascontiguousarray(np.asarray(Qn).T)))
        mats.append(host)
        Q = dp.snapshot_matrix(w.n, w.k)
        Q.copy_(host.t())
        dp.dopinf_transform(Q, w.var_row_offsets())
        red = dp.dopinf_reduce(dp.dopinf_gram(Q, mode=dp.GRAM_OZAKI_FP64), r_cap=r_cap, r_fixed=r_cap)
        refs.append(dp.dopinf_learn(red["Qhat"], r_list, b1, b2, n_steps, mode=mode, dt=dt))
    sp = StreamingPipeline(mats[0], base.var_row_offsets(), r_cap, r_list, b1, b2, n_steps, mode=mode, dt=dt,
                           record_times=True)
    outs = sp.run(mats + mats[::-1])
    up, span, wait = sp.step_times(5)
    assert up > 0.0 and span > 0.0 and wait >= 0.0
    assert len(outs) == 6
    for out, ref in zip(outs, refs + refs[::-1]):
        assert out["flags"] == 0
        assert out["best"] == ref["best"]
        assert torch.equal(out["train_err"], ref["train_err"].cpu())
        assert torch.equal(out["status"], ref["status"].cpu())
        assert torch.equal(out["O_best"], ref["O_best"].cpu())
    with pytest.raises(ValueError):
        sp.result(0)


def test_batched_learn_graph_large_r_of_one_kernel_shape(dp):
    """Problems with r above 32 whose launches share one kernel (the same rows per CTA) but
    differ in shared-memory size, the larger first, captured together and replayed twice in
    both arithmetics: each equal to its own learn call."""
    from paper_2504_14338_gb300 import synth
    from paper_2504_14338_gb300.graph import BatchedLearnGraph
    from test_gpu_parity import _reduced_large
    Qh = _reduced_large(64)
    problems = [dict(Qhat=torch.from_numpy(np.ascontiguousarray(Qh[:r].T)).cuda().t(), r_list=[r],
                     beta1=synth.logspace(-4, 0, 2), beta2=synth.logspace(0, 4, 2)) for r in (60, 48, 36, 52)]
    prev = dp.dopinf_tune_rollout_arith(0)
    try:
        for arith in (dp.ROLLOUT_FP64, dp.ROLLOUT_DW):
            dp.dopinf_tune_rollout_arith(arith)
            bg = BatchedLearnGraph(problems, 400, mode=dp.CONTINUOUS_RK4, dt=1e-2).capture()
            for _ in range(2):
                bg.replay()
                torch.cuda.synchronize()
                for pr, out in zip(problems, bg.out):
                    ref = dp.dopinf_learn(pr["Qhat"], pr["r_list"], pr["beta1"], pr["beta2"], 400,
                                          mode=dp.CONTINUOUS_RK4, dt=1e-2)
                    assert int(out["best"].item()) == ref["best"]
                    for key in ("train_err", "growth", "status", "steps", "O_best"):
                        assert torch.equal(out[key], ref[key]), key
            del bg
    finally:
        dp.dopinf_tune_rollout_arith(prev)
