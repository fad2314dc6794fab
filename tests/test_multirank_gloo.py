"""World-size-2 CPU ranks (gloo) running the paper's partitioned algorithm with the oracle:
row blocks per rank, MAX of the scales, SUM of the Gram partials, MIN of (error, index) over
the pair ranges.  The combined results must equal the single-process ones."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2504_14338_gb300 import partition as P


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    from paper_2504_14338_gb300 import synth
    w = synth.Workload("t", 2, 301, 60, 4, var_scales=(1e-2, 1e2), seed=4)
    Q, _ = synth.snapshots_numpy(w)
    return w, np.ascontiguousarray(Q)


def _worker(rank, size, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    from oracle import dopinf_oracle as O
    w, Q = _problem()
    rows = P.rank_rows(w.n_per_var, w.n_vars, rank, size)
    Ql = Q[rows]
    # Step II: local centring; the scale needs the global MAX of the local max-abs values
    Qc, mean, _, _ = O.transform(Ql, P.local_var_offsets(w.n_per_var, w.n_vars, rank, size), scale=False)
    nl = len(rows) // w.n_vars
    loc = torch.tensor([np.abs(Qc[j * nl:(j + 1) * nl]).max() for j in range(w.n_vars)], dtype=torch.float64)
    dist.all_reduce(loc, op=dist.ReduceOp.MAX)
    scale = loc.numpy()
    for j in range(w.n_vars):
        Qc[j * nl:(j + 1) * nl] /= scale[j]
    # Step III: SUM of the Gram partials
    D = torch.from_numpy(O.gram(Qc))
    dist.all_reduce(D, op=dist.ReduceOp.SUM)
    red = O.reduce(D.numpy(), r_fixed=4)
    # Step IV: pairs split across ranks, MIN of (error, index)
    b1, b2 = w.beta1s(), w.beta2s()
    pairs = [(x, y) for x in b1 for y in b2]
    a, b = P.block_range(len(pairs), rank, size)
    errs, valid = [], []
    for (x, y) in pairs[a:b]:
        res = O.learn(red["Qhat"], [4], [x], [y], n_steps=w.k)
        errs.append(res["train_err"][0])
        valid.append(bool(res["valid"][0]))
    mine = P.best_of(errs, valid, a)
    allb = [None] * size
    dist.all_gather_object(allb, mine)
    out[rank] = dict(scale=scale, D=D.numpy(), best=P.merge_best(allb))
    dist.destroy_process_group()


def test_block_range_matches_paper_split():
    # floor split, remainder to the last rank (Section 3.2, distribute_nx; Section 3.5)
    assert [P.block_range(10, r, 3) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert [P.block_range(146339, r, 8) for r in (0, 7)] == [(0, 18292), (128044, 146339)]
    rows = P.rank_rows(5, 2, 1, 2)
    assert rows.tolist() == [2, 3, 4, 7, 8, 9]
    assert P.merge_best([(0.5, 7), (0.5, 3), (float("inf"), -1)]) == (0.5, 3)


@pytest.mark.timeout(300)
def test_two_gloo_ranks_match_single_process():
    from oracle import dopinf_oracle as O
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    w, Q = _problem()
    Qt, _, scale, _ = O.transform(Q, w.var_row_offsets())
    D = O.gram(Qt)
    for r in range(2):
        assert np.array_equal(out[r]["scale"], scale)          # MAX reduction is exact
        assert np.allclose(out[r]["D"], D, rtol=0, atol=1e-12 * np.abs(D).max())
    red = O.reduce(D, r_fixed=4)
    res = O.learn(red["Qhat"], [4], w.beta1s(), w.beta2s(), n_steps=w.k)
    assert out[0]["best"][1] == out[1]["best"][1] == res["best"]
