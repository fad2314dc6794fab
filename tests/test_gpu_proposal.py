"""The learned (beta1, beta2, r) proposal, trained on the GPU by the library's kernels on grid-
search labels of seeded systems, against the method without it (the full grid search) and
against the same network untrained, on held-out seeds."""
import numpy as np
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
    from paper_2504_14338_gb300 import proposal as P
    spec = P.ProposalSpec(r_list=(4, 8, 12), n_b1=6, n_b2=6, k_range=(200, 260), r_true_range=(5, 16),
                          n_per_var=500)
    ws = dp.Workspace("cuda")
    X, y, kept = P.dataset(spec, range(0, 160), ws)
    return dp, P, spec, ws, X, y


def test_training_lowers_the_loss(setup):
    dp, P, spec, ws, X, y = setup
    assert X.shape[0] >= 100 and X.shape[1] == 64
    model = P.train(spec, X, y, steps=800)
    assert model["losses"][-1] < 0.7 * model["losses"][0]


def test_proposal_beats_untrained_and_cuts_the_search(setup):
    dp, P, spec, ws, X, y = setup
    model = P.train(spec, X, y, steps=800)
    untrained = P.train(spec, X, y, steps=1, lr=0.0)
    seeds = range(5000, 5040)
    res = P.evaluate(spec, model, seeds, ws)
    base = P.evaluate(spec, untrained, seeds, ws)
    print({k: v for k, v in res.items() if k != "rows"})
    print({k: v for k, v in base.items() if k != "rows"})
    # with the grid as fallback every selection is valid; the trained network needs far fewer
    # candidate evaluations than the grid and than the untrained network
    assert res["n"] >= 20
    assert res["work_ratio"] >= 5.0
    assert res["work_ratio"] >= base["work_ratio"]
    assert res["median_error_ratio"] <= base["median_error_ratio"] + 1e-12
