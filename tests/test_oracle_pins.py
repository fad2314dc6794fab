"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test pins one oracle function to something other than the oracle itself: a closed
form on a hand-made input, a value printed in the paper, a textbook identity evaluated by
an independent library routine (SVD, least squares, matrix powers), or brute force on a
tiny input.  None of these calls the CUDA library.
"""
import json
import os

import numpy as np
import pytest

from oracle import dopinf_oracle as O
from paper_2504_14338_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- Step II
def test_transform_closed_form():
    # two variables: rows 0-1 are variable 0, row 2 is variable 1 (Step II, Section 3.3)
    Q = np.array([[1.0, 2.0, 3.0, 6.0], [4.0, 4.0, 4.0, 4.0], [-1.0, 0.0, 1.0, 0.0]])
    Qt, mean, scale, flags = O.transform(Q, [0, 2, 3])
    assert mean.tolist() == [3.0, 4.0, 0.0]
    assert scale.tolist() == [3.0, 1.0]
    expect = np.array([[-2.0 / 3.0, -1.0 / 3.0, 0.0, 1.0], [0, 0, 0, 0], [-1.0, 0.0, 1.0, 0.0]])
    assert np.array_equal(Qt, expect)
    assert flags == 0


def test_transform_sum_is_sequential_in_time():
    # A sequential left-to-right sum gives ((1e16 + 1) - 1e16) + 1 = 1, a pairwise one 0.
    Q = np.array([[1e16, 1.0, -1e16, 1.0]])
    _, mean, _, _ = O.transform(Q, [0, 1], scale=False)
    assert mean[0] == 0.25


def test_transform_invariants_random():
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((300, 37)) * np.array([1e-3] * 100 + [1e4] * 200)[:, None] + 5.0
    Qt, mean, scale, flags = O.transform(Q, [0, 100, 300])
    assert flags == 0
    for a, b in [(0, 100), (100, 300)]:
        assert np.max(np.abs(Qt[a:b])) == 1.0           # max-abs scaling reaches exactly 1
    # centred rows, to the rounding of the offset 5 relative to the scale (~3e-3)
    assert np.max(np.abs(Qt.mean(axis=1))) < 1e-11
    # the undo of the transform returns the data (scaled, centred, shifted back)
    back = Qt * np.repeat(scale, [100, 200])[:, None] + mean[:, None]
    assert np.allclose(back, Q, rtol=1e-13, atol=1e-9)


def test_transform_fp32_steps():
    Q = np.array([[1.0, 2.0, 4.0], [0.5, 0.25, 0.25]], dtype=np.float32)
    Qt, mean, scale, flags = O.transform(Q, [0, 2])
    assert Qt.dtype == np.float32
    assert mean.tolist() == [7.0 / 3.0, 1.0 / 3.0]
    # centred in FP64 then rounded to FP32; the scale is the FP32 max-abs
    c = (Q.astype(np.float64) - mean[:, None]).astype(np.float32)
    s = np.float32(max(abs(c.min()), abs(c.max())))
    assert scale[0] == float(s) == float(np.float32(4.0 - 7.0 / 3.0))
    assert np.array_equal(Qt, c / s)


def test_transform_flags():
    Q = np.ones((4, 3))
    _, _, scale, flags = O.transform(Q, [0, 2, 4])
    assert flags & O.ZERO_SCALE and scale.tolist() == [1.0, 1.0]
    Q[1, 1] = np.nan
    _, _, _, flags = O.transform(Q, [0, 4])
    assert flags & O.NONFINITE


# ----------------------------------------------------------------------------- Step III
def test_gram_eigenvalues_are_squared_singular_values():
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((57, 9))
    D = O.gram(Q)
    sig = np.linalg.svd(Q, compute_uv=False)          # eq. thin_svd, an independent routine
    lam, U = O.eig_desc(D)
    assert np.allclose(lam, sig ** 2, rtol=1e-12, atol=1e-12 * sig[0] ** 2)
    assert np.isclose(np.trace(D), np.sum(Q * Q), rtol=1e-14)
    assert np.array_equal(D, D.T)


def test_gram_promotes_fp32_exactly():
    rng = np.random.default_rng(2)
    Q32 = rng.standard_normal((40, 5)).astype(np.float32)
    D = O.gram(Q32)
    # products of two FP32 numbers are exact in FP64; a 3-term sum per entry of exact
    # small integers checks the promotion
    Qi = np.array([[1, 2], [3, 4], [5, 6]], dtype=np.float32) * np.float32(1 + 2 ** -20)
    Di = O.gram(Qi)
    f = (1 + 2 ** -20) ** 2
    assert Di[0, 1] == (1 * 2 + 3 * 4 + 5 * 6) * f
    assert D.dtype == np.float64


def test_eig_desc_decomposition_and_sign_rule():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((30, 12))
    D = X.T @ X
    lam, U = O.eig_desc(D)
    assert np.all(np.diff(lam) <= 0)
    assert np.allclose(U.T @ U, np.eye(12), atol=1e-13)
    assert np.linalg.norm(U @ np.diag(lam) @ U.T - D) <= 1e-13 * lam[0] * 12
    for j in range(12):
        i = np.argmax(np.abs(U[:, j]))
        assert U[i, j] > 0
    # eigenvalues of an SPD matrix are its singular values (independent routine)
    assert np.allclose(lam, np.linalg.svd(D, compute_uv=False), rtol=1e-12)


def test_energy_rank_strict_threshold():
    lam = np.array([5.0, 3.0, 1.0, 1.0])
    assert O.energy_rank(lam, 10.0, 0.79) == 2
    assert O.energy_rank(lam, 10.0, 0.8) == 3          # 8/10 is not > 0.8 (strict, Step III)
    assert O.energy_rank(lam, 10.0, 0.0) == 1
    assert O.energy_rank(lam, 10.0, 1.0) == 0          # never exceeded
    lam = 1.0 / np.arange(1, 101) ** 3
    total = lam.sum()
    r = O.energy_rank(lam, total, 0.9996)
    assert np.cumsum(lam)[r - 1] / total > 0.9996 >= np.cumsum(lam)[r - 2] / total


def test_projection_equals_explicit_pod_basis():
    # eq. dOpInf_projection: Qhat = T_r^T D = V_r^T Q with V_r the leading left singular vectors
    rng = np.random.default_rng(4)
    Q = rng.standard_normal((80, 11)) @ np.diag(2.0 ** -np.arange(11)) @ rng.standard_normal((11, 11))
    Q -= Q.mean(axis=1, keepdims=True)
    D = O.gram(Q)
    red = O.reduce(D, r_fixed=4)
    V, S, Wt = np.linalg.svd(Q, full_matrices=False)
    for j in range(4):                                  # align the SVD's signs to the oracle's
        if np.dot(Wt[j], red["U"][:, j]) < 0:
            V[:, j] *= -1
    Qhat_pod = V[:, :4].T @ Q
    assert np.allclose(red["Qhat"], Qhat_pod, rtol=0, atol=1e-11 * S[0])
    assert np.allclose(red["Qhat"] @ red["Qhat"].T, np.diag(S[:4] ** 2), atol=1e-10 * S[0] ** 2)
    assert np.max(np.abs(red["Qhat"].sum(axis=1))) < 1e-10 * S[0]   # centred data: zero-mean rows
    # eq. MoS_POD_basis: V_r = Q T_r
    assert np.allclose(Q @ red["Tr"], V[:, :4], atol=1e-11)


def test_projection_rejects_zero_eigenvalue():
    Q = np.array([[1.0, -1.0], [2.0, -2.0]])
    D = O.gram(Q)
    lam, U = O.eig_desc(D)
    with pytest.raises(ValueError):
        O.projection(D, U, lam, 2)


# ----------------------------------------------------------------------------- Step IV
def test_qhat_sq_order_hand_example():
    # the non-redundant products of Step IV, ordered i-major with j >= i
    q = np.array([2.0, 3.0, 5.0])
    assert O.qhat_sq(q).tolist() == [4.0, 6.0, 10.0, 9.0, 15.0, 25.0]
    Qh = np.array([[2.0, 3.0, 5.0], [1.0, -1.0, 0.5]])
    assert O.qhat_sq(Qh).tolist() == [[4, 6, 10, 9, 15, 25], [1, -1, 0.5, 1, -0.5, 0.25]]
    Dh = O.data_matrix(Qh)
    assert Dh.shape == (2, 3 + 6 + 1) and np.all(Dh[:, -1] == 1.0)
    assert np.array_equal(Dh[:, :3], Qh)


def test_regularised_solution_matches_augmented_least_squares():
    # eq. OpInf_reg: min ||Dhat O^T - Y||^2 + beta1 (||A||^2 + ||c||^2) + beta2 ||H||^2 equals the
    # plain least-squares problem [Dhat; sqrt(diag reg)] O^T = [Y; 0], solved here by SVD.
    rng = np.random.default_rng(5)
    r = 3
    Qh = rng.standard_normal((r, 40))
    Dhat, Y = O.learning_data(Qh, r)
    b1, b2 = 0.3, 7.0
    reg = O.regulariser(r, b1, b2)
    assert reg.tolist() == [b1] * 3 + [b2] * 6 + [b1]
    G, B = O.normal_equations(Dhat, Y)
    Oc, ok = O.solve_cholesky(G, B, reg)
    assert ok
    aug = np.vstack([Dhat, np.diag(np.sqrt(reg))])
    rhs = np.vstack([Y, np.zeros((len(reg), r))])
    Ols = np.linalg.lstsq(aug, rhs, rcond=None)[0].T
    assert np.allclose(Oc, Ols, rtol=1e-10, atol=1e-12)
    assert np.allclose(O.solve_lu(G, B, reg), Ols, rtol=1e-10, atol=1e-12)
    A, H, c = O.split_operators(Oc, r)
    assert A.shape == (3, 3) and H.shape == (3, 6) and c.shape == (3,)


def test_cholesky_breakdown_is_reported():
    G = np.array([[1.0, 2.0], [2.0, 1.0]])   # indefinite
    O_, ok = O.solve_cholesky(G, np.ones((2, 1)), np.zeros(2))
    assert not ok and O_ is None


def _tensor_map(A, H3, c, x):
    return A @ x + np.einsum("ijk,j,k->i", H3, x, x) + c


def test_discrete_opinf_recovers_known_quadratic_map():
    # beta -> 0 on data of an exact discrete quadratic map lifted by an orthonormal basis:
    # the learned map equals the true map in POD coordinates, F_hat(q) = R^T F(R q), R = X T_r.
    rng = np.random.default_rng(6)
    r = 3
    th = 0.9
    A = 0.97 * np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 0.5]])
    H3 = rng.standard_normal((r, r, r)) * 0.05
    H3 = 0.5 * (H3 + H3.transpose(0, 2, 1))
    c = np.array([0.1, -0.05, 0.2])
    X = np.empty((r, 60))
    X[:, 0] = [1.0, 0.0, 0.3]
    for t in range(59):
        X[:, t + 1] = _tensor_map(A, H3, c, X[:, t])
    Phi, _ = np.linalg.qr(rng.standard_normal((200, r)))
    Q = Phi @ X
    D = O.gram(Q)
    red = O.reduce(D, r_fixed=r)
    R = X @ red["Tr"]                         # Phi^T V_r, orthogonal
    assert np.allclose(R.T @ R, np.eye(r), atol=1e-10)
    Dhat, Y = O.learning_data(red["Qhat"], r)
    G, B = O.normal_equations(Dhat, Y)
    Op, ok = O.solve_cholesky(G, B, O.regulariser(r, 1e-14, 1e-14))
    assert ok
    for q in rng.standard_normal((5, r)):
        assert np.allclose(O.rom_step_discrete(Op, r, q), R.T @ _tensor_map(A, H3, c, R @ q),
                           rtol=1e-7, atol=1e-7)
    # the learned model reproduces the training data: training error ~ 0
    Qt = O.rollout(Op, r, red["Qhat"][:, 0], 60)
    assert O.train_error(red["Qhat"].T, Qt) < 1e-6


def test_continuous_opinf_recovers_rk4_system_to_fd_order():
    # continuous mode on RK4 data of a known system: central differences are second order,
    # so the learned right-hand side matches the true one to O(dt^2).
    w = synth.Workload("pin", 1, 50, 400, 3, dt=1e-3, stride=1, noise_rel=0.0, seed=7)
    X, (A, H3, c) = synth.trajectory(w)
    rng = np.random.default_rng(8)
    Phi, _ = np.linalg.qr(rng.standard_normal((50, 3)))
    Q = Phi @ X
    red = O.reduce(O.gram(Q), r_fixed=3)
    R = X @ red["Tr"]
    Dhat, Y = O.learning_data(red["Qhat"], 3, mode="continuous", dt=w.snap_dt)
    G, B = O.normal_equations(Dhat, Y)
    Op, ok = O.solve_cholesky(G, B, O.regulariser(3, 1e-14, 1e-14))
    assert ok
    for t in (50, 200, 350):
        q = red["Qhat"][:, t]
        f_true = R.T @ _tensor_map(A, H3, c, R @ q)
        assert np.linalg.norm(O.rom_rhs(Op, 3, q) - f_true) < 1e-3 * np.linalg.norm(f_true)


def test_discrete_rollout_affine_closed_form():
    rng = np.random.default_rng(9)
    r = 4
    A = rng.standard_normal((r, r)) * 0.3
    c = rng.standard_normal(r)
    Op = np.hstack([A, np.zeros((r, r * (r + 1) // 2)), c[:, None]])
    q0 = rng.standard_normal(r)
    Qt = O.rollout(Op, r, q0, 7)
    for t in range(7):
        expect = np.linalg.matrix_power(A, t) @ q0 + sum(np.linalg.matrix_power(A, j) @ c for j in range(t))
        assert np.allclose(Qt[t], expect, rtol=1e-12, atol=1e-12)


def test_rk4_linear_closed_form_and_order():
    # classical RK4 on q' = A q multiplies by the degree-4 Taylor polynomial of exp(hA)
    from scipy.linalg import expm
    rng = np.random.default_rng(10)
    r = 3
    A = rng.standard_normal((r, r))
    Op = np.hstack([A, np.zeros((r, 6)), np.zeros((r, 1))])
    q0 = rng.standard_normal(r)
    h = 0.05
    hA = h * A
    P = np.eye(r) + hA + hA @ hA / 2 + hA @ hA @ hA / 6 + hA @ hA @ hA @ hA / 24
    Qt = O.rollout(Op, r, q0, 11, mode="continuous", dt=h)
    assert np.allclose(Qt[10], np.linalg.matrix_power(P, 10) @ q0, rtol=1e-12)
    errs = []
    for hh in (0.02, 0.01):
        n = int(round(0.4 / hh))
        errs.append(np.linalg.norm(O.rollout(Op, r, q0, n + 1, "continuous", hh)[n] - expm(0.4 * A) @ q0))
    assert 12 < errs[0] / errs[1] < 20                  # fourth order


def test_rk4_conserves_energy_of_energy_preserving_quadratic():
    rng = np.random.default_rng(11)
    r = 4
    _, H3, _ = synth.quadratic_system(r, rng)
    S = rng.standard_normal((r, r))
    A = S - S.T                                          # skew: x^T A x = 0
    Op = np.hstack([A, synth.unique_quadratic(H3), np.zeros((r, 1))])
    q0 = rng.standard_normal(r)
    Qt = O.rollout(Op, r, q0, 201, mode="continuous", dt=1e-3)
    nrm = np.linalg.norm(Qt, axis=1)
    assert np.max(np.abs(nrm - nrm[0])) < 1e-9 * nrm[0]


def test_train_error_is_per_time_step_norm_over_modes():
    Qh = np.array([[3.0, 4.0], [1.0, 0.0], [0.0, 2.0]])
    Qt = np.array([[3.0, 4.0], [1.0, 1.0], [0.0, 2.5]])
    # per time step: 0, sqrt(1/1) = 1, sqrt(0.25/4) = 0.25; maximum 1
    assert O.train_error(Qh, Qt) == 1.0
    assert O.growth_ratio(np.array([[0.0, 3.0]]), np.array([0.0, 0.0]), np.array([1.0, 2.0])) == 1.5


def test_learn_selection_and_ties():
    w = synth.WORKLOADS["small"]
    X, _ = synth.trajectory(w)
    rng = np.random.default_rng(12)
    Phi, _ = np.linalg.qr(rng.standard_normal((64, w.r_true)))
    Q = Phi @ X
    Qt, _, _, _ = O.transform(Q, [0, 32, 64])
    red = O.reduce(O.gram(Qt), r_fixed=4)
    b = [1e-6, 1e-6, 1e-2]                               # a repeated value makes an exact tie
    res = O.learn(red["Qhat"], [3, 4], b, [1e-3], n_steps=w.k)
    assert res["valid"].any()
    P = len(res["candidates"])
    assert P == 6
    valid_err = np.where(res["valid"], res["train_err"], np.inf)
    best = res["best"]
    assert best == int(np.argmin(valid_err))            # lowest flat index among equal minima
    assert res["candidates"][0] == (3, 1e-6, 1e-3)      # r-major, then beta1, then beta2
    if res["valid"][0]:
        assert res["train_err"][0] == res["train_err"][1]
    none = O.learn(red["Qhat"], [3], [1e-6], [1e-3], n_steps=w.k, max_growth=0.0)
    assert none["best"] == -1


def test_grid_matches_printed_optimum():
    # Section 4 prints beta1* = 7.19e-8 and beta2* = 51.79, members of the Step IV grids
    # logspace(-10, 0, 8) and logspace(-4, 4, 8): this pins base 10, inclusive endpoints.
    g = json.load(open(os.path.join(GOLDEN, "paper_grid.json")))
    B1 = synth.logspace(*g["beta1_grid"])
    B2 = synth.logspace(*g["beta2_grid"])
    # the printed values are the grid members cut (not rounded) to the printed digits:
    # exactly one member of each grid lies in [printed, printed + one unit of the last digit)
    for grid, idx, val, unit in ((B1, g["beta1_index"], g["beta1_opt_printed"], 1e-10),
                                 (B2, g["beta2_index"], g["beta2_opt_printed"], 1e-2)):
        inside = [i for i, v in enumerate(grid) if val <= v < val + unit]
        assert inside == [idx]
    assert B1[0] == 1e-10 and B1[-1] == 1.0 and B2[0] == 1e-4 and B2[-1] == 1e4


# ----------------------------------------------------------------------------- Step V
def test_lift_recovers_the_snapshots_with_every_mode():
    """With r equal to the rank of the centred data, V_r V_r^T is the projector onto its range:
    lifting the reduced coordinates of the training data (Qhat = V_r^T Q) returns the
    transformed snapshots, and undoing the transform returns the raw snapshots."""
    rng = np.random.default_rng(11)
    n, k, rank = 400, 30, 7
    Q = rng.standard_normal((n, rank)) @ rng.standard_normal((rank, k)) + rng.standard_normal((n, 1)) * 3.0
    Q[200:] *= 50.0
    offs = [0, 200, 400]
    Qt, mean, scale, _ = O.transform(Q, offs)
    # the numerical rank of the centred, scaled data (at most 7: centring may remove a direction)
    lam = O.reduce(O.gram(Qt), r_fixed=1)["lam"]
    r = int(np.sum(lam > 1e-10 * lam[0]))
    red = O.reduce(O.gram(Qt), r_fixed=r)
    rows = np.array([0, 5, 199, 200, 333, 399])
    X = O.lift(Qt, red["Tr"], red["Qhat"], rows, mean, scale, offs)
    assert np.allclose(X, Q[rows], rtol=1e-10, atol=1e-10 * np.abs(Q).max())
    Y = O.lift(Qt, red["Tr"], red["Qhat"], rows)
    assert np.allclose(Y, Qt[rows], atol=1e-12)


def test_lift_basis_equals_left_singular_vectors():
    """V_r = Q T_r are the leading left singular vectors of Q (sign-aligned), computed here by
    numpy's SVD: the lifted rows equal U_r[rows] Sigma_r W_r^T restricted to the rows."""
    rng = np.random.default_rng(12)
    Q = rng.standard_normal((120, 15)) @ np.diag(0.7 ** np.arange(15))
    red = O.reduce(O.gram(Q), r_fixed=5)
    U, S, Wt = np.linalg.svd(Q, full_matrices=False)
    V = O.pod_basis_rows(Q, red["Tr"], np.arange(120))
    s = np.sign(np.sum(U[:, :5] * V, axis=0))
    assert np.allclose(V, U[:, :5] * s, atol=1e-12)
    Qtilde = rng.standard_normal((5, 9))
    rows = [3, 77, 119]
    assert np.allclose(O.lift(Q, red["Tr"], Qtilde, rows), (U[:, :5] * s)[rows] @ Qtilde, atol=1e-12)


def test_lift_inverse_transform_by_hand():
    """The inverse transform on a hand input: y * scale + mean per row, with the row's variable."""
    Q = np.eye(3)
    Tr = np.eye(3)[:, :2]
    Qtilde = np.array([[1.0, 2.0], [3.0, 4.0]])
    X = O.lift(Q, Tr, Qtilde, [0, 1, 2], np.array([10.0, 20.0, 30.0]), np.array([2.0, 5.0]), [0, 2, 3])
    assert X.tolist() == [[12.0, 14.0], [26.0, 28.0], [30.0, 30.0]]


def test_transform_std_scaling_closed_form():
    """Scaling by the standard deviation of the centred variable (Section 3.3's alternative):
    a variable whose centred values are +-a has standard deviation a; a constant variable is
    left unscaled and flagged; afterwards every variable has unit RMS."""
    Q = np.array([[1.0, 5.0, 1.0, 5.0], [10.0, 14.0, 10.0, 14.0], [7.0, 7.0, 7.0, 7.0]])
    Qt, mean, scale, flags = O.transform(Q, [0, 2, 3], scaling="std")
    assert scale.tolist() == [2.0, 1.0]
    assert np.array_equal(Qt[:2], np.array([[-1.0, 1.0, -1.0, 1.0]] * 2))
    assert flags == 2
    rng = np.random.default_rng(5)
    R = rng.standard_normal((500, 40)) * np.repeat([3e-3, 7e2], 250)[:, None] + 1.0
    Rt, _, s, _ = O.transform(R, [0, 250, 500], scaling="std")
    for a, b in [(0, 250), (250, 500)]:
        assert abs(np.sqrt(np.mean(Rt[a:b] ** 2)) - 1.0) < 1e-13
    # equals numpy's population standard deviation of the centred block
    C = R - R.mean(axis=1, keepdims=True)
    assert np.allclose(s, [C[:250].std(), C[250:].std()], rtol=1e-13)


def test_qr_solve_equals_normal_equations_and_lstsq():
    """The QR route of the regularised problem: on a well-conditioned problem it equals the
    Cholesky solution of the normal equations and numpy's lstsq of the stacked system; on an
    ill-conditioned one (tiny beta, nearly dependent columns) its residual of the regularised
    normal equations stays at the rounding level of the stacked matrix, not of its square."""
    rng = np.random.default_rng(21)
    Qh = rng.standard_normal((5, 80))
    Dh, Y = O.learning_data(Qh, 5)
    G, B = O.normal_equations(Dh, Y)
    reg = O.regulariser(5, 1e-1, 1e-1)
    Oq, ok = O.solve_qr(Dh, Y, reg)
    Oc, _ = O.solve_cholesky(G, B, reg)
    assert ok and np.allclose(Oq, Oc, rtol=1e-10, atol=1e-12)
    A = np.vstack([Dh, np.diag(np.sqrt(reg))])
    b = np.vstack([Y, np.zeros((Dh.shape[1], 5))])
    assert np.allclose(Oq.T, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-10, atol=1e-12)
    # nearly collinear data: the stacked system's conditioning, not its square
    Qh2 = Qh.copy()
    Qh2[1] = Qh2[0] * (1 + 1e-7) + 1e-9 * rng.standard_normal(80)
    Dh2, Y2 = O.learning_data(Qh2, 5)
    reg2 = O.regulariser(5, 1e-12, 1e-12)
    Oq2, ok2 = O.solve_qr(Dh2, Y2, reg2)
    A2 = np.vstack([Dh2, np.diag(np.sqrt(reg2))])
    b2 = np.vstack([Y2, np.zeros((Dh2.shape[1], 5))])
    ref = np.linalg.lstsq(A2, b2, rcond=None)[0]
    assert ok2
    # the least-squares residual norm is the minimum: QR reaches it to rounding
    r_qr = np.linalg.norm(A2 @ Oq2.T - b2)
    r_ref = np.linalg.norm(A2 @ ref - b2)
    assert r_qr <= r_ref * (1 + 1e-8) + 1e-12
