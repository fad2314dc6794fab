"""Plain FP64 CPU oracle for the dOpInf hot path (Farcas et al., arXiv 2504.14338).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or link this
module: only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code, headers, tables
or helpers with the CUDA library; the only thing both sides consume is the seeded
input generator module, which contains none of the method's arithmetic.

Every function follows one step of the paper (Section 3.3 Step II, Section 3.4 Step III,
Section 3.5 Step IV, Section 3.6 Step V) in the paper's order and notation.  Library primitives (numpy
matmul, ``np.linalg.eigh``, ``np.linalg.solve``, ``np.linalg.cholesky``) serve as steps;
there is no blocking or fusion beyond what the paper's definitions state.

Readings of the paper that the oracle adopts where it is silent or ambiguous:
  * centering is by per-row temporal mean, summed sequentially in time (Step II);
  * scaling divides each variable block by the global max-abs of its centered values;
    a block whose max-abs is 0 is left unscaled (scale := 1) and flagged;
  * FP32 storage: row sums and means in FP64; centered = fp32(fp64(x) - mean);
    scale = fp32 max-abs; scaled = centered / scale rounded in FP32;
  * the retained-energy denominator is trace(D) (equal to the eigenvalue sum in exact
    arithmetic), the comparison is strict (eq. ret_energy, with tau = 0.9996 as in the Step III code);
  * eigenvector sign: the entry of largest magnitude is positive (lowest index on ties);
  * the regulariser is beta (not beta^2) on the diagonal: beta1 on the r linear and the
    constant entries, beta2 on the s = r(r+1)/2 quadratic entries (eq. OpInf_reg);
  * the normal equations are solved by Cholesky (LU, as the paper's solve, is available
    for comparison); a non-positive pivot marks the candidate invalid;
  * a candidate is valid iff its rollout is finite and its growth ratio < max_growth;
    selection takes the minimum training error over valid candidates, ties broken by the
    lowest flat index (r-major, then beta1, then beta2, i.e. the Cartesian-product order);
  * continuous mode (eq. ROM_quad_time_cont): derivatives by second-order central differences on the
    interior snapshots t = 1..k-2, RK4 rollout with the snapshot spacing as step.

Parity pins are in tests/test_oracle_pins.py.  Every function here is pinned.
"""
import numpy as np
from scipy.linalg import solve_triangular

__all__ = [
    "transform", "gram", "eig_desc", "energy_rank", "projection", "qhat_sq",
    "data_matrix", "normal_equations", "regulariser", "solve_cholesky", "solve_lu", "solve_qr",
    "split_operators", "rom_step_discrete", "rom_rhs", "rk4_step", "rollout",
    "train_error", "growth_ratio", "learn", "reduce", "pipeline", "pod_basis_rows", "lift",
]

NONFINITE = 1
ZERO_SCALE = 2


# --------------------------------------------------------------------------------------
# Step II (Section 3.3): centering by the temporal mean, max-abs scaling per variable.
# --------------------------------------------------------------------------------------
def transform(Q, var_row_offsets, center=True, scale=True, scaling="maxabs"):
    """Centre each row by its temporal mean and scale each variable by its max-abs.

    Q: (n, k) float64 or float32 array, rows stacked variable-major.
    var_row_offsets: n_vars + 1 row offsets; variable j owns rows [off[j], off[j+1]).
    scaling: "maxabs" (the Step II code) or "std", the other strategy Section 3.3 names: the
    standard deviation of the variable's centred values, sqrt(sum c^2 / (rows * k)), in FP64.
    Returns (Q_transformed (same dtype), row_mean float64 (n,), var_scale float64 (n_vars,),
    flags) where flags has NONFINITE / ZERO_SCALE bits.
    """
    Q = np.array(Q, copy=True)
    n, k = Q.shape
    is32 = Q.dtype == np.float32
    flags = 0
    if not np.all(np.isfinite(Q)):
        flags |= NONFINITE
    # temporal mean of each row, the sum taken in time order in FP64
    acc = np.zeros(n, dtype=np.float64)
    for t in range(k):
        acc += Q[:, t].astype(np.float64)
    mean = acc / np.float64(k) if k > 0 else acc
    if center:
        if is32:
            Q = (Q.astype(np.float64) - mean[:, None]).astype(np.float32)
        else:
            Q = Q - mean[:, None]
    n_vars = len(var_row_offsets) - 1
    var_scale = np.ones(n_vars, dtype=np.float64)
    if scale:
        for j in range(n_vars):
            a, b = int(var_row_offsets[j]), int(var_row_offsets[j + 1])
            block = Q[a:b, :]
            if block.size == 0:
                continue
            if scaling == "std":
                c = block.astype(np.float64)
                s = Q.dtype.type(np.sqrt(np.sum(c * c) / c.size))
            else:
                s = max(abs(block.min()), abs(block.max()))
            if not np.isfinite(s):
                flags |= NONFINITE
            if s == 0:
                flags |= ZERO_SCALE
                s = Q.dtype.type(1)
            var_scale[j] = float(s)
            Q[a:b, :] = block / Q.dtype.type(s)
    return Q, mean, var_scale, flags


# --------------------------------------------------------------------------------------
# Step III (Section 3.4): method of snapshots, eqs. mos_partitioned .. dOpInf_projection.
# --------------------------------------------------------------------------------------
def gram(Q):
    """D = Q^T Q in FP64 (eq. mos_partitioned); FP32 data are promoted exactly first."""
    Q64 = np.asarray(Q, dtype=np.float64)
    return Q64.T @ Q64


def eig_desc(D):
    """Eigenpairs of the symmetric D sorted by descending eigenvalue (eq. mos_Sigma_W).

    Sign rule: the largest-magnitude entry of each eigenvector is made positive,
    the lowest index winning ties.
    """
    lam, U = np.linalg.eigh(np.asarray(D, dtype=np.float64))
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    U = U[:, order].copy()
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
    return lam, U


def energy_rank(lam, total, tau):
    """Smallest r whose cumulative energy fraction exceeds tau (eq. ret_energy); 0 if none does.

    lam: descending eigenvalues (possibly only the leading ones); total: the energy sum.
    """
    cum = 0.0
    for i, l in enumerate(lam):
        cum += float(l)
        if cum / total > tau:
            return i + 1
    return 0


def projection(D, U, lam, r):
    """T_r = U_r Lambda_r^{-1/2} and Qhat = T_r^T D (eqs. MoS_POD_basis, dOpInf_projection)."""
    if r <= 0 or lam[r - 1] <= 0:
        raise ValueError("lambda_r <= 0: reduced dimension exceeds the numerical rank")
    Tr = U[:, :r] @ np.diag(lam[:r] ** -0.5)
    Qhat = Tr.T @ D
    return Tr, Qhat


def reduce(D, tau=0.9996, r_fixed=0, r_cap=None):
    """Eigensolve, retained-energy rank and projection of Step III.

    Returns dict with r, eigenvalues (descending, all k), U, Tr (k x r_cap), Qhat (r_cap x k),
    trace.  Qhat for any r <= r_cap is the leading r rows.
    """
    D = np.asarray(D, dtype=np.float64)
    k = D.shape[0]
    lam, U = eig_desc(D)
    trace = float(np.trace(D))
    r = int(r_fixed) if r_fixed > 0 else energy_rank(lam, trace, tau)
    if r_cap is None:
        r_cap = r
    Tr, Qhat = projection(D, U, lam, max(r_cap, r))
    return dict(r=r, lam=lam, U=U, Tr=Tr, Qhat=Qhat, trace=trace, k=k)


# --------------------------------------------------------------------------------------
# Step IV (Section 3.5): quadratic OpInf, eqs. ROM_quad_time_cont .. OpInf_data_matrices_discrete.
# --------------------------------------------------------------------------------------
def qhat_sq(Qh):
    """Non-redundant quadratic products q_i q_j, i <= j, ordered i-major.

    Qh: (K, r) snapshots as rows, or (r,) a single state.
    """
    Qh = np.asarray(Qh, dtype=np.float64)
    if Qh.ndim == 1:
        r = Qh.shape[0]
        return np.concatenate([Qh[i] * Qh[i:] for i in range(r)])
    K, r = Qh.shape
    return np.concatenate([Qh[:, i:i + 1] * Qh[:, i:] for i in range(r)], axis=1)


def data_matrix(Qh1):
    """Dhat = [Qhat_1^T | (Qhat_1^T kron Qhat_1^T)_unique | 1] with rows = snapshots."""
    Qh1 = np.asarray(Qh1, dtype=np.float64)
    K = Qh1.shape[0]
    return np.concatenate([Qh1, qhat_sq(Qh1), np.ones((K, 1))], axis=1)


def learning_data(Qhat, r, mode="discrete", dt=1.0):
    """Rows of the data matrix and the targets for one reduced dimension r.

    Qhat: (>=r, k) reduced data, columns = snapshots.  Discrete (eq. OpInf_data_matrices_discrete): inputs are
    snapshots 0..k-2 and targets 1..k-1.  Continuous (eq. ROM_quad_time_cont): inputs are snapshots
    1..k-2 and targets the central differences (q_{t+1} - q_{t-1}) / (2 dt).
    Returns (Dhat, Y) with Y of shape (K, r).
    """
    Qr = np.asarray(Qhat, dtype=np.float64)[:r, :].T  # (k, r)
    if mode == "discrete":
        X, Y = Qr[:-1, :], Qr[1:, :]
    elif mode == "continuous":
        X = Qr[1:-1, :]
        Y = (Qr[2:, :] - Qr[:-2, :]) / (2.0 * dt)
    else:
        raise ValueError(mode)
    return data_matrix(X), Y


def normal_equations(Dhat, Y):
    """G = Dhat^T Dhat and B = Dhat^T Y of the least-squares problem eq. OpInf_reg."""
    return Dhat.T @ Dhat, Dhat.T @ Y


def regulariser(r, beta1, beta2):
    """Diagonal of the Tikhonov term of eq. OpInf_reg: beta1 on A and c, beta2 on H."""
    s = r * (r + 1) // 2
    reg = np.empty(r + s + 1)
    reg[:r] = beta1
    reg[r:r + s] = beta2
    reg[r + s:] = beta1
    return reg


def solve_cholesky(G, B, reg):
    """O^T = (G + diag(reg))^{-1} B by Cholesky; returns (O (r x d), ok)."""
    M = G + np.diag(reg)
    try:
        L = np.linalg.cholesky(M)
    except np.linalg.LinAlgError:
        return None, False
    Z = solve_triangular(L, B, lower=True)        # forward substitution
    X = solve_triangular(L.T, Z, lower=False)     # back substitution
    return X.T, True


def solve_lu(G, B, reg):
    """The paper's own route: np.linalg.solve (LU) of the regularised normal equations."""
    return np.linalg.solve(G + np.diag(reg), B).T


def solve_qr(Dhat, Y, reg):
    """The regularised least-squares problem of eq. OpInf_reg without forming the normal
    equations: min ||Dhat O^T - Y||^2 + ||diag(sqrt(reg)) O^T||^2 as the least-squares solution of
    the stacked system [Dhat; diag(sqrt(reg))] O^T = [Y; 0], by a Householder QR (numpy) and a
    triangular solve.  Returns (O (r x d), ok); ok is False when R has a zero diagonal entry."""
    Dhat = np.asarray(Dhat, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    d = Dhat.shape[1]
    A = np.vstack([Dhat, np.diag(np.sqrt(np.asarray(reg, dtype=np.float64)))])
    b = np.vstack([Y, np.zeros((d, Y.shape[1]))])
    Qm, R = np.linalg.qr(A, mode="reduced")
    if np.any(np.diag(R) == 0) or not np.all(np.isfinite(R)):
        return None, False
    X = solve_triangular(R, Qm.T @ b, lower=False)
    return X.T, True


def split_operators(O, r):
    """Ahat = O[:, :r], Hhat = O[:, r:r+s], chat = O[:, r+s]."""
    s = r * (r + 1) // 2
    return O[:, :r], O[:, r:r + s], O[:, r + s]


def rom_step_discrete(O, r, q):
    """One step of the discrete quadratic ROM, eq. ROM_quad_time_discrete."""
    A, H, c = split_operators(O, r)
    return A @ q + H @ qhat_sq(q) + c


def rom_rhs(O, r, q):
    """Right-hand side of the continuous quadratic ROM, eq. ROM_quad_time_cont."""
    A, H, c = split_operators(O, r)
    return A @ q + H @ qhat_sq(q) + c


def rk4_step(O, r, q, dt):
    """Classical fourth-order Runge-Kutta step of the continuous ROM."""
    k1 = rom_rhs(O, r, q)
    k2 = rom_rhs(O, r, q + 0.5 * dt * k1)
    k3 = rom_rhs(O, r, q + 0.5 * dt * k2)
    k4 = rom_rhs(O, r, q + dt * k3)
    return q + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def rollout(O, r, q0, n_steps, mode="discrete", dt=1.0):
    """Trajectory of n_steps states (the initial state included), rows = time."""
    Qt = np.zeros((n_steps, r))
    Qt[0] = q0
    with np.errstate(all="ignore"):
        for t in range(n_steps - 1):
            if mode == "discrete":
                Qt[t + 1] = rom_step_discrete(O, r, Qt[t])
            else:
                Qt[t + 1] = rk4_step(O, r, Qt[t], dt)
    return Qt


def train_error(Qhat_train, Qtilde_train):
    """Max over time of the relative 2-norm error over modes (Step IV's training error)."""
    num = np.sum((Qtilde_train - Qhat_train) ** 2, axis=1)
    den = np.sum(Qhat_train ** 2, axis=1)
    return float(np.max(np.sqrt(num / den)))


def growth_ratio(Qtilde, mean_train, max_diff_train):
    """Max deviation of the rollout from the training mean over the training one."""
    return float(np.max(np.abs(Qtilde - mean_train)) / np.max(max_diff_train))


def learn(Qhat, r_list, beta1s, beta2s, n_steps, mode="discrete", dt=1.0,
          max_growth=1.2, keep_trajectories=False):
    """Grid search of Step IV over every (r, beta1, beta2), r-major then beta1 then beta2.

    Qhat: (r_max, k) reduced data.  Returns dict with per-candidate arrays train_err,
    growth, valid (bool), chol_ok, the best flat index (-1 if none valid), best r, beta1,
    beta2, best operators O (r x d) and best trajectory (n_steps x r).
    """
    Qhat = np.asarray(Qhat, dtype=np.float64)
    k = Qhat.shape[1]
    cands = [(r, b1, b2) for r in r_list for b1 in beta1s for b2 in beta2s]
    P = len(cands)
    err = np.full(P, np.inf)
    gro = np.full(P, np.inf)
    valid = np.zeros(P, dtype=bool)
    chol_ok = np.zeros(P, dtype=bool)
    ops, trajs = {}, {}
    cache = {}
    for idx, (r, b1, b2) in enumerate(cands):
        if r not in cache:
            Dhat, Y = learning_data(Qhat, r, mode, dt)
            G, B = normal_equations(Dhat, Y)
            Qr = Qhat[:r, :].T
            mean_train = np.mean(Qr, axis=0)
            max_diff_train = np.max(np.abs(Qr - mean_train), axis=0)
            cache[r] = (G, B, Qr, mean_train, max_diff_train)
        G, B, Qr, mean_train, max_diff_train = cache[r]
        O, ok = solve_cholesky(G, B, regulariser(r, b1, b2))
        chol_ok[idx] = ok
        if not ok:
            continue
        Qt = rollout(O, r, Qr[0], n_steps, mode, dt)
        ops[idx] = O
        if keep_trajectories:
            trajs[idx] = Qt
        if not np.all(np.isfinite(Qt)):
            continue
        err[idx] = train_error(Qr[:k], Qt[:k])
        gro[idx] = growth_ratio(Qt, mean_train, max_diff_train)
        valid[idx] = gro[idx] < max_growth
    best = -1
    for idx in range(P):
        if valid[idx] and (best < 0 or err[idx] < err[best]):
            best = idx
    out = dict(train_err=err, growth=gro, valid=valid, chol_ok=chol_ok, best=best,
               candidates=cands, ops=ops, trajs=trajs)
    if best >= 0:
        r, b1, b2 = cands[best]
        out.update(r=r, beta1=b1, beta2=b2, O=ops[best],
                   Qtilde=rollout(ops[best], r, Qhat[:r, 0], n_steps, mode, dt))
    return out


# --------------------------------------------------------------------------------------
# Step V (Section 3.6): the reduced solution back in the original coordinates.
# --------------------------------------------------------------------------------------
def pod_basis_rows(Q, Tr, rows):
    """Rows of the rank-r POD basis V_r = Q T_r (eq. MoS_POD_basis), at the given row indices
    of the transformed snapshot matrix Q (n x k)."""
    Q64 = np.asarray(Q, dtype=np.float64)
    return Q64[np.asarray(rows, dtype=np.int64), :] @ np.asarray(Tr, dtype=np.float64)


def lift(Q, Tr, Qtilde, rows, row_mean=None, var_scale=None, var_row_offsets=None):
    """Step V: the reduced solution Qtilde (r x n_t, column t = state t) lifted at the given rows:
    V_r[rows] Qtilde, then the inverse of Step II's transform, x = (scale of the row's variable)
    * y + (the row's temporal mean); either part is skipped when its argument is None.
    Returns (len(rows), n_t)."""
    rows = np.asarray(rows, dtype=np.int64)
    Y = pod_basis_rows(Q, Tr, rows) @ np.asarray(Qtilde, dtype=np.float64)
    if var_scale is not None:
        var = np.searchsorted(np.asarray(var_row_offsets), rows, side="right") - 1
        Y = Y * np.asarray(var_scale, dtype=np.float64)[var][:, None]
    if row_mean is not None:
        Y = Y + np.asarray(row_mean, dtype=np.float64)[rows][:, None]
    return Y


def pipeline(Q, var_row_offsets, r_list=None, beta1s=(), beta2s=(), n_steps=0,
             mode="discrete", dt=1.0, tau=0.9996, max_growth=1.2):
    """Steps II-IV end to end: transform, Gram, reduce, learn."""
    Qt, mean, scale, flags = transform(Q, var_row_offsets)
    D = gram(Qt)
    r_max = max(r_list) if r_list else 0
    red = reduce(D, tau=tau, r_fixed=0 if not r_list else r_max, r_cap=r_max or None)
    r_list = r_list or [red["r"]]
    res = learn(red["Qhat"], r_list, beta1s, beta2s, n_steps, mode, dt, max_growth)
    return dict(Q=Qt, mean=mean, scale=scale, flags=flags, D=D, reduce=red, learn=res)
