"""Seeded synthetic inputs for the dOpInf hot path (shared by the tests, the bench and the
checker; holds none of the method's arithmetic).

The paper's Navier-Stokes snapshots and the detonation data are not available, so every
input is generated from a seeded quadratic dynamical system that is lifted to n rows:

* generating system (dimension r_true): x' = A x + H(x, x) + c.  A = omega (G - G^T) / (2 sqrt r)
  - 0.1 I with G Gaussian: a rotation with frequencies of order omega whose symmetric part
  is exactly -0.1 I, which bounds every trajectory together with an energy-preserving H
  (x^T H(x, x) = 0 for all x; H = S - sym3(S) for a random S symmetric in its last two
  indices).  c has entries N(0, 0.01) (variance 0.01).  The system is integrated with
  classical RK4 at step dt from x0 ~ N(0, 1); every stride-th state is one snapshot, so
  the snapshot spacing is dt * stride;
* lift: Q = L X + noise, L an n x r_true matrix with orthonormal columns (QR of a
  Gaussian), optionally re-shaped so that the squared singular values of L X decay as
  i^-p; the noise is Gaussian with standard deviation noise_rel times the RMS entry of
  L X; each variable block of rows is multiplied by its own scale factor.

Named workloads (sizes of the paper's example and of the GB300 benchmark set):
  small     n = 2 x 2048,   k = 200,  r_true = 6
  stepflow  n = 3 x 400000, k = 600,  r_true = 40, variable scales 1e-2, 1e1, 1e3
  rdre      n = 8 x 1.5e6,  k = 2000, r_true = 120, FP32, lambda_i ~ i^-3, noise 1e-6
  paper     n = 2 x 146339, k = 600,  r_true = 12 (the Navier-Stokes example's shape)
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass
class Workload:
    name: str
    n_vars: int
    n_per_var: int
    k: int
    r_true: int
    dt: float = 1e-3
    stride: int = 10
    omega: float = 2 * np.pi
    h_scale: float = 1.0
    noise_rel: float = 1e-4
    var_scales: tuple = ()
    decay: float = 0.0          # 0: plain lift; p > 0: squared singular values ~ i^-p
    dtype: str = "f64"
    r_list: tuple = ()
    n_beta1: int = 4
    n_beta2: int = 4
    beta1_range: tuple = (-8.0, 2.0)
    beta2_range: tuple = (-8.0, 2.0)
    n_steps: int = 1000
    mode: str = "discrete"
    seed: int = 1234

    @property
    def n(self):
        return self.n_vars * self.n_per_var

    @property
    def snap_dt(self):
        """Time between snapshots (the step of continuous-mode rollouts)."""
        return self.dt * self.stride

    def var_row_offsets(self):
        return np.arange(self.n_vars + 1, dtype=np.int64) * self.n_per_var

    def beta1s(self):
        return logspace(self.beta1_range[0], self.beta1_range[1], self.n_beta1)

    def beta2s(self):
        return logspace(self.beta2_range[0], self.beta2_range[1], self.n_beta2)


WORKLOADS = {
    "small": Workload("small", 2, 2048, 200, 6, r_list=(6,), n_steps=1000, seed=1234),
    "stepflow": Workload("stepflow", 3, 400_000, 600, 40, var_scales=(1e-2, 1e1, 1e3),
                         r_list=(10, 20, 30), n_beta1=8, n_beta2=8,
                         beta1_range=(-10.0, 0.0), beta2_range=(-4.0, 4.0),
                         n_steps=5000, mode="continuous", seed=1235),
    "rdre": Workload("rdre", 8, 1_500_000, 2000, 120, noise_rel=1e-6, decay=3.0,
                     dtype="f32", r_list=(100,), seed=1236),
    "paper": Workload("paper", 2, 146_339, 600, 12, r_list=(10,), n_beta1=8, n_beta2=8,
                      beta1_range=(-10.0, 0.0), beta2_range=(-4.0, 4.0), n_steps=1200,
                      seed=1237),
}


def logspace(lo, hi, num):
    """num values 10**e, e evenly spaced on [lo, hi] with both ends included."""
    if num == 1:
        return np.array([10.0 ** lo])
    e = lo + (hi - lo) * np.arange(num) / (num - 1)
    return 10.0 ** e


def quadratic_system(r, rng, omega=2 * np.pi, h_scale=1.0):
    """(A, H3, c): A (r, r), H3 (r, r, r) energy preserving and symmetric in (j, k), c (r,)."""
    G = rng.standard_normal((r, r))
    A = omega * (G - G.T) / (2.0 * np.sqrt(r)) - 0.1 * np.eye(r)
    S = rng.standard_normal((r, r, r)) * (h_scale / r)
    S = 0.5 * (S + S.transpose(0, 2, 1))
    sym = (S + S.transpose(0, 2, 1) + S.transpose(1, 0, 2) + S.transpose(1, 2, 0)
           + S.transpose(2, 0, 1) + S.transpose(2, 1, 0)) / 6.0
    H3 = S - sym
    c = rng.standard_normal(r) * 0.1
    return A, H3, c


def unique_quadratic(H3):
    """Matrix form (r, r(r+1)/2) of a tensor symmetric in its last two indices, columns
    ordered (i, j) with i <= j, i-major: the entry multiplies x_i x_j."""
    r = H3.shape[0]
    cols = []
    for i in range(r):
        for j in range(i, r):
            cols.append(H3[:, i, j] * (1.0 if i == j else 2.0))
    return np.stack(cols, axis=1)


def _field(A, H3, c, x):
    return A @ x + np.einsum("ijk,j,k->i", H3, x, x) + c


def integrate_rk4(A, H3, c, x0, dt, k, stride=1):
    """k states (x0 included, every stride-th RK4 step) of the generating system."""
    X = np.empty((A.shape[0], k))
    x = np.array(x0, dtype=np.float64)
    for t in range(k):
        X[:, t] = x
        for _ in range(stride):
            k1 = _field(A, H3, c, x)
            k2 = _field(A, H3, c, x + 0.5 * dt * k1)
            k3 = _field(A, H3, c, x + 0.5 * dt * k2)
            k4 = _field(A, H3, c, x + dt * k3)
            x = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return X


def trajectory(w: Workload):
    """Reduced trajectory X (r_true, k) and the generating system of a workload."""
    rng = np.random.default_rng(w.seed)
    A, H3, c = quadratic_system(w.r_true, rng, w.omega, w.h_scale)
    x0 = rng.standard_normal(w.r_true)
    X = integrate_rk4(A, H3, c, x0, w.dt, w.k, w.stride)
    return X, (A, H3, c)


def lift_matrix_small(w: Workload, X, rng):
    """Dense lift L (n, r_true) in numpy, for workloads that fit in host memory."""
    G = rng.standard_normal((w.n, w.r_true))
    L, _ = np.linalg.qr(G)
    if w.decay > 0:
        L = L @ _decay_shaper(X, w.decay)
    return L


def _decay_shaper(X, p):
    """M with M X having squared singular values proportional to i^-p."""
    U, S, _ = np.linalg.svd(X, full_matrices=False)
    s = np.arange(1, len(S) + 1, dtype=np.float64) ** (-p / 2.0)
    return U @ np.diag(s * S[0] / S) @ U.T


def snapshots_numpy(w: Workload):
    """Full snapshot matrix Q (n, k) in host memory (float64 or float32) plus metadata."""
    X, sysm = trajectory(w)
    rng = np.random.default_rng(w.seed + 1_000_003)
    L = lift_matrix_small(w, X, rng)
    Q = L @ X
    if w.noise_rel > 0:
        rms = np.linalg.norm(Q) / np.sqrt(Q.size)
        Q += rng.standard_normal(Q.shape) * (w.noise_rel * rms)
    if w.var_scales:
        for j, s in enumerate(w.var_scales):
            Q[j * w.n_per_var:(j + 1) * w.n_per_var, :] *= s
    Q = np.asfortranarray(Q.astype(np.float32 if w.dtype == "f32" else np.float64))
    return Q, dict(X=X, L=L, system=sysm)


def snapshots_torch(w: Workload, device, col_major=True, traj=None):
    """The same construction on a torch device, for workloads too large for the host.

    Returns Q as a torch tensor of shape (k, n) whose row t is snapshot t (i.e. the
    column-major n x k matrix with leading dimension n).  Draws come from torch's
    generator seeded with the workload seed, so values differ from snapshots_numpy.
    traj: the trajectory of w as trajectory(w) returns it, when it was formed elsewhere
    (it is the host-side part of the cost, a few seconds at r_true = 40, k = 1500).
    """
    import torch
    X, _ = trajectory(w) if traj is None else traj
    g = torch.Generator(device=device)
    g.manual_seed(w.seed)
    G = torch.randn(w.n, w.r_true, generator=g, device=device, dtype=torch.float64)
    # orthonormal columns by CholeskyQR applied twice (matrix products on the device, the
    # r_true x r_true Cholesky factor on the host)
    for _ in range(2):
        R = np.linalg.cholesky((G.T @ G).cpu().numpy()).T
        G = G @ torch.from_numpy(np.linalg.inv(R)).to(device)
    L = G
    Mn = X if w.decay <= 0 else _decay_shaper(X, w.decay) @ X
    M = torch.from_numpy(Mn).to(device)
    noise_std = w.noise_rel * np.linalg.norm(Mn) / np.sqrt(w.n * w.k)  # ||L M||_F = ||M||_F
    dt = torch.float32 if w.dtype == "f32" else torch.float64
    QT = torch.empty(w.k, w.n, device=device, dtype=dt)
    sc = torch.ones(w.n, device=device, dtype=torch.float64)
    if w.var_scales:
        for j, s in enumerate(w.var_scales):
            sc[j * w.n_per_var:(j + 1) * w.n_per_var] = s
    step = max(1, (1 << 27) // max(w.n, 1))
    for t0 in range(0, w.k, step):
        t1 = min(w.k, t0 + step)
        blk = (L @ M[:, t0:t1]).T
        if w.noise_rel > 0:
            blk += torch.randn(blk.shape, generator=g, device=device,
                               dtype=torch.float64) * noise_std
        QT[t0:t1] = (blk * sc).to(dt)
    return QT
