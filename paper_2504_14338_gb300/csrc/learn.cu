// Step IV of dOpInf (Section 3.5): quadratic Operator Inference with a grid search over the
// regularisation pairs (eqs. OpInf_reg, OpInf_data_matrices_discrete) and over reduced
// dimensions r, the training error / growth selection of Step IV, all on the GPU.
//
// Per r (a principal block of the reduced data Qhat):
//   build_features  data matrix Dhat = [q, (q_i q_j)_{i<=j}, 1] (K x d, column-major) and the
//                   targets Y (K x r): the shifted snapshots (discrete) or central differences
//                   (continuous);
//   tn_product      G = Dhat^T Dhat (symmetric) and B = Dhat^T Y in FP64;
//   train_stats     temporal mean mu of the reference and max_{t<k,i} |qhat - mu|;
// Then schur_solve (schur.cu) solves (G + diag(reg)) O^T = B for every (r, beta1, beta2) by
// block elimination of the quadratic unknowns, shared across beta1, and the rollouts run every
// candidate (a thread-block cluster each; rollout.cu) with the fused training error / growth
// epilogue: one launch per r, largest first, chained by programmatic dependent launch so that
// they run side by side, in the arithmetic set by dopinf_tune_rollout_arith (with double-word
// FP32, an FP64 pass over the candidates it hands back follows).  Then
// select_best takes the lowest training error among valid candidates (lowest index on ties).
// Everything else is FP64.
#include "common.cuh"

#include <algorithm>
#include <math.h>
#include <vector>

namespace dopinf {
namespace {

constexpr int LB = 256;

__global__ void __launch_bounds__(LB) build_features(const double* __restrict__ Qhat, int64_t ldqh, int r, int d,
                                                     int64_t K, int64_t t0, int mode, double dt,
                                                     double* __restrict__ Dh, double* __restrict__ Y) {
  const int s = d - r - 1;
  const int64_t nD = K * d, nY = K * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nD + nY; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nD) {
      const int64_t tp = e % K;
      const int a = (int)(e / K);
      const double* q = Qhat + (t0 + tp) * ldqh;
      double v;
      if (a < r) {
        v = q[a];
      } else if (a < r + s) {
        int idx = a - r, i = 0;
        while (idx >= r - i) {
          idx -= r - i;
          ++i;
        }
        v = q[i] * q[i + idx];
      } else {
        v = 1.0;
      }
      Dh[e] = v;
    } else {
      const int64_t f = e - nD;
      const int64_t tp = f % K;
      const int i = (int)(f / K);
      const int64_t t = t0 + tp;
      double v;
      if (mode == DOPINF_DISCRETE)
        v = Qhat[i + (t + 1) * ldqh];
      else
        v = (Qhat[i + (t + 1) * ldqh] - Qhat[i + (t - 1) * ldqh]) / (2.0 * dt);
      Y[f] = v;
    }
  }
}

// Per r: the temporal mean mu of the reference data, denom = max_{t<k,i} |qhat - mu| (the
// growth ratio's denominator), and 1 / ||qhat_t||^2 for every t < k (the training error's
// denominators, so that the rollouts multiply instead of dividing on their critical path).
__global__ void __launch_bounds__(LB) train_stats(const double* __restrict__ Qhat, int64_t ldqh, int r, int64_t k,
                                                  double* __restrict__ mu, double* __restrict__ denom,
                                                  double* __restrict__ inv_den) {
  for (int64_t t = threadIdx.x; t < k; t += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += Qhat[i + t * ldqh] * Qhat[i + t * ldqh];
    inv_den[t] = 1.0 / s;
  }
  __shared__ double sh[LB];
  double dev = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    double s = 0.0;
    for (int64_t t = 0; t < k; ++t) s += Qhat[i + t * ldqh];
    const double m = s / (double)k;
    mu[i] = m;
    for (int64_t t = 0; t < k; ++t) dev = fmax(dev, fabs(Qhat[i + t * ldqh] - m));
  }
  sh[threadIdx.x] = dev;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) mx = fmax(mx, sh[i]);
    *denom = mx;
  }
}

__global__ void select_best(const double* err, const int* status, int n_cand, int* best) {
  if (threadIdx.x != 0) return;
  int b = -1;
  for (int c = 0; c < n_cand; ++c)
    if (status[c] == 0 && (b < 0 || err[c] < err[b])) b = c;
  *best = b;
}

constexpr int kMaxR = 64;  // entries of the r list

// Workspace layout, one for the size query (base == nullptr) and for the entry point.
struct LearnWs {
  SchurUnit* units;
  SchurCand* cands;
  RolloutCand* roll;
  double *mu, *denom, *invden, *Dh, *Y;
  double *G[kMaxR], *B[kMaxR], *E[kMaxR], *S[kMaxR], *O[kMaxR];
  double* qr;          // QR solver: one stacked system per candidate of an r (reused across r)
  size_t qr_stride;    // doubles per candidate slice
  size_t O_off[kMaxR];  // byte offset of O[i] in the workspace
  int r_stride;  // largest r of the list: stride of the per-r vectors (mu)
  int64_t k_stride;  // snapshots: stride of the per-r training-error denominators
  int *best, *unit_fail;
  void* tn;
  size_t tn_bytes, used;
};

int g_solver = DOPINF_SOLVE_CHOLESKY;  // tunable: solver of the regularised problems
constexpr int kQrMaxD = 1024;          // widest operator the QR solver takes (one CTA per candidate)

LearnWs carve_learn(void* base, int64_t K, const int* r_list, int n_r, int n_b1, int n_b2) {
  const int n_pairs = n_b1 * n_b2;
  Carver c(base);
  LearnWs w;
  int d_max = 0, r_max = 0;
  for (int i = 0; i < n_r; ++i) {
    if (dim_d(r_list[i]) > d_max) d_max = dim_d(r_list[i]);
    if (r_list[i] > r_max) r_max = r_list[i];
  }
  const int n_cand = n_r * n_pairs;
  w.r_stride = r_max;
  w.units = c.take<SchurUnit>((size_t)n_r * n_b2);
  w.cands = c.take<SchurCand>(n_cand);
  w.roll = c.take<RolloutCand>(n_cand);
  w.unit_fail = c.take<int>((size_t)n_r * n_b2);
  w.mu = c.take<double>((size_t)n_r * r_max);
  w.denom = c.take<double>(n_r);
  w.k_stride = K + 1;
  w.invden = c.take<double>((size_t)n_r * (K + 1));
  w.best = c.take<int>(1);
  w.Dh = c.take<double>((size_t)K * d_max);
  w.Y = c.take<double>((size_t)K * r_max);
  for (int i = 0; i < n_r; ++i) {
    const size_t r = r_list[i], d = dim_d(r_list[i]);
    w.G[i] = c.take<double>(d * d);
    w.B[i] = c.take<double>(d * r);
    w.E[i] = c.take<double>((size_t)n_b2 * schur_unit_doubles((int)r));
    w.S[i] = c.take<double>((size_t)n_pairs * schur_cand_doubles((int)r));
    w.O_off[i] = c.used;
    w.O[i] = c.take<double>((size_t)n_pairs * r * d);
  }
  size_t tb = 0;
  for (int i = 0; i < n_r; ++i) {
    const int r = r_list[i], d = dim_d(r);
    size_t a = tn_workspace(K, d, d, 1), b = tn_workspace(K, d, r, 0);
    tb = a > tb ? a : tb;
    tb = b > tb ? b : tb;
  }
  w.tn_bytes = tb;
  w.tn = c.take<char>(tb);
  w.qr = nullptr;
  w.qr_stride = 0;
  if (g_solver == DOPINF_SOLVE_QR) {
    for (int i = 0; i < n_r; ++i) {
      const size_t q = qr_solve_doubles(K, r_list[i]);
      w.qr_stride = q > w.qr_stride ? q : w.qr_stride;
    }
    w.qr = c.take<double>(w.qr_stride * (size_t)n_pairs);
  }
  w.used = c.used;
  return w;
}

}  // namespace
}  // namespace dopinf

using namespace dopinf;

static int64_t learn_rows(int64_t k, int mode) { return mode == DOPINF_DISCRETE ? k - 1 : k - 2; }

DOPINF_API size_t dopinf_learn_workspace(int r_max, int64_t k, const int* r_list, int n_r, int n_b1, int n_b2) {
  (void)r_max;
  if (!r_list || n_r < 1 || n_r > kMaxR || n_b1 < 1 || n_b2 < 1 || k < 3) return 0;
  return carve_learn(nullptr, k - 1, r_list, n_r, n_b1, n_b2).used;
}

DOPINF_API size_t dopinf_learn_operator_offset(int64_t k, const int* r_list, int n_r, int n_b1, int n_b2, int cand) {
  if (!r_list || n_r < 1 || n_r > kMaxR || n_b1 < 1 || n_b2 < 1 || k < 3) return (size_t)-1;
  const int n_pairs = n_b1 * n_b2;
  if (cand < 0 || cand >= n_r * n_pairs) return (size_t)-1;
  for (int i = 0; i < n_r; ++i)
    if (r_list[i] < 1 || r_list[i] > 255) return (size_t)-1;
  const LearnWs w = carve_learn(nullptr, k - 1, r_list, n_r, n_b1, n_b2);
  const int ir = cand / n_pairs, p = cand % n_pairs;
  const size_t r = r_list[ir], d = dim_d(r_list[ir]);
  return w.O_off[ir] + (size_t)p * r * d * sizeof(double);
}

namespace dopinf {
namespace {

constexpr int kMaxB = 64;  // entries of each beta list

// The grid as kernel parameters, so that the candidate tables are built on the device (no host
// copies: the launch sequence can be captured into a CUDA graph).
struct LearnGrid {
  int n_r, n_b1, n_b2;
  int r_list[kMaxR];
  double beta1[kMaxB], beta2[kMaxB];
  LearnWs w;
};

__global__ void build_tables(const LearnGrid g) {
  const int n_pairs = g.n_b1 * g.n_b2;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < g.n_r * g.n_b2; u += gridDim.x * blockDim.x) {
    const int ir = u / g.n_b2, i2 = u % g.n_b2;
    const int r = g.r_list[ir], sq = r * (r + 1) / 2;
    SchurUnit U;
    U.G = g.w.G[ir];
    U.B = g.w.B[ir];
    U.E = g.w.E[ir] + (size_t)i2 * ((size_t)(sq + 2 * r + 1) * (sq + 2 * r + 1));
    U.b2 = g.beta2[i2];
    U.r = r;
    U.d = dim_d(r);
    U.s = sq;
    U.m = r + 1;
    U.N = sq + 2 * r + 1;
    U.unit = u;
    g.w.units[u] = U;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.n_r * n_pairs; c += gridDim.x * blockDim.x) {
    const int ir = c / n_pairs, p = c % n_pairs, i2 = p % g.n_b2;
    const int r = g.r_list[ir], d = dim_d(r), sq = r * (r + 1) / 2, N = sq + 2 * r + 1;
    SchurCand S;
    S.E = g.w.E[ir] + (size_t)i2 * ((size_t)N * N);
    S.O = g.w.O[ir] + (size_t)p * r * d;
    S.scratch = g.w.S[ir] + (size_t)p * ((size_t)(r + 1) * (r + 1) + (size_t)(r + 1) * r);
    S.b1 = g.beta1[p / g.n_b2];
    S.r = r;
    S.s = sq;
    S.m = r + 1;
    S.N = N;
    S.unit = ir * g.n_b2 + i2;
    S.cand = c;
    g.w.cands[c] = S;
    RolloutCand R;
    R.O = S.O;
    R.ldo = r;
    R.r = r;
    R.d = d;
    R.cand = c;
    R.mu = g.w.mu + (size_t)ir * g.w.r_stride;
    R.denom = g.w.denom + ir;
    R.inv_den = g.w.invden + (size_t)ir * g.w.k_stride;
    g.w.roll[c] = R;
  }
}

// The operators of the best candidate into O_best (r_max x d_max, ld r_max); best < 0 flags
// DOPINF_FLAG_NO_STABLE.  The candidate's r and d come from the table.
__global__ void gather_best(const int* best, const SchurCand* cands, int r_max, double* O_best, int* best_out,
                            unsigned* flags) {
  const int b = *best;
  if (threadIdx.x == 0 && best_out) *best_out = b;
  if (b < 0) {
    if (threadIdx.x == 0 && flags) atomicOr(flags, DOPINF_FLAG_NO_STABLE);
    return;
  }
  const SchurCand c = cands[b];
  const int r = c.r, d = dim_d(r);
  for (int e = threadIdx.x; e < r * d; e += blockDim.x) O_best[(e % r) + (size_t)(e / r) * r_max] = c.O[e];
}

// Checks of every argument; the largest r and d of the list on success.
int learn_check(const double* Qhat, int r_max, int64_t k, int64_t ldqh, const int* r_list, int n_r,
                const double* beta1, int n_b1, const double* beta2, int n_b2, int mode, double dt, int64_t n_steps,
                double max_growth, const double* train_err, const double* growth, const int* cand_status,
                const double* O_best, void* ws, size_t ws_bytes, int* r_used, int* d_max) {
  if (!Qhat || r_max < 1 || ldqh < r_max || !r_list || n_r < 1 || n_r > kMaxR || !beta1 || !beta2 || n_b1 < 1 ||
      n_b2 < 1 || !train_err || !growth || !cand_status || !O_best)
    return DOPINF_E_ARG;
  if (n_b1 > kMaxB || n_b2 > kMaxB) return DOPINF_E_UNSUPPORTED;
  if (mode != DOPINF_DISCRETE && mode != DOPINF_CONTINUOUS_RK4) return DOPINF_E_ARG;
  if (mode == DOPINF_CONTINUOUS_RK4 && !(dt > 0.0)) return DOPINF_E_ARG;
  const int64_t K = learn_rows(k, mode);
  if (K < 1 || n_steps < k || !(max_growth > 0.0)) return DOPINF_E_ARG;
  *d_max = 0;
  *r_used = 0;
  for (int i = 0; i < n_r; ++i) {
    if (r_list[i] < 1 || r_list[i] > r_max || r_list[i] > 255) return DOPINF_E_ARG;
    *d_max = dim_d(r_list[i]) > *d_max ? dim_d(r_list[i]) : *d_max;
    *r_used = r_list[i] > *r_used ? r_list[i] : *r_used;
  }
  for (int i = 0; i < n_b1; ++i)
    if (!(beta1[i] >= 0.0)) return DOPINF_E_ARG;
  for (int i = 0; i < n_b2; ++i)
    if (!(beta2[i] >= 0.0)) return DOPINF_E_ARG;
  if (!ws || ws_bytes < dopinf_learn_workspace(r_max, k, r_list, n_r, n_b1, n_b2) || misaligned(ws))
    return DOPINF_E_ARG;
  // rollouts: every r must fit one of the two kernels (r <= 92); the QR solver: d <= 1024
  for (int i = 0; i < n_r; ++i) {
    if (!rollout_supported(r_list[i]) || !rollout_shape(r_list[i])) return DOPINF_E_UNSUPPORTED;
    if (g_solver == DOPINF_SOLVE_QR && dim_d(r_list[i]) > kQrMaxD) return DOPINF_E_UNSUPPORTED;
  }
  return DOPINF_OK;
}

// The whole learn step on the stream, no synchronisation, no host copies.  ev (optional): 4
// events recorded around the data + normal equations, the solves and the rollouts.
int learn_launch(const double* Qhat, int r_max, int64_t k, int64_t ldqh, const int* r_list, int n_r,
                 const double* beta1, int n_b1, const double* beta2, int n_b2, int mode, double dt, int64_t n_steps,
                 double max_growth, double* train_err, double* growth, int* cand_status, int64_t* cand_steps,
                 int* best_dev, double* O_best, unsigned* dev_flags, int r_used, int d_max, void* ws,
                 cudaStream_t st, cudaEvent_t* ev) {
  const int64_t K = learn_rows(k, mode);
  // the workspace is laid out for K = k - 1 rows, which covers both modes
  LearnWs w = carve_learn(ws, k - 1, r_list, n_r, n_b1, n_b2);
  const int n_pairs = n_b1 * n_b2, n_cand = n_r * n_pairs, n_units = n_r * n_b2;
  // candidate c = (ir * n_b1 + i1) * n_b2 + i2; unit = ir * n_b2 + i2
  LearnGrid g;
  g.n_r = n_r;
  g.n_b1 = n_b1;
  g.n_b2 = n_b2;
  for (int i = 0; i < n_r; ++i) g.r_list[i] = r_list[i];
  for (int i = 0; i < n_b1; ++i) g.beta1[i] = beta1[i];
  for (int i = 0; i < n_b2; ++i) g.beta2[i] = beta2[i];
  g.w = w;
  build_tables<<<(n_cand + 255) / 256, 256, 0, st>>>(g);
  DOPINF_TRY(launch_status());
  // the unit table's sizes on the host too: they set the grids of the panel launches
  std::vector<SchurUnit> un(n_units);
  for (int u = 0; u < n_units; ++u) {
    const int r = r_list[u / n_b2], sq = r * (r + 1) / 2;
    un[u].r = r;
    un[u].s = sq;
    un[u].m = r + 1;
    un[u].N = sq + 2 * r + 1;
  }
  if (ev) DOPINF_CUDA(cudaEventRecord(ev[0], st));
  const int64_t t0 = mode == DOPINF_DISCRETE ? 0 : 1;
  for (int ir = 0; ir < n_r; ++ir) {
    const int r = r_list[ir], d = dim_d(r);
    const int64_t tot = K * (d + r);
    const unsigned blocks = (unsigned)((tot + LB - 1) / LB < 4096 ? (tot + LB - 1) / LB : 4096);
    build_features<<<blocks, LB, 0, st>>>(Qhat, ldqh, r, d, K, t0, mode, dt, w.Dh, w.Y);
    DOPINF_TRY(launch_status());
    if (g_solver == DOPINF_SOLVE_QR) {
      // this r's candidates from the stacked systems, before the next r rebuilds Dhat
      DOPINF_TRY(qr_solve(w.Dh, w.Y, K, r, w.units, w.cands, ir * n_pairs, n_pairs, w.qr, w.qr_stride, cand_status,
                          st));
    } else {
      DOPINF_TRY(tn_product(w.Dh, K, w.Dh, K, DOPINF_F64, K, d, d, 1, 0, w.G[ir], d, w.tn, w.tn_bytes, st));
      DOPINF_TRY(tn_product(w.Dh, K, w.Y, K, DOPINF_F64, K, d, r, 0, 0, w.B[ir], d, w.tn, w.tn_bytes, st));
    }
    train_stats<<<1, LB, 0, st>>>(Qhat, ldqh, r, k, w.mu + (size_t)ir * w.r_stride, w.denom + ir,
                                  w.invden + (size_t)ir * w.k_stride);
    DOPINF_TRY(launch_status());
  }
  if (ev) DOPINF_CUDA(cudaEventRecord(ev[1], st));
  if (g_solver != DOPINF_SOLVE_QR)
    DOPINF_TRY(schur_solve(w.units, un.data(), n_units, w.cands, n_cand, w.unit_fail, cand_status, st));
  if (ev) DOPINF_CUDA(cudaEventRecord(ev[2], st));
  RolloutBatch bt = {};
  bt.cands = w.roll;
  bt.n_cand = n_cand;
  bt.r_max = r_used;
  bt.d_max = d_max;
  bt.mode = mode;
  bt.dt = dt;
  bt.n_steps = n_steps;
  bt.q0 = Qhat;
  bt.metrics = 1;
  bt.Qhat = Qhat;
  bt.ldqh = ldqh;
  bt.k = k;
  bt.max_growth = max_growth;
  bt.train_err = train_err;
  bt.growth = growth;
  bt.status = cand_status;
  bt.steps = cand_steps;
  {
    // one launch per r, largest r (longest evaluations) first; each later launch is chained
    // behind the one before by programmatic dependent launch, so all run side by side
    int order[kMaxR];
    for (int i = 0; i < n_r; ++i) order[i] = i;
    std::sort(order, order + n_r, [&](int a, int b) { return r_list[a] > r_list[b] || (r_list[a] == r_list[b] && a < b); });
    bt.arith = rollout_arith();
    for (int j = 0; j < n_r; ++j) {
      const int ir = order[j];
      DOPINF_TRY(launch_rollouts_rank(bt, ir * n_pairs, n_pairs, r_list[ir], j > 0, st));
    }
    if (bt.arith == DOPINF_ROLLOUT_DW) {
      // the FP64 pass over whatever the double-word pass handed back (usually nothing: its
      // CTAs return at once); it starts once every double-word launch has completed
      bt.arith = DOPINF_ROLLOUT_FP64;
      bt.redo = 1;
      for (int j = 0; j < n_r; ++j) {
        const int ir = order[j];
        DOPINF_TRY(launch_rollouts_rank(bt, ir * n_pairs, n_pairs, r_list[ir], j > 0, st));
      }
    }
  }
  if (ev) DOPINF_CUDA(cudaEventRecord(ev[3], st));
  select_best<<<1, 32, 0, st>>>(train_err, cand_status, n_cand, w.best);
  gather_best<<<1, 256, 0, st>>>(w.best, w.cands, r_max, O_best, best_dev, dev_flags);
  return launch_status();
}

}  // namespace
}  // namespace dopinf

DOPINF_API int dopinf_learn_async(const double* Qhat, int r_max, int64_t k, int64_t ldqh, const int* r_list, int n_r,
                                  const double* beta1, int n_b1, const double* beta2, int n_b2, int mode, double dt,
                                  int64_t n_steps, double max_growth, double* train_err, double* growth,
                                  int* cand_status, int64_t* cand_steps, int* best_dev, double* O_best,
                                  unsigned* dev_flags, void* ws, size_t ws_bytes, void* stream) {
  if (!best_dev || !dev_flags) return DOPINF_E_ARG;
  int r_used = 0, d_max = 0;
  DOPINF_TRY(learn_check(Qhat, r_max, k, ldqh, r_list, n_r, beta1, n_b1, beta2, n_b2, mode, dt, n_steps, max_growth,
                         train_err, growth, cand_status, O_best, ws, ws_bytes, &r_used, &d_max));
  return learn_launch(Qhat, r_max, k, ldqh, r_list, n_r, beta1, n_b1, beta2, n_b2, mode, dt, n_steps, max_growth,
                      train_err, growth, cand_status, cand_steps, best_dev, O_best, dev_flags, r_used, d_max,
                      ws, as_stream(stream), nullptr);
}

DOPINF_API int dopinf_learn(const double* Qhat, int r_max, int64_t k, int64_t ldqh, const int* r_list, int n_r,
                            const double* beta1, int n_b1, const double* beta2, int n_b2, int mode, double dt,
                            int64_t n_steps, double max_growth, double* train_err, double* growth, int* cand_status,
                            int64_t* cand_steps, int* best_out, double* O_best, double* stage_ms, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!best_out) return DOPINF_E_ARG;
  int r_used = 0, d_max = 0;
  DOPINF_TRY(learn_check(Qhat, r_max, k, ldqh, r_list, n_r, beta1, n_b1, beta2, n_b2, mode, dt, n_steps, max_growth,
                         train_err, growth, cand_status, O_best, ws, ws_bytes, &r_used, &d_max));
  cudaStream_t st = as_stream(stream);
  // optional stage timings (CUDA events on this stream): data + normal equations, solves, rollouts
  cudaEvent_t ev[4] = {};
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int i = 0; i < 4; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } ev_guard{ev};
  if (stage_ms)
    for (int i = 0; i < 4; ++i) DOPINF_CUDA(cudaEventCreate(&ev[i]));
  LearnWs w = carve_learn(ws, k - 1, r_list, n_r, n_b1, n_b2);
  DOPINF_TRY(learn_launch(Qhat, r_max, k, ldqh, r_list, n_r, beta1, n_b1, beta2, n_b2, mode, dt, n_steps, max_growth,
                          train_err, growth, cand_status, cand_steps, nullptr, O_best, nullptr, r_used, d_max,
                          ws, st, stage_ms ? ev : nullptr));
  int best = -1;
  DOPINF_CUDA(cudaMemcpyAsync(&best, w.best, sizeof(int), cudaMemcpyDeviceToHost, st));
  DOPINF_CUDA(cudaStreamSynchronize(st));
  *best_out = best;
  if (stage_ms)
    for (int i = 0; i < 3; ++i) {
      float ms = 0.f;
      DOPINF_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
      stage_ms[i] = ms;
    }
  return best < 0 ? DOPINF_E_NO_STABLE : DOPINF_OK;
}

DOPINF_API int dopinf_tune_rollout_rows_large(int rows) { return rollout_set_rows_big(rows); }

DOPINF_API int dopinf_tune_learn_solver(int solver) {
  const int prev = g_solver;
  if (solver == DOPINF_SOLVE_CHOLESKY || solver == DOPINF_SOLVE_QR) g_solver = solver;
  return prev;
}

DOPINF_API int dopinf_tune_rollout_rows(int rows) { return rollout_set_rows(rows); }

DOPINF_API int dopinf_tune_rollout_arith(int arith) { return rollout_set_arith(arith); }
