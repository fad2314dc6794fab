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
//   chol_solve      one CTA per (beta1, beta2): (G + diag(reg)) X = B by Cholesky, O = X^T;
//   rollouts        one CTA per candidate with the fused training error / growth epilogue.
// Then select_best takes the lowest training error among valid candidates (lowest index on
// ties).  Everything is FP64.
#include "common.cuh"
#include <math.h>

namespace dopinf {
namespace {

constexpr int LB = 256;
constexpr int CB = 512;

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

__global__ void __launch_bounds__(LB) train_stats(const double* __restrict__ Qhat, int64_t ldqh, int r, int64_t k,
                                                  double* __restrict__ mu, double* __restrict__ denom) {
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

// One CTA per regularisation pair of one r.  M (d x d) and X (d x r) live in the workspace
// (L2-resident for the sizes of Step IV).  Right-looking Cholesky M = L L^T, then
// L Z = B, L^T X = Z.  A non-positive or non-finite pivot marks the candidate (status 1).
__global__ void __launch_bounds__(CB) chol_solve(const double* __restrict__ G, const double* __restrict__ B, int r,
                                                 int d, const double* __restrict__ beta1, const double* __restrict__ beta2,
                                                 int n_b2, double* __restrict__ Mws, double* __restrict__ Xws,
                                                 double* __restrict__ Oall, int* __restrict__ status, int cand0) {
  __shared__ int s_fail;
  const int p = blockIdx.x;
  const double b1 = beta1[p / n_b2], b2 = beta2[p % n_b2];
  const int s = d - r - 1;
  double* M = Mws + (size_t)p * d * d;
  double* X = Xws + (size_t)p * d * r;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = CB / 32;
  for (int64_t e = tid; e < (int64_t)d * d; e += CB) {
    const int i = (int)(e % d), c = (int)(e / d);
    double v = G[e];
    if (i == c) v += (i < r || i == r + s) ? b1 : b2;
    M[e] = v;
  }
  for (int64_t e = tid; e < (int64_t)d * r; e += CB) X[e] = B[e];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < d; ++j) {
    const double piv = M[j + (size_t)j * d];
    if (!(piv > 0.0) || !isfinite(piv)) {
      if (tid == 0) s_fail = 1;
      break;
    }
    const double ljj = sqrt(piv), inv = 1.0 / ljj;
    for (int i = j + 1 + tid; i < d; i += CB) M[i + (size_t)j * d] *= inv;
    __syncthreads();
    if (tid == 0) M[j + (size_t)j * d] = ljj;
    for (int c = j + 1 + w; c < d; c += nw) {
      const double lc = M[c + (size_t)j * d];
      double* col = M + (size_t)c * d;
      const double* lj = M + (size_t)j * d;
      for (int i = c + lane; i < d; i += 32) col[i] = fma(-lj[i], lc, col[i]);
    }
    __syncthreads();
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) status[cand0 + p] = 1;
    return;
  }
  // forward: L Z = B (column j of L scales row j, then updates the rows below)
  for (int j = 0; j < d; ++j) {
    const double inv = 1.0 / M[j + (size_t)j * d];
    for (int c = tid; c < r; c += CB) X[j + (size_t)c * d] *= inv;
    __syncthreads();
    const int64_t rows = d - j - 1;
    for (int64_t e = tid; e < rows * r; e += CB) {
      const int i = j + 1 + (int)(e % rows), c = (int)(e / rows);
      X[i + (size_t)c * d] = fma(-M[i + (size_t)j * d], X[j + (size_t)c * d], X[i + (size_t)c * d]);
    }
    __syncthreads();
  }
  // backward: L^T X = Z
  for (int j = d - 1; j >= 0; --j) {
    const double inv = 1.0 / M[j + (size_t)j * d];
    for (int c = tid; c < r; c += CB) X[j + (size_t)c * d] *= inv;
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)j * r; e += CB) {
      const int i = (int)(e % j), c = (int)(e / j);
      X[i + (size_t)c * d] = fma(-M[j + (size_t)i * d], X[j + (size_t)c * d], X[i + (size_t)c * d]);
    }
    __syncthreads();
  }
  double* O = Oall + (size_t)p * r * d;  // r x d, ld r
  for (int64_t e = tid; e < (int64_t)r * d; e += CB) {
    const int i = (int)(e % r), a = (int)(e / r);
    O[e] = X[a + (size_t)i * d];
  }
  if (tid == 0) status[cand0 + p] = 0;
}

__global__ void select_best(const double* err, const int* status, int n_cand, int* best) {
  if (threadIdx.x != 0) return;
  int b = -1;
  for (int c = 0; c < n_cand; ++c)
    if (status[c] == 0 && (b < 0 || err[c] < err[b])) b = c;
  *best = b;
}

struct LearnWs {
  double *beta1, *beta2, *Oall, *mu, *denom, *Dh, *Y, *G, *B, *M, *X;
  int* best;
  void* tn;
  size_t tn_bytes, used;
  size_t o_off[64];
};

inline int dim_d(int r) { return r + r * (r + 1) / 2 + 1; }

LearnWs carve_learn(void* base, int64_t K, const int* r_list, int n_r, int n_b1, int n_b2) {
  Carver c(base);
  LearnWs w;
  int d_max = 0, r_max = 0;
  size_t o_total = 0;
  for (int i = 0; i < n_r; ++i) {
    w.o_off[i] = o_total;
    o_total += (size_t)n_b1 * n_b2 * r_list[i] * dim_d(r_list[i]);
    if (dim_d(r_list[i]) > d_max) d_max = dim_d(r_list[i]);
    if (r_list[i] > r_max) r_max = r_list[i];
  }
  const int n_pairs = n_b1 * n_b2;
  w.beta1 = c.take<double>(n_b1);
  w.beta2 = c.take<double>(n_b2);
  w.Oall = c.take<double>(o_total);
  w.mu = c.take<double>(r_max);
  w.denom = c.take<double>(1);
  w.best = c.take<int>(1);
  w.Dh = c.take<double>((size_t)K * d_max);
  w.Y = c.take<double>((size_t)K * r_max);
  w.G = c.take<double>((size_t)d_max * d_max);
  w.B = c.take<double>((size_t)d_max * r_max);
  w.M = c.take<double>((size_t)n_pairs * d_max * d_max);
  w.X = c.take<double>((size_t)n_pairs * d_max * r_max);
  size_t tb = 0;
  for (int i = 0; i < n_r; ++i) {
    const int r = r_list[i], d = dim_d(r);
    size_t a = tn_workspace(K, d, d, 1), b = tn_workspace(K, d, r, 0);
    tb = a > tb ? a : tb;
    tb = b > tb ? b : tb;
  }
  w.tn_bytes = tb;
  w.tn = c.take<char>(tb);
  w.used = c.used;
  return w;
}

}  // namespace
}  // namespace dopinf

using namespace dopinf;

static int64_t learn_rows(int64_t k, int mode) { return mode == DOPINF_DISCRETE ? k - 1 : k - 2; }

DOPINF_API size_t dopinf_learn_workspace(int r_max, int64_t k, const int* r_list, int n_r, int n_b1, int n_b2) {
  (void)r_max;
  if (!r_list || n_r < 1 || n_r > 64 || n_b1 < 1 || n_b2 < 1 || k < 3) return 0;
  return carve_learn(nullptr, k - 1, r_list, n_r, n_b1, n_b2).used;
}

DOPINF_API int dopinf_learn(const double* Qhat, int r_max, int64_t k, int64_t ldqh, const int* r_list, int n_r,
                            const double* beta1, int n_b1, const double* beta2, int n_b2, int mode, double dt,
                            int64_t n_steps, double max_growth, double* train_err, double* growth, int* cand_status,
                            int* best_out, double* O_best, void* ws, size_t ws_bytes, void* stream) {
  if (!Qhat || r_max < 1 || ldqh < r_max || !r_list || n_r < 1 || n_r > 64 || !beta1 || !beta2 || n_b1 < 1 ||
      n_b2 < 1 || !train_err || !growth || !cand_status || !best_out || !O_best)
    return DOPINF_E_ARG;
  if (mode != DOPINF_DISCRETE && mode != DOPINF_CONTINUOUS_RK4) return DOPINF_E_ARG;
  if (mode == DOPINF_CONTINUOUS_RK4 && !(dt > 0.0)) return DOPINF_E_ARG;
  const int64_t K = learn_rows(k, mode);
  if (K < 1 || n_steps < k || !(max_growth > 0.0)) return DOPINF_E_ARG;
  for (int i = 0; i < n_r; ++i)
    if (r_list[i] < 1 || r_list[i] > r_max || r_list[i] > 255) return DOPINF_E_ARG;
  for (int i = 0; i < n_b1; ++i)
    if (!(beta1[i] >= 0.0)) return DOPINF_E_ARG;
  for (int i = 0; i < n_b2; ++i)
    if (!(beta2[i] >= 0.0)) return DOPINF_E_ARG;
  if (!ws || ws_bytes < dopinf_learn_workspace(r_max, k, r_list, n_r, n_b1, n_b2) || misaligned(ws))
    return DOPINF_E_ARG;
  cudaStream_t st = as_stream(stream);
  // the workspace is laid out for K = k - 1 rows, which covers both modes
  LearnWs w = carve_learn(ws, k - 1, r_list, n_r, n_b1, n_b2);
  const int n_pairs = n_b1 * n_b2, n_cand = n_r * n_pairs;
  DOPINF_CUDA(cudaMemcpyAsync(w.beta1, beta1, sizeof(double) * n_b1, cudaMemcpyHostToDevice, st));
  DOPINF_CUDA(cudaMemcpyAsync(w.beta2, beta2, sizeof(double) * n_b2, cudaMemcpyHostToDevice, st));
  const int64_t t0 = mode == DOPINF_DISCRETE ? 0 : 1;
  for (int ir = 0; ir < n_r; ++ir) {
    const int r = r_list[ir], d = dim_d(r);
    const int64_t tot = K * (d + r);
    const unsigned blocks = (unsigned)((tot + LB - 1) / LB < 4096 ? (tot + LB - 1) / LB : 4096);
    build_features<<<blocks, LB, 0, st>>>(Qhat, ldqh, r, d, K, t0, mode, dt, w.Dh, w.Y);
    DOPINF_TRY(launch_status());
    DOPINF_TRY(tn_product(w.Dh, K, w.Dh, K, DOPINF_F64, K, d, d, 1, 0, w.G, d, w.tn, w.tn_bytes, st));
    DOPINF_TRY(tn_product(w.Dh, K, w.Y, K, DOPINF_F64, K, d, r, 0, 0, w.B, d, w.tn, w.tn_bytes, st));
    train_stats<<<1, LB, 0, st>>>(Qhat, ldqh, r, k, w.mu, w.denom);
    chol_solve<<<n_pairs, CB, 0, st>>>(w.G, w.B, r, d, w.beta1, w.beta2, n_b2, w.M, w.X, w.Oall + w.o_off[ir],
                                        cand_status, ir * n_pairs);
    DOPINF_TRY(launch_status());
    RolloutArgs a = {};
    a.O = w.Oall + w.o_off[ir];
    a.o_stride = (int64_t)r * d;
    a.ldo = r;
    a.r = r;
    a.d = d;
    a.mode = mode;
    a.dt = dt;
    a.n_steps = n_steps;
    a.q0 = Qhat;
    a.Qhat = Qhat;
    a.ldqh = ldqh;
    a.k = k;
    a.mu = w.mu;
    a.denom = w.denom;
    a.max_growth = max_growth;
    a.train_err = train_err;
    a.growth = growth;
    a.status = cand_status;
    a.cand0 = ir * n_pairs;
    DOPINF_TRY(launch_rollouts(a, n_pairs, true, false, st));
  }
  select_best<<<1, 32, 0, st>>>(train_err, cand_status, n_cand, w.best);
  DOPINF_TRY(launch_status());
  int best = -1;
  DOPINF_CUDA(cudaMemcpyAsync(&best, w.best, sizeof(int), cudaMemcpyDeviceToHost, st));
  DOPINF_CUDA(cudaStreamSynchronize(st));
  *best_out = best;
  if (best < 0) return DOPINF_E_NO_STABLE;
  const int ir = best / n_pairs, p = best % n_pairs, r = r_list[ir], d = dim_d(r);
  const double* src = w.Oall + w.o_off[ir] + (size_t)p * r * d;
  DOPINF_CUDA(cudaMemcpy2DAsync(O_best, sizeof(double) * r_max, src, sizeof(double) * r, sizeof(double) * r, d,
                                cudaMemcpyDeviceToDevice, st));
  DOPINF_CUDA(cudaStreamSynchronize(st));
  return DOPINF_OK;
}
