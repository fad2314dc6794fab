// The regularised least-squares problem of Step IV (Section 3.5, eq. OpInf_reg) solved without
// the normal equations: for each candidate (r, beta1, beta2), the stacked system
//     [Dhat; diag(sqrt(reg))] O^T = [Y; 0]      (m = K + d rows, d unknowns, r right-hand sides)
// is reduced by Householder reflections (R = upper triangle, the right-hand sides carried along)
// and O^T follows by back substitution.  The conditioning is that of the stacked matrix, the
// square root of the normal equations'.  One CTA per candidate, 256 threads: a reflector per
// column (its norm by a block reduction), applied to the trailing columns and the right-hand
// sides, one column per warp at a time; the matrix lives in the candidate's workspace slice.
#include "common.cuh"
#include <math.h>

namespace dopinf {
namespace {

constexpr int QB = 256;
constexpr int QW = QB / 32;

__device__ double qr_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < QW; ++i) s += sh[i];  // fixed order
    sh[QW] = s;
  }
  __syncthreads();
  return sh[QW];
}

struct QrArgs {
  const double* Dh;  // K x d (ld K) data matrix of this r
  const double* Y;   // K x r (ld K) targets
  const SchurUnit* units;
  const SchurCand* cands;  // the candidates of this r start at cand0
  int cand0;
  int64_t K;
  int r, d;
  double* work;    // per candidate: m x (d + r), ld m
  size_t stride;   // doubles per candidate slice
  int* status;     // per candidate (global index)
};

__global__ void __launch_bounds__(QB) qr_candidates(QrArgs q) {
  __shared__ double sh[QW + 1];
  __shared__ double s_tau;
  const SchurCand cd = q.cands[q.cand0 + blockIdx.x];
  const double b2 = q.units[cd.unit].b2, b1 = cd.b1;
  const int r = q.r, d = q.d, s = d - r - 1;
  const int64_t K = q.K, m = K + d, lda = m;
  const int nc = d + r;
  double* A = q.work + (size_t)blockIdx.x * q.stride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the stacked system [Dhat | Y; diag(sqrt(reg)) | 0]
  for (int c = 0; c < nc; ++c) {
    const double rg = c < r ? b1 : (c < r + s ? b2 : b1);
    for (int64_t i = threadIdx.x; i < m; i += QB) {
      double v;
      if (c < d)
        v = i < K ? q.Dh[i + (int64_t)c * K] : (i - K == c ? sqrt(rg) : 0.0);
      else
        v = i < K ? q.Y[i + (int64_t)(c - d) * K] : 0.0;
      A[i + (int64_t)c * lda] = v;
    }
  }
  __syncthreads();
  bool bad = false;
  for (int j = 0; j < d; ++j) {
    // reflector of column j (rows j..m-1): A[j, j] <- beta, A[j+1.., j] <- v (v_j = 1)
    double* col = A + (int64_t)j * lda;
    const double alpha = col[j];  // read before the block sum's barriers: thread 0 overwrites it below
    double part = 0.0;
    for (int64_t i = j + 1 + threadIdx.x; i < m; i += QB) part = fma(col[i], col[i], part);
    const double sigma = qr_block_sum(part, sh);
    double tau = 0.0, beta = alpha;
    if (sigma != 0.0 || alpha < 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, sigma));
      beta = alpha > 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      const double scal = 1.0 / (alpha - beta);
      for (int64_t i = j + 1 + threadIdx.x; i < m; i += QB) col[i] *= scal;
    }
    if (threadIdx.x == 0) {
      col[j] = beta;
      s_tau = tau;
    }
    __syncthreads();
    tau = s_tau;
    bad = bad || beta == 0.0 || !isfinite(beta);
    if (tau != 0.0) {
      // H_j applied to the trailing columns and the right-hand sides, a column per warp
      for (int c = j + 1 + warp; c < nc; c += QW) {
        double* a = A + (int64_t)c * lda;
        double dot = lane == 0 ? a[j] : 0.0;
        for (int64_t i = j + 1 + lane; i < m; i += 32) dot = fma(col[i], a[i], dot);
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const double sc = tau * dot;
        if (lane == 0) a[j] -= sc;
        for (int64_t i = j + 1 + lane; i < m; i += 32) a[i] = fma(-sc, col[i], a[i]);
      }
    }
    __syncthreads();
  }
  // back substitution R X = (Q^T b)[0:d], the r right-hand sides in columns d .. d + r - 1
  for (int i = d - 1; i >= 0; --i) {
    const double rii = A[i + (int64_t)i * lda];
    if (threadIdx.x < r) {
      double* x = A + (int64_t)(d + threadIdx.x) * lda;
      x[i] = x[i] / rii;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)i * r; e += QB) {
      const int t = (int)(e / i), l = (int)(e % i);
      double* x = A + (int64_t)(d + t) * lda;
      x[l] = fma(-A[l + (int64_t)i * lda], x[i], x[l]);
    }
    __syncthreads();
  }
  // O (r x d, ld r): O[t, c] = X[c, t]
  for (int64_t e = threadIdx.x; e < (int64_t)r * d; e += QB) {
    const int t = (int)(e % r), c = (int)(e / r);
    cd.O[e] = A[c + (int64_t)(d + t) * lda];
  }
  if (threadIdx.x == 0) q.status[cd.cand] = bad ? 1 : 0;
}

}  // namespace

size_t qr_solve_doubles(int64_t K, int r) {
  const int64_t d = dim_d(r);
  return (size_t)(K + d) * (size_t)(d + r);
}

int qr_solve(const double* Dh, const double* Y, int64_t K, int r, const SchurUnit* units, const SchurCand* cands,
             int cand0, int n, double* work, size_t stride, int* cand_status, cudaStream_t st) {
  QrArgs q;
  q.Dh = Dh;
  q.Y = Y;
  q.units = units;
  q.cands = cands;
  q.cand0 = cand0;
  q.K = K;
  q.r = r;
  q.d = dim_d(r);
  q.work = work;
  q.stride = stride;
  q.status = cand_status;
  qr_candidates<<<n, QB, 0, st>>>(q);
  return launch_status();
}

}  // namespace dopinf
