// Rollouts of learned quadratic ROMs (Section 3.5): the discrete map of
// eq. ROM_quad_time_discrete, or classical RK4 on eq. ROM_quad_time_cont, with the training
// error and growth criterion of Step IV fused into the time loop.
//
// One CTA per candidate.  The operator O = [A | H | c] (r x d) is staged row-major in shared
// memory (operators up to about 200 KB, i.e. r <= 36); each right-hand-side evaluation
// builds phi = [q, (q_i q_j)_{i<=j}, 1] in shared memory and forms O phi with one warp per
// output row.  The time loop is sequential; candidates run concurrently.
#include "common.cuh"
#include <math.h>

namespace dopinf {

namespace {
constexpr int RB = 256;  // threads per rollout CTA
constexpr int NW = RB / 32;
}  // namespace


namespace {

__device__ __forceinline__ void rhs_eval(const double* __restrict__ Os, const unsigned short* __restrict__ pi,
                                         const unsigned short* __restrict__ pj, int r, int d, const double* x,
                                         double* phi, double* out) {
  const int s = d - r - 1;
  for (int a = threadIdx.x; a < d; a += RB) {
    double v;
    if (a < r)
      v = x[a];
    else if (a < r + s)
      v = x[pi[a - r]] * x[pj[a - r]];
    else
      v = 1.0;
    phi[a] = v;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = w; i < r; i += NW) {
    const double* row = Os + (size_t)i * d;
    double acc = 0.0;
    for (int a = lane; a < d; a += 32) acc = fma(row[a], phi[a], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] = acc;
  }
  __syncthreads();
}

template <bool kMetrics, bool kTraj>
__global__ void __launch_bounds__(RB) rollout_kernel(RolloutArgs a) {
  extern __shared__ double sm[];
  const int r = a.r, d = a.d, s = d - r - 1;
  const int c = blockIdx.x;
  // shared layout: O row-major (r*d), q(r) x(r) k1..k4(4r) phi(d) pairs(2*s shorts)
  double* Os = sm;
  double* q = sm + (size_t)r * d;
  double* xs = q + r;
  double* k1 = xs + r;
  double* k2 = k1 + r;
  double* k3 = k2 + r;
  double* k4 = k3 + r;
  double* phi = k4 + r;
  unsigned short* pi = reinterpret_cast<unsigned short*>(phi + d);
  unsigned short* pj = pi + s;
  __shared__ int s_stop;
  if (kMetrics && a.status[a.cand0 + c] != 0) {  // factorisation failed: nothing to roll out
    if (threadIdx.x == 0) {
      a.train_err[a.cand0 + c] = INFINITY;
      a.growth[a.cand0 + c] = INFINITY;
    }
    return;
  }
  const double* Og = a.O + (size_t)c * a.o_stride;
  for (int64_t e = threadIdx.x; e < (int64_t)r * d; e += RB) {
    const int i = (int)(e / d), col = (int)(e % d);
    Os[e] = Og[i + (size_t)col * a.ldo];
  }
  const double* Orow = Os;
  for (int i = threadIdx.x; i < r; i += RB) {
    // pair table: column r + off(i) + (j - i) multiplies x_i x_j
    int off = i * r - i * (i - 1) / 2;
    for (int j = i; j < r; ++j) {
      pi[off + j - i] = (unsigned short)i;
      pj[off + j - i] = (unsigned short)j;
    }
  }
  for (int i = threadIdx.x; i < r; i += RB) q[i] = a.q0[i];
  if (threadIdx.x == 0) s_stop = 0;
  __syncthreads();
  const double dt = a.dt;
  double err = 0.0, gnum = 0.0;
  int st = 0;
  int64_t t = 0;
  for (;; ++t) {
    // ---- metrics and output of state t (warp 0) ----
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      bool fin = true;
      double dev = 0.0, num = 0.0, den = 0.0;
      for (int i = lane; i < r; i += 32) {
        const double v = q[i];
        fin = fin && isfinite(v);
        if (kMetrics) {
          dev = fmax(dev, fabs(v - a.mu[i]));
          if (t < a.k) {
            const double h = a.Qhat[i + t * a.ldqh];
            num += (v - h) * (v - h);
            den += h * h;
          }
        }
        if (kTraj) a.traj[t * r + i] = v;
      }
      fin = __all_sync(0xffffffffu, fin);
      if (kMetrics) {
        for (int o = 16; o > 0; o >>= 1) {
          dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
          num += __shfl_xor_sync(0xffffffffu, num, o);
          den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        if (fin) {
          gnum = fmax(gnum, dev);
          if (t < a.k) err = fmax(err, sqrt(num / den));
        }
      }
      if (lane == 0) {
        int stop = 0;
        if (!fin) {
          st = 2;
          stop = 1;
        } else if (kMetrics && gnum / *a.denom >= a.max_growth) {
          st = 3;
          stop = 1;
        }
        if (t + 1 >= a.n_steps) stop = 1;
        s_stop = stop;
      }
    }
    __syncthreads();
    if (s_stop) break;
    // ---- advance ----
    // (products and sums rounded separately, in the order q + (dt/6)((k1 + 2 k2) + 2 k3) + k4)
    if (a.mode == DOPINF_DISCRETE) {
      rhs_eval(Orow, pi, pj, r, d, q, phi, k1);
      for (int i = threadIdx.x; i < r; i += RB) q[i] = k1[i];
    } else {
      const double h2 = 0.5 * dt, h6 = dt / 6.0;
      rhs_eval(Orow, pi, pj, r, d, q, phi, k1);
      for (int i = threadIdx.x; i < r; i += RB) xs[i] = __dadd_rn(q[i], __dmul_rn(h2, k1[i]));
      __syncthreads();
      rhs_eval(Orow, pi, pj, r, d, xs, phi, k2);
      for (int i = threadIdx.x; i < r; i += RB) xs[i] = __dadd_rn(q[i], __dmul_rn(h2, k2[i]));
      __syncthreads();
      rhs_eval(Orow, pi, pj, r, d, xs, phi, k3);
      for (int i = threadIdx.x; i < r; i += RB) xs[i] = __dadd_rn(q[i], __dmul_rn(dt, k3[i]));
      __syncthreads();
      rhs_eval(Orow, pi, pj, r, d, xs, phi, k4);
      for (int i = threadIdx.x; i < r; i += RB) {
        const double sum = __dadd_rn(__dadd_rn(__dadd_rn(k1[i], 2.0 * k2[i]), 2.0 * k3[i]), k4[i]);
        q[i] = __dadd_rn(q[i], __dmul_rn(h6, sum));
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (kMetrics) {
      const int ci = a.cand0 + c;
      a.status[ci] = st;
      a.train_err[ci] = st == 0 ? err : INFINITY;
      a.growth[ci] = st == 2 ? INFINITY : gnum / *a.denom;
    }
    if (kTraj && a.finite) *a.finite = st == 2 ? 0 : 1;
  }
}

size_t rollout_smem(int r, int d) {
  const int s = d - r - 1;
  return ((size_t)r * d + 6 * (size_t)r + d) * sizeof(double) + 2 * (size_t)s * sizeof(unsigned short) + 16;
}

}  // namespace

// Shared memory budget: the operator is staged only when it fits.
constexpr size_t kRolloutSmemMax = 200 * 1024;

int launch_rollouts(const RolloutArgs& a, int n_cand, bool metrics, bool traj, cudaStream_t st) {
  const size_t smem = rollout_smem(a.r, a.d);
  if (smem > kRolloutSmemMax) return DOPINF_E_UNSUPPORTED;  // operator larger than shared memory
  if (metrics && !traj) {
    DOPINF_CUDA(cudaFuncSetAttribute(rollout_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRolloutSmemMax));
    rollout_kernel<true, false><<<n_cand, RB, smem, st>>>(a);
  } else if (!metrics && traj) {
    DOPINF_CUDA(cudaFuncSetAttribute(rollout_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRolloutSmemMax));
    rollout_kernel<false, true><<<n_cand, RB, smem, st>>>(a);
  } else {
    return DOPINF_E_ARG;
  }
  return launch_status();
}

}  // namespace dopinf

using namespace dopinf;

DOPINF_API int dopinf_rollout(const double* O, int r, int64_t ldo, const double* q0, int64_t n_steps, int mode,
                              double dt, double* Qtilde, int* finite, void* stream) {
  if (!O || !q0 || !Qtilde || r < 1 || r > 255 || ldo < r || n_steps < 1) return DOPINF_E_ARG;
  if (mode != DOPINF_DISCRETE && mode != DOPINF_CONTINUOUS_RK4) return DOPINF_E_ARG;
  RolloutArgs a = {};
  a.O = O;
  a.o_stride = 0;
  a.ldo = ldo;
  a.r = r;
  a.d = r + r * (r + 1) / 2 + 1;
  a.mode = mode;
  a.dt = dt;
  a.n_steps = n_steps;
  a.q0 = q0;
  a.traj = Qtilde;
  a.finite = finite;
  return launch_rollouts(a, 1, false, true, as_stream(stream));
}
