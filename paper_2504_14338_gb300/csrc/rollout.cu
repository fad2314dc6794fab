// Rollouts of learned quadratic ROMs (Section 3.5): the discrete map of
// eq. ROM_quad_time_discrete, or classical RK4 on eq. ROM_quad_time_cont, with the training
// error and growth criterion of Step IV fused into the time loop.
//
// One thread-block cluster of C CTAs per candidate, every candidate of every r in one launch.
// CTA rank j of the cluster keeps rows [j*rc, (j+1)*rc) of the operator O = [A | H | c]
// (rc = ceil(r / C)) row-major in its shared memory.  Each right-hand-side evaluation builds
// phi = [q, (q_i q_j)_{i<=j}, 1] locally (the state is replicated), forms its rows of O phi
// with one warp per row, and stores them into the shared memory of every CTA of the cluster
// (distributed shared memory); a hardware cluster barrier then makes the full vector visible
// everywhere.  The stage results are double-buffered by step parity, so a CTA that runs ahead
// never overwrites values a slower peer is still reading.  The RK4 combination, the metrics
// and the early-exit decision are computed identically in every CTA, so the cluster stays in
// lockstep without further communication.  FP64 throughput per SM is small on GB300, so each
// stage state is formed once (r values) before its feature build rather than inside it.
#include "common.cuh"
#include <cooperative_groups.h>
#include <math.h>

namespace cg = cooperative_groups;

namespace dopinf {
namespace {

constexpr int RB = 256;  // threads per CTA
constexpr int NW = RB / 32;

struct SmemLayout {
  size_t o, q, xs, kb, phi, mu, pi, pj, total;
};

// Shared layout for a CTA holding rc operator rows of width d_max, vectors of r_max.
__host__ __device__ inline SmemLayout smem_layout(int rc, int r_max, int d_max) {
  SmemLayout L;
  size_t off = 0;
  L.o = off;
  off += (size_t)rc * d_max * sizeof(double);
  L.q = off;
  off += (size_t)r_max * sizeof(double);
  L.xs = off;
  off += (size_t)r_max * sizeof(double);
  L.kb = off;  // [2 step parities][4 stages][r_max]
  off += (size_t)8 * r_max * sizeof(double);
  L.phi = off;
  off += (size_t)d_max * sizeof(double);
  L.mu = off;
  off += (size_t)r_max * sizeof(double);
  const int s_max = d_max - r_max - 1 > 0 ? d_max - r_max - 1 : 1;
  L.pi = off;
  off += (size_t)s_max * sizeof(unsigned short);
  L.pj = off;
  off += (size_t)s_max * sizeof(unsigned short);
  L.total = (off + 15) / 16 * 16;
  return L;
}

// Rows [i0, i1) of O phi, stored into buffer `dst` of every CTA of the cluster.
__device__ __forceinline__ void eval_rows(cg::cluster_group& cl, const double* Os, int i0, int i1, int d,
                                          const double* phi, double* dst) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = (int)cl.num_blocks();
  for (int i = i0 + w; i < i1; i += NW) {
    const double* row = Os + (size_t)(i - i0) * d;
    double acc = 0.0;
    for (int a = lane; a < d; a += 32) acc = fma(row[a], phi[a], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane < C) {
      double* remote = cl.map_shared_rank(dst, (unsigned)lane);
      remote[i] = acc;
    }
  }
}

__device__ __forceinline__ void build_phi(const double* x, int r, int d, const unsigned short* pi,
                                          const unsigned short* pj, double* phi) {
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
}

__global__ void __launch_bounds__(RB, 5) rollout_kernel(RolloutBatch bt) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int cid = blockIdx.x / C;
  const RolloutCand cd = bt.cands ? bt.cands[cid] : bt.one;
  const int r = cd.r, d = cd.d;
  const int rc = (r + C - 1) / C;
  const int i0 = rank * rc < r ? rank * rc : r;
  const int i1 = i0 + rc < r ? i0 + rc : r;
  const SmemLayout L = smem_layout(bt.rc_max, bt.r_max, bt.d_max);
  double* Os = reinterpret_cast<double*>(smraw + L.o);
  double* q = reinterpret_cast<double*>(smraw + L.q);
  double* xs = reinterpret_cast<double*>(smraw + L.xs);
  double* kb = reinterpret_cast<double*>(smraw + L.kb);
  double* phi = reinterpret_cast<double*>(smraw + L.phi);
  double* mu = reinterpret_cast<double*>(smraw + L.mu);
  unsigned short* pi = reinterpret_cast<unsigned short*>(smraw + L.pi);
  unsigned short* pj = reinterpret_cast<unsigned short*>(smraw + L.pj);
  __shared__ int s_stop;

  // a failed factorisation (the same for every CTA of the cluster): nothing to roll out
  if (bt.metrics && bt.status[cd.cand] != 0) {
    if (rank == 0 && threadIdx.x == 0) {
      bt.train_err[cd.cand] = INFINITY;
      bt.growth[cd.cand] = INFINITY;
    }
    return;
  }
  for (int64_t e = threadIdx.x; e < (int64_t)(i1 - i0) * d; e += RB) {
    const int i = i0 + (int)(e / d), a = (int)(e % d);
    Os[e] = cd.O[i + (size_t)a * cd.ldo];
  }
  for (int i = threadIdx.x; i < r; i += RB) {
    const int off = i * r - i * (i - 1) / 2;  // column r + off(i) + (j - i) multiplies x_i x_j
    for (int j = i; j < r; ++j) {
      pi[off + j - i] = (unsigned short)i;
      pj[off + j - i] = (unsigned short)j;
    }
  }
  for (int i = threadIdx.x; i < r; i += RB) {
    q[i] = bt.q0[i];
    mu[i] = bt.metrics ? cd.mu[i] : 0.0;
  }
  if (threadIdx.x == 0) s_stop = 0;
  cl.sync();  // every CTA initialised before any remote store

  const double dt = bt.dt, h2 = 0.5 * dt, h6 = dt / 6.0;
  const double denom = bt.metrics ? *cd.denom : 1.0;
  // max over t < k of num/den (the training error is its square root: sqrt is monotone and
  // correctly rounded, so this is the maximum of the square roots), and the bits of the
  // largest |q - mu| (non-negative doubles order like their bit patterns)
  double rat = 0.0;
  unsigned long long gnumb = 0ull;
  // growth >= max_growth, decided without a division outside a band of 2^-40 around the
  // threshold (the division and the product each round by 2^-53)
  const double thr = bt.max_growth * denom;
  const bool band_ok = denom > 0.0 && isfinite(thr) && thr > 0.0;
  const unsigned long long band_lo =
      band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 - 0x1p-40)) : 0ull;
  const unsigned long long band_hi =
      band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 + 0x1p-40)) : ~0ull;
  int st = 0;
  int64_t t_end = 0;  // the last state whose metrics were formed (= steps advanced)
  for (int64_t t = 0;; ++t) {
    t_end = t;
    // ---- metrics and output of state t (warp 0 of every CTA, identical results) ----
    // They sit in front of the step's first evaluation, so they avoid the FP64 pipe where the
    // result does not change: max |q - mu| as an integer maximum of the (non-negative) bit
    // patterns, the training error as the maximum of num/den with one square root at the end,
    // and the growth test against a band around max_growth * denom (the division only inside).
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      bool fin = true;
      unsigned long long devb = 0ull;
      double num = 0.0, den = 0.0;
      for (int i = lane; i < r; i += 32) {
        const double v = q[i];
        fin = fin && isfinite(v);
        if (bt.metrics) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v - mu[i]));
          devb = b > devb ? b : devb;
          if (t < bt.k) {
            const double h = bt.Qhat[i + t * bt.ldqh];
            num += (v - h) * (v - h);
            den += h * h;
          }
        }
        if (bt.traj && rank == 0) bt.traj_out[t * r + i] = v;
      }
      fin = __all_sync(0xffffffffu, fin);
      if (bt.metrics) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long ob = __shfl_xor_sync(0xffffffffu, devb, o);
          devb = ob > devb ? ob : devb;
          if (t < bt.k) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
          }
        }
        if (fin) {
          gnumb = devb > gnumb ? devb : gnumb;
          if (t < bt.k) rat = fmax(rat, num / den);
        }
      }
      if (lane == 0) {
        int stop = 0;
        if (!fin) {
          st = 2;
          stop = 1;
        } else if (bt.metrics && gnumb >= band_lo &&
                   (gnumb > band_hi || __longlong_as_double((long long)gnumb) / denom >= bt.max_growth)) {
          st = 3;
          stop = 1;
        }
        if (t + 1 >= bt.n_steps) stop = 1;
        s_stop = stop;
      }
    }
    __syncthreads();
    if (s_stop) break;
    double* kp = kb + (size_t)(t & 1) * 4 * bt.r_max;  // this step's stage buffers
    double* k1 = kp;
    double* k2 = kp + bt.r_max;
    double* k3 = kp + 2 * bt.r_max;
    double* k4 = kp + 3 * bt.r_max;
    if (bt.mode == DOPINF_DISCRETE) {
      build_phi(q, r, d, pi, pj, phi);
      __syncthreads();
      eval_rows(cl, Os, i0, i1, d, phi, k1);
      cl.sync();
      for (int i = threadIdx.x; i < r; i += RB) q[i] = k1[i];
    } else {
      // products and sums rounded separately, in the order q + (dt/6)(((k1 + 2 k2) + 2 k3) + k4)
      build_phi(q, r, d, pi, pj, phi);
      __syncthreads();
      eval_rows(cl, Os, i0, i1, d, phi, k1);
      cl.sync();
      for (int i = threadIdx.x; i < r; i += RB) xs[i] = __dadd_rn(q[i], __dmul_rn(h2, k1[i]));
      __syncthreads();
      build_phi(xs, r, d, pi, pj, phi);
      __syncthreads();
      eval_rows(cl, Os, i0, i1, d, phi, k2);
      cl.sync();
      for (int i = threadIdx.x; i < r; i += RB) xs[i] = __dadd_rn(q[i], __dmul_rn(h2, k2[i]));
      __syncthreads();
      build_phi(xs, r, d, pi, pj, phi);
      __syncthreads();
      eval_rows(cl, Os, i0, i1, d, phi, k3);
      cl.sync();
      for (int i = threadIdx.x; i < r; i += RB) xs[i] = __dadd_rn(q[i], __dmul_rn(dt, k3[i]));
      __syncthreads();
      build_phi(xs, r, d, pi, pj, phi);
      __syncthreads();
      eval_rows(cl, Os, i0, i1, d, phi, k4);
      cl.sync();
      for (int i = threadIdx.x; i < r; i += RB) {
        const double sum = __dadd_rn(__dadd_rn(__dadd_rn(k1[i], 2.0 * k2[i]), 2.0 * k3[i]), k4[i]);
        q[i] = __dadd_rn(q[i], __dmul_rn(h6, sum));
      }
    }
    __syncthreads();
  }
  cl.sync();  // no CTA leaves while a peer may still store into its shared memory
  if (rank == 0 && threadIdx.x == 0) {
    if (bt.steps) bt.steps[cd.cand] = t_end;
    if (bt.metrics) {
      bt.status[cd.cand] = st;
      bt.train_err[cd.cand] = st == 0 ? sqrt(rat) : INFINITY;
      bt.growth[cd.cand] = st == 2 ? INFINITY : __longlong_as_double((long long)gnumb) / denom;
    }
    if (bt.traj && bt.finite) *bt.finite = st == 2 ? 0 : 1;
  }
}

constexpr size_t kRolloutSmemMax = 200 * 1024;

}  // namespace

size_t rollout_smem_bytes(int cluster, int r_max, int d_max) {
  return smem_layout((r_max + cluster - 1) / cluster, r_max, d_max).total;
}

int rollout_cluster_size(int r_max, int d_max, int want) {
  int c = 1;
  while (c < want && c < 8) c *= 2;
  while (c < 8 && rollout_smem_bytes(c, r_max, d_max) > kRolloutSmemMax) c *= 2;
  return rollout_smem_bytes(c, r_max, d_max) <= kRolloutSmemMax ? c : 0;
}

int launch_rollouts(RolloutBatch bt, int cluster, cudaStream_t st) {
  if (cluster < 1 || cluster > 8 || bt.n_cand < 1) return DOPINF_E_ARG;
  bt.rc_max = (bt.r_max + cluster - 1) / cluster;
  const size_t smem = rollout_smem_bytes(cluster, bt.r_max, bt.d_max);
  if (smem > kRolloutSmemMax) return DOPINF_E_UNSUPPORTED;
  DOPINF_CUDA(cudaFuncSetAttribute(rollout_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRolloutSmemMax));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(bt.n_cand * cluster), 1, 1);
  cfg.blockDim = dim3(RB, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DOPINF_CUDA(cudaLaunchKernelEx(&cfg, rollout_kernel, bt));
  return launch_status();
}

}  // namespace dopinf

using namespace dopinf;

DOPINF_API int dopinf_rollout(const double* O, int r, int64_t ldo, const double* q0, int64_t n_steps, int mode,
                              double dt, double* Qtilde, int* finite, void* stream) {
  if (!O || !q0 || !Qtilde || r < 1 || r > 255 || ldo < r || n_steps < 1) return DOPINF_E_ARG;
  if (mode != DOPINF_DISCRETE && mode != DOPINF_CONTINUOUS_RK4) return DOPINF_E_ARG;
  const int d = r + r * (r + 1) / 2 + 1;
  const int cluster = rollout_cluster_size(r, d, r >= 16 ? 4 : 1);
  if (!cluster) return DOPINF_E_UNSUPPORTED;
  RolloutBatch bt = {};
  bt.cands = nullptr;  // the single candidate travels inside the launch arguments
  bt.one.O = O;
  bt.one.ldo = ldo;
  bt.one.r = r;
  bt.one.d = d;
  bt.one.cand = 0;
  bt.n_cand = 1;
  bt.r_max = r;
  bt.d_max = d;
  bt.mode = mode;
  bt.dt = dt;
  bt.n_steps = n_steps;
  bt.q0 = q0;
  bt.traj = 1;
  bt.traj_out = Qtilde;
  bt.finite = finite;
  return launch_rollouts(bt, cluster, as_stream(stream));
}
