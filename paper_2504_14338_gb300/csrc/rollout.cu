// Rollouts of learned quadratic ROMs (Section 3.5): the discrete map of
// eq. ROM_quad_time_discrete, or classical RK4 on eq. ROM_quad_time_cont, with the training
// error and growth criterion of Step IV fused into the time loop.  Two kernels:
//  * rollout_cols_kernel (below, r <= 32, the path of the workloads): column-owned layout,
//    one launch per r, FP64 or double-word FP32 arithmetic;
//  * rollout_kernel (r > 32): the row-split layout described here.
//
// Row-split kernel: one thread-block cluster of C CTAs per candidate, every candidate of every r
// in one launch.
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

#include <map>
#include <type_traits>
#include <mutex>
#include <utility>

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
      if (bt.steps) bt.steps[cd.cand] = 0;
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

// ---------------------------------------------------------------------------------------
// Column-owned rollouts for r <= 32.  FP64 issue on GB300 is one warp instruction per 64
// cycles per SM sub-partition, so the critical path of one evaluation is the number of FP64
// warp instructions each sub-partition executes, plus the exchange.  This layout keeps that
// number small and the exchange to one cluster barrier:
//  * 128 threads (one warp per sub-partition); one cluster of C = ceil(r / RC) CTAs per
//    candidate, CTA j owning rows [j RC, j RC + RC) (C <= 16);
//  * thread tid owns the columns a = tid + 128 t (t < NT) of phi: its entries O[i][a] for the
//    CTA's rows and the index pair forming phi_a stay in registers for the whole rollout, and
//    it builds those phi_a itself from the stage state, so phi never passes through shared
//    memory;
//  * a transposed butterfly reduces the RC row sums of a warp in five levels (one add per
//    level for all RC rows), the four warp sums of each row go to shared memory, and after
//    the cluster barrier the lane that owns state entry i (warp 0, lane i) pulls the owner
//    CTA's four partial sums of row i and adds them in a fixed order.
// Every CTA forms the same state, and the row sums are the same binary tree over the 128
// column partial sums whatever RC and C are, so the results do not depend on the launch shape.
//
// Two arithmetics share the layout.  FP64 (DW = false): every operation in binary64.
// Double-word (DW = true): numbers are unevaluated sums h + l of two binary32 values (about 48
// significant bits) on the FP32 pipe, which issues 64 times faster than the FP64 pipe here.
// The dot products are compensated (each product split exactly with an FMA, each partial sum
// with TwoSum, the errors gathered in a second word: the Dot2 scheme of Ogita, Rump and Oishi,
// SIAM J. Sci. Comput. 26 (2005), applied to double-word operands), and the state updates use
// the double-word sum and product of Joldes, Muller and Popescu (ACM TOMS 44, 2017: the
// accurate sum, relative error <= 3u^2, and the product with the low-by-low term, <= 5u^2,
// u = 2^-24).  The metrics and the decisions stay in FP64 on the exactly converted state.  A
// candidate whose operator or initial state lies outside [-2^60, 2^60], or whose double-word
// state stops being finite, is marked for the FP64 kernel (status 4), which then rolls it out
// again from the start, so the statuses are those of the FP64 arithmetic.
constexpr int RB5 = 128;
constexpr int NW5 = RB5 / 32;
constexpr int kMaxR5 = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kStatusRedo = 4;           // double-word run handed to the FP64 kernel
constexpr double kDwRange = 0x1p60;      // magnitude bound of double-word inputs

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- double-word arithmetic (binary32 pairs); the _rn intrinsics keep every rounding explicit
struct dw {
  float h, l;
};
__device__ __forceinline__ dw two_sum(float a, float b) {  // a + b = h + l exactly
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {  // exact when |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw dw_add(dw x, dw y) {
  const dw s = two_sum(x.h, y.h), t = two_sum(x.l, y.l);
  const dw v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);
  const float tl1 = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l));
  const float cl2 = __fmaf_rn(x.l, y.h, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
__device__ __forceinline__ dw dw_twice(dw x) { return {2.0f * x.h, 2.0f * x.l}; }
__device__ __forceinline__ dw dw_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dw_value(dw x) { return (double)x.h + (double)x.l; }  // exact

// compensated partial sum s + c of a dot product: s carries the rounded sum, c the errors
struct csum {
  float s, c;
};
__device__ __forceinline__ csum csum_add(csum x, csum y) {
  const dw t = two_sum(x.s, y.s);
  return {t.h, __fadd_rn(__fadd_rn(x.c, y.c), t.l)};
}
__device__ __forceinline__ double shfl_x(double v, int o) { return __shfl_xor_sync(kFull, v, o); }
__device__ __forceinline__ csum shfl_x(csum v, int o) {
  return {__shfl_xor_sync(kFull, v.s, o), __shfl_xor_sync(kFull, v.c, o)};
}
__device__ __forceinline__ double add_v(double a, double b) { return a + b; }
__device__ __forceinline__ csum add_v(csum a, csum b) { return csum_add(a, b); }

// Warp sum of each of the RC values per lane; lane L returns the sum of row L >> (5 - log2 RC).
// At each level a lane keeps half of its values and adds the half its partner sends, so the
// tree of every row is the full butterfly over the 32 lanes (the same for every RC); partners
// form identical sums because both additions are commutative.
template <int RC, typename V>
__device__ __forceinline__ V warp_rows_sum(const V (&acc)[RC], int lane) {
  V k;
  if constexpr (RC == 1) {
    k = add_v(acc[0], shfl_x(acc[0], 16));
  } else if constexpr (RC == 2) {
    const bool up = lane & 16;
    k = add_v(up ? acc[1] : acc[0], shfl_x(up ? acc[0] : acc[1], 16));
  } else {
    static_assert(RC == 4, "RC is 1, 2 or 4");
    const bool up = lane & 16;
    const V k0 = add_v(up ? acc[2] : acc[0], shfl_x(up ? acc[0] : acc[2], 16));
    const V k1 = add_v(up ? acc[3] : acc[1], shfl_x(up ? acc[1] : acc[3], 16));
    const bool up8 = lane & 8;
    k = add_v(up8 ? k1 : k0, shfl_x(up8 ? k0 : k1, 8));
  }
#pragma unroll
  for (int o = (RC == 4 ? 4 : 8); o > 0; o >>= 1) k = add_v(k, shfl_x(k, o));
  return k;
}

template <int NT, int RC, bool DW>
__global__ void __launch_bounds__(RB5, DW ? 5 : 6) rollout_cols_kernel(RolloutBatch bt, int cand0) {
  using Part = typename std::conditional<DW, csum, double>::type;
  __shared__ double xs[kMaxR5 + 2];    // FP64 stage state; xs[r] = 1, xs[r + 1] = 0
  __shared__ float xh[kMaxR5 + 2];     // double-word stage state (high, low words)
  __shared__ float xl[kMaxR5 + 2];
  __shared__ Part part[2][NW5][RC];    // warp sums of this CTA's rows, by evaluation parity
  __shared__ int s_stop, s_bad;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) pdl_trigger();  // a dependent rollout launch may start filling free SMs
  const RolloutCand cd = bt.cands ? bt.cands[cand0 + (int)(blockIdx.x / C)] : bt.one;
  const int r = cd.r, d = cd.d, i0 = rank * RC;

  // which candidates this launch rolls out: status 0 (a later FP64 pass: status 4 only)
  const int want = (!DW && bt.redo) ? kStatusRedo : 0;
  bool run = !(bt.metrics && bt.status[cd.cand] != want);
  if (!run && !bt.redo && rank == 0 && tid == 0 && bt.status[cd.cand] != kStatusRedo) {
    // a failed factorisation (the same for every CTA of the cluster): nothing to roll out
    bt.train_err[cd.cand] = INFINITY;
    bt.growth[cd.cand] = INFINITY;
    if (bt.steps) bt.steps[cd.cand] = 0;
  }

  // this thread's columns: operator entries of the CTA's rows and the phi index pair
  double o[DW ? 1 : NT][DW ? 1 : RC];
  float oh[DW ? NT : 1][DW ? RC : 1], ol[DW ? NT : 1][DW ? RC : 1];
  unsigned pr[NT];
  if (run) {
    bool bad = false;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int a = tid + RB5 * t;
      int ia, ib;
      if (a < r) {  // linear term: q_a * 1
        ia = a;
        ib = r;
      } else if (a < d - 1) {  // quadratic term q_i q_j, i <= j, i-major
        const int q = a - r;
        int i = 0;
        while (i + 1 < r && (i + 1) * (2 * r - i) / 2 <= q) ++i;
        ia = i;
        ib = i + q - i * (2 * r - i + 1) / 2;
      } else if (a == d - 1) {  // constant term: 1 * 1
        ia = r;
        ib = r;
      } else {  // past the last column: 0 * 0 against a zero operator entry
        ia = r + 1;
        ib = r + 1;
      }
      pr[t] = (unsigned)ia | ((unsigned)ib << 8);
#pragma unroll
      for (int rho = 0; rho < RC; ++rho) {
        const int i = i0 + rho;
        const double v = (a < d && i < r) ? cd.O[i + (size_t)a * cd.ldo] : 0.0;
        if constexpr (DW) {
          bad = bad || !(fabs(v) <= kDwRange);
          const dw w = dw_of(v);
          oh[t][rho] = w.h;
          ol[t][rho] = w.l;
        } else {
          o[t][rho] = v;
        }
      }
    }
    if constexpr (DW) {
      // the double-word range is a property of the candidate: agree on it across the cluster
      if (warp == 0 && lane < r) bad = bad || !(fabs(bt.q0[lane]) <= kDwRange);
      const int any = __syncthreads_or(bad);
      if (tid == 0) s_bad = any;
      cl.sync();
      int peer = 0;
      if (tid < C) peer = *cl.map_shared_rank(&s_bad, (unsigned)tid);
      if (__syncthreads_or(peer)) {
        run = false;
        if (rank == 0 && tid == 0) bt.status[cd.cand] = kStatusRedo;
      }
      cl.sync();  // every CTA has read its peers' flags before any of them leaves
    }
  }

  if (run) {
    // state entry `lane` lives in warp 0 (registers) and in the stage state in shared memory
    const bool own = warp == 0 && lane < r;
    double qv = own ? bt.q0[lane] : 0.0;
    dw qw = dw_of(qv);
    const double mu = (own && bt.metrics) ? cd.mu[lane] : 0.0;
    double hcur = (own && bt.metrics && bt.k > 0) ? bt.Qhat[lane] : 0.0;
    if (own) {
      xs[lane] = qv;
      xh[lane] = qw.h;
      xl[lane] = qw.l;
    }
    if (tid == 0) {
      xs[r] = 1.0;
      xs[r + 1] = 0.0;
      xh[r] = 1.0f;
      xl[r] = 0.0f;
      xh[r + 1] = 0.0f;
      xl[r + 1] = 0.0f;
    }
    const double dt = bt.dt, h2 = 0.5 * dt, h6 = dt / 6.0;
    const dw dtw = dw_of(dt), h2w = dw_of(h2), h6w = dw_of(h6);
    const double denom = bt.metrics ? *cd.denom : 1.0;
    // metrics as in the row-split kernel: max of num/den (one square root at the end), the
    // largest |q - mu| as an integer maximum of bit patterns, growth decided by a band of
    // 2^-40 around max_growth * denom with the division only inside it
    double rat = 0.0;
    unsigned long long gnumb = 0ull;
    const double thr = bt.max_growth * denom;
    const bool band_ok = denom > 0.0 && isfinite(thr) && thr > 0.0;
    const unsigned long long band_lo =
        band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 - 0x1p-40)) : 0ull;
    const unsigned long long band_hi =
        band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 + 0x1p-40)) : ~0ull;
    int st = 0;

    // metrics of state t (warp 0); lane 0 publishes the stop decision
    auto check = [&](int64_t t) {
      if constexpr (DW) qv = dw_value(qw);
      bool fin = !own || isfinite(qv);
      unsigned long long devb = 0ull;
      double num = 0.0, den = 0.0;
      if (own && bt.metrics) {
        devb = (unsigned long long)__double_as_longlong(fabs(qv - mu));
        if (t < bt.k) {
          num = (qv - hcur) * (qv - hcur);
          den = hcur * hcur;
        }
      }
      if (own && bt.traj && rank == 0) bt.traj_out[t * r + lane] = qv;
      fin = __all_sync(kFull, fin);
      int stop = 0;
      if (bt.metrics) {
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
          const unsigned long long ob = __shfl_xor_sync(kFull, devb, o2);
          devb = ob > devb ? ob : devb;
        }
        if (t < bt.k) {
          const double nd[2] = {num, den};
          const double v = warp_rows_sum<2>(nd, lane);  // lanes < 16: num, lanes >= 16: den
          num = v;
          den = __shfl_sync(kFull, v, 16);
        }
        if (lane == 0 && fin) {
          gnumb = devb > gnumb ? devb : gnumb;
          if (t < bt.k) rat = fmax(rat, num / den);
        }
      }
      if (lane == 0) {
        if (!fin) {
          st = DW ? kStatusRedo : 2;
          stop = 1;
        } else if (bt.metrics && gnumb >= band_lo &&
                   (gnumb > band_hi || __longlong_as_double((long long)gnumb) / denom >= bt.max_growth)) {
          st = 3;
          stop = 1;
        }
        if (t + 1 >= bt.n_steps) stop = 1;
        s_stop = stop;
      }
    };

    // one right-hand-side evaluation at the stage state; returns entry `lane` to warp 0.
    // with_check: warp 0 forms the metrics of state t between its arrival at the cluster
    // barrier and its wait there, so they overlap the exchange instead of lengthening the step
    unsigned e = 0;
    auto eval = [&](bool with_check, int64_t t) {
      Part acc[RC];
#pragma unroll
      for (int rho = 0; rho < RC; ++rho) acc[rho] = Part{};
#pragma unroll
      for (int t2 = 0; t2 < NT; ++t2) {
        const unsigned ia = pr[t2] & 0xffu, ib = pr[t2] >> 8;
        if constexpr (DW) {
          // phi = x_i x_j as a double-word (the low-by-low term is below u^2 |phi|)
          const float ah = xh[ia], al = xl[ia], bh = xh[ib], bl = xl[ib];
          const float ph = __fmul_rn(ah, bh);
          const float pl = __fmaf_rn(al, bh, __fmaf_rn(ah, bl, __fmaf_rn(ah, bh, -ph)));
#pragma unroll
          for (int rho = 0; rho < RC; ++rho) {
            const float p = __fmul_rn(oh[t2][rho], ph);
            const float err =
                __fmaf_rn(ol[t2][rho], ph, __fmaf_rn(oh[t2][rho], pl, __fmaf_rn(oh[t2][rho], ph, -p)));
            const dw u = two_sum(acc[rho].s, p);
            acc[rho].s = u.h;
            acc[rho].c = __fadd_rn(acc[rho].c, __fadd_rn(u.l, err));
          }
        } else {
          const double ph = xs[ia] * xs[ib];
#pragma unroll
          for (int rho = 0; rho < RC; ++rho) acc[rho] = fma(o[t2][rho], ph, acc[rho]);
        }
      }
      const Part v = warp_rows_sum<RC>(acc, lane);
      const int buf = (int)(e & 1u);
      if ((lane & (32 / RC - 1)) == 0) part[buf][warp][lane / (32 / RC)] = v;
      // release of every CTA's partial sums ... acquire of its peers'
      asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
      if (with_check && warp == 0) {
        check(t);
        __syncwarp();
      }
      asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
      Part k{};
      if (own) {
        const int owner = lane / RC, rho = lane - owner * RC;
        const Part* pp = cl.map_shared_rank(&part[buf][0][0], (unsigned)owner);
        k = add_v(add_v(pp[0 * RC + rho], pp[1 * RC + rho]), add_v(pp[2 * RC + rho], pp[3 * RC + rho]));
      }
      ++e;
      return k;
    };
    // state arithmetic of the two kinds
    auto set_stage = [&](double v, dw w) {
      if constexpr (DW) {
        xh[lane] = w.h;
        xl[lane] = w.l;
      } else {
        xs[lane] = v;
      }
    };
    auto as_dw = [](csum c) { return two_sum(c.s, c.c); };

    __syncthreads();
    // Step t: the first evaluation at state t carries the metrics of state t; if they stop
    // the rollout, that evaluation is discarded and state t is the last one (t_end = t).
    int64_t t_end = 0;
    for (int64_t t = 0;; ++t) {
      t_end = t;
      // the reference state of step t + 1 for the training error, fetched a step early
      double hnext = 0.0;
      if (own && bt.metrics && t + 1 < bt.k) hnext = bt.Qhat[lane + (t + 1) * bt.ldqh];
      const Part k1 = eval(true, t);
      if (bt.mode == DOPINF_DISCRETE) {
        if constexpr (DW) {
          const dw n = as_dw(k1);
          if (own) set_stage(0.0, n);
          __syncthreads();
          if (s_stop) break;
          qw = n;
        } else {
          if (own) set_stage(k1, dw{});
          __syncthreads();
          if (s_stop) break;
          qv = k1;
        }
      } else if constexpr (DW) {
        // the RK4 combination q + (dt/6)(((k1 + 2 k2) + 2 k3) + k4) in double-word arithmetic
        const dw a1 = as_dw(k1);
        if (own) set_stage(0.0, dw_add(qw, dw_mul(h2w, a1)));
        __syncthreads();
        if (s_stop) break;
        const dw a2 = as_dw(eval(false, t));
        if (own) set_stage(0.0, dw_add(qw, dw_mul(h2w, a2)));
        __syncthreads();
        const dw a3 = as_dw(eval(false, t));
        if (own) set_stage(0.0, dw_add(qw, dw_mul(dtw, a3)));
        __syncthreads();
        const dw a4 = as_dw(eval(false, t));
        if (own) {
          const dw sum = dw_add(dw_add(dw_add(a1, dw_twice(a2)), dw_twice(a3)), a4);
          qw = dw_add(qw, dw_mul(h6w, sum));
          set_stage(0.0, qw);
        }
        __syncthreads();
      } else {
        // products and sums rounded separately, in the order q + (dt/6)(((k1 + 2 k2) + 2 k3) + k4)
        if (own) set_stage(__dadd_rn(qv, __dmul_rn(h2, k1)), dw{});
        __syncthreads();
        if (s_stop) break;
        const double k2 = eval(false, t);
        if (own) set_stage(__dadd_rn(qv, __dmul_rn(h2, k2)), dw{});
        __syncthreads();
        const double k3 = eval(false, t);
        if (own) set_stage(__dadd_rn(qv, __dmul_rn(dt, k3)), dw{});
        __syncthreads();
        const double k4 = eval(false, t);
        if (own) {
          const double sum = __dadd_rn(__dadd_rn(__dadd_rn(k1, 2.0 * k2), 2.0 * k3), k4);
          qv = __dadd_rn(qv, __dmul_rn(h6, sum));
          set_stage(qv, dw{});
        }
        __syncthreads();
      }
      hcur = hnext;
    }
    cl.sync();  // no CTA leaves while a peer may still read its partial sums
    if (rank == 0 && tid == 0) {
      if (DW && st == kStatusRedo) {
        bt.status[cd.cand] = kStatusRedo;  // the FP64 kernel rolls this candidate out again
      } else {
        if (bt.steps) bt.steps[cd.cand] = t_end;
        if (bt.metrics) {
          bt.status[cd.cand] = st;
          bt.train_err[cd.cand] = st == 0 ? sqrt(rat) : INFINITY;
          bt.growth[cd.cand] = st == 2 ? INFINITY : __longlong_as_double((long long)gnumb) / denom;
        }
        if (bt.traj && bt.finite) *bt.finite = st == 2 ? 0 : 1;
      }
    }
  }
  // a rollout launch chained behind another by programmatic dependent launch completes only
  // after the one before it (so the stream's next operation sees every candidate's results)
  if (blockIdx.x == gridDim.x - 1 && tid == 0) pdl_wait();
}

template <int NT, int RC, bool DW>
void* cols_kernel_ptr() {
  return reinterpret_cast<void*>(&rollout_cols_kernel<NT, RC, DW>);
}

void* cols_kernel(int nt, int rc, bool dw) {
  using F = void* (*)();
  static const F tab[2][5][3] = {
      {{cols_kernel_ptr<1, 1, false>, cols_kernel_ptr<1, 2, false>, cols_kernel_ptr<1, 4, false>},
       {cols_kernel_ptr<2, 1, false>, cols_kernel_ptr<2, 2, false>, cols_kernel_ptr<2, 4, false>},
       {cols_kernel_ptr<3, 1, false>, cols_kernel_ptr<3, 2, false>, cols_kernel_ptr<3, 4, false>},
       {cols_kernel_ptr<4, 1, false>, cols_kernel_ptr<4, 2, false>, cols_kernel_ptr<4, 4, false>},
       {cols_kernel_ptr<5, 1, false>, cols_kernel_ptr<5, 2, false>, cols_kernel_ptr<5, 4, false>}},
      {{cols_kernel_ptr<1, 1, true>, cols_kernel_ptr<1, 2, true>, cols_kernel_ptr<1, 4, true>},
       {cols_kernel_ptr<2, 1, true>, cols_kernel_ptr<2, 2, true>, cols_kernel_ptr<2, 4, true>},
       {cols_kernel_ptr<3, 1, true>, cols_kernel_ptr<3, 2, true>, cols_kernel_ptr<3, 4, true>},
       {cols_kernel_ptr<4, 1, true>, cols_kernel_ptr<4, 2, true>, cols_kernel_ptr<4, 4, true>},
       {cols_kernel_ptr<5, 1, true>, cols_kernel_ptr<5, 2, true>, cols_kernel_ptr<5, 4, true>}},
  };
  const int ri = rc == 1 ? 0 : rc == 2 ? 1 : rc == 4 ? 2 : -1;
  if (nt < 1 || nt > 5 || ri < 0) return nullptr;
  return tab[dw ? 1 : 0][nt - 1][ri]();
}

int g_rows_want = 4;  // tunable: rows of O per CTA in the column-owned rollouts

// Whether a cluster of c CTAs of this kernel can be resident (sizes above 8 need the
// non-portable attribute and enough SMs in one GPC); cached per kernel and size.
bool cluster_fits(void* fn, int c) {
  static std::mutex mu;
  static std::map<std::pair<void*, int>, bool> cache;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(fn, c);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  bool ok = true, refused = false;
  if (c > 8) {
    ok = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    refused = !ok;
  }
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c, 1, 1);
    cfg.blockDim = dim3(RB5, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t q = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
    refused = refused || q != cudaSuccess;
    ok = q == cudaSuccess && n >= 1;
  }
  // a refused size is an answer, not an error to report later: clear the error this query
  // raised (and only then, so that no earlier error of the caller's is swallowed)
  if (refused) cudaGetLastError();
  cache[key] = ok;
  return ok;
}

}  // namespace

bool rollout_cols_supported(int r) { return r >= 1 && r <= kMaxR5 && (dim_d(r) + RB5 - 1) / RB5 <= 5; }

// Rows per CTA and cluster size of the column-owned kernel for rank r (0 if none fits), for
// both arithmetics (the FP64 kernel re-runs what the double-word one hands back).
int rollout_cols_shape(int r, int* rows, int* cluster) {
  if (!rollout_cols_supported(r)) return 0;
  const int nt = (dim_d(r) + RB5 - 1) / RB5;
  for (int rc = g_rows_want; rc <= 4; rc *= 2) {
    const int c = (r + rc - 1) / rc;
    if (c > 16) continue;
    void* f64 = cols_kernel(nt, rc, false);
    void* fdw = cols_kernel(nt, rc, true);
    if (f64 && fdw && cluster_fits(f64, c) && cluster_fits(fdw, c)) {
      *rows = rc;
      *cluster = c;
      return 1;
    }
  }
  return 0;
}

int g_arith = DOPINF_ROLLOUT_DW;  // tunable: arithmetic of the learn rollouts

int rollout_set_arith(int a) {
  const int prev = g_arith;
  if (a == DOPINF_ROLLOUT_FP64 || a == DOPINF_ROLLOUT_DW) g_arith = a;
  return prev;
}

int rollout_arith() { return g_arith; }

int rollout_set_rows(int rc) {
  const int prev = g_rows_want;
  if (rc == 1 || rc == 2 || rc == 4) g_rows_want = rc;
  return prev;
}

// Candidates [cand0, cand0 + n) of one rank r with the column-owned kernel.  chained: launch
// with programmatic stream serialisation behind the previous rollout launch on the stream.
int launch_rollouts_cols(RolloutBatch bt, int cand0, int n, int r, bool chained, cudaStream_t st) {
  int rc = 0, c = 0;
  if (n < 1 || !rollout_cols_shape(r, &rc, &c)) return DOPINF_E_UNSUPPORTED;
  void* fn = cols_kernel((dim_d(r) + RB5 - 1) / RB5, rc, bt.arith == DOPINF_ROLLOUT_DW);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * c), 1, 1);
  cfg.blockDim = dim3(RB5, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 2 : 1;
  void* args[] = {&bt, &cand0};
  DOPINF_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
  return launch_status();
}

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
  const int d = dim_d(r);
  int rc = 0, c_cols = 0;
  const bool cols = rollout_cols_shape(r, &rc, &c_cols) != 0;
  const int cluster = cols ? 0 : rollout_cluster_size(r, d, r >= 16 ? 4 : 1);
  if (!cols && !cluster) return DOPINF_E_UNSUPPORTED;
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
  bt.arith = DOPINF_ROLLOUT_FP64;
  if (cols) return launch_rollouts_cols(bt, 0, 1, r, false, as_stream(stream));
  return launch_rollouts(bt, cluster, as_stream(stream));
}
