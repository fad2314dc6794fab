// Rollouts of learned quadratic ROMs (Section 3.5): the discrete map of
// eq. ROM_quad_time_discrete, or classical RK4 on eq. ROM_quad_time_cont, with the training
// error and growth criterion of Step IV fused into the time loop.  One thread-block cluster
// per candidate, one launch per r (largest first), later launches chained by programmatic
// dependent launch so that they run side by side.  Two layouts of the same computation:
//  * rollout_cols_kernel (r <= 32): the operator in registers, 128 threads per CTA;
//  * rollout_big_kernel (32 < r <= 92): the operator rows in shared memory, 256 threads.
// Both in FP64 or in double-word FP32 arithmetic (with an FP64 pass over what the
// double-word pass hands back).
#include "common.cuh"
#include <cooperative_groups.h>
#include <math.h>

#include <map>
#include <type_traits>
#include <mutex>
#include <tuple>
#include <utility>

namespace cg = cooperative_groups;

namespace dopinf {
namespace {

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
constexpr size_t kSmemCeiling = 227 * 1024 - 64;  // dynamic shared memory a CTA may request
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

// Warp sum of each of the RC values per lane (RC = 1, 2, 4, 8); lane L returns the sum of row
// L >> (5 - log2 RC).
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
  } else if constexpr (RC == 4) {
    const bool up = lane & 16;
    const V k0 = add_v(up ? acc[2] : acc[0], shfl_x(up ? acc[0] : acc[2], 16));
    const V k1 = add_v(up ? acc[3] : acc[1], shfl_x(up ? acc[1] : acc[3], 16));
    const bool up8 = lane & 8;
    k = add_v(up8 ? k1 : k0, shfl_x(up8 ? k0 : k1, 8));
  } else {
    static_assert(RC == 8, "RC is 1, 2, 4 or 8");
    const bool up = lane & 16;
    V h[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) h[m] = add_v(up ? acc[4 + m] : acc[m], shfl_x(up ? acc[m] : acc[4 + m], 16));
    const bool up8 = lane & 8;
    const V j0 = add_v(up8 ? h[2] : h[0], shfl_x(up8 ? h[0] : h[2], 8));
    const V j1 = add_v(up8 ? h[3] : h[1], shfl_x(up8 ? h[1] : h[3], 8));
    const bool up4 = lane & 4;
    k = add_v(up4 ? j1 : j0, shfl_x(up4 ? j0 : j1, 4));
  }
#pragma unroll
  for (int o = (RC == 8 ? 2 : RC == 4 ? 4 : 8); o > 0; o >>= 1) k = add_v(k, shfl_x(k, o));
  return k;
}

template <int NT, int RC, bool DW>
__global__ void __launch_bounds__(RB5, RC == 8 ? 3 : (DW ? 5 : 6)) rollout_cols_kernel(RolloutBatch bt, int cand0) {
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
    // metrics: the largest num/den (one square root at the end), the largest |q - mu| as an
    // integer maximum of bit patterns.  FP64: growth decided by a band
    // of 2^-40 around max_growth * denom with the division only inside it.  Double-word: the
    // state differs from the FP64 one by rounding, so a growth inside a band of 2^-20 around
    // the threshold hands the candidate to the FP64 kernel instead of deciding it here; since
    // the growth maximum only rises, a candidate stopped for growth above the band stops at
    // the same step in FP64, and a valid one stays below the threshold there too.
    // the training error as the largest num_t / ||qhat_t||^2, with the reciprocals formed once
    // per r, held as the bits of a non-negative double (an integer maximum)
    unsigned long long ratb = 0ull;
    unsigned long long gnumb = 0ull;
    const double thr = bt.max_growth * denom;
    const bool band_ok = denom > 0.0 && isfinite(thr) && thr > 0.0;
    const double bw = DW ? 0x1p-20 : 0x1p-40;
    const unsigned long long band_lo =
        band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 - bw)) : 0ull;
    const unsigned long long band_hi =
        band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 + bw)) : ~0ull;
    int st = 0;
    double icur = (lane == 0 && bt.metrics && bt.k > 0) ? cd.inv_den[0] : 0.0;

    // metrics of state t (warp 0); lane 0 publishes the stop decision.  The finiteness test and
    // the maxima are integer operations on the encodings (FP64 issue is scarce on this path).
    auto check = [&](int64_t t) {
      if constexpr (DW) qv = dw_value(qw);
      bool fin = !own || ((((unsigned long long)__double_as_longlong(qv)) >> 52) & 0x7ffull) != 0x7ffull;
      unsigned long long devb = 0ull;
      double num = 0.0;
      if (own && bt.metrics) {
        devb = (unsigned long long)__double_as_longlong(qv - mu) & 0x7fffffffffffffffull;
        if (t < bt.k) num = (qv - hcur) * (qv - hcur);
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
          const double v1[1] = {num};
          num = warp_rows_sum<1>(v1, lane);
        }
        if (lane == 0 && fin) {
          gnumb = devb > gnumb ? devb : gnumb;
          if (t < bt.k) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(num * icur);
            ratb = b > ratb ? b : ratb;
          }
        }
      }
      if (lane == 0) {
        if (!fin) {
          st = DW ? kStatusRedo : 2;
          stop = 1;
        } else if (bt.metrics && gnumb >= band_lo) {
          if constexpr (DW) {
            st = gnumb > band_hi ? 3 : kStatusRedo;
            stop = 1;
          } else if (gnumb > band_hi || __longlong_as_double((long long)gnumb) / denom >= bt.max_growth) {
            st = 3;
            stop = 1;
          }
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
      double hnext = 0.0, inext = 0.0;
      if (own && bt.metrics && t + 1 < bt.k) hnext = bt.Qhat[lane + (t + 1) * bt.ldqh];
      if (lane == 0 && warp == 0 && bt.metrics && t + 1 < bt.k) inext = cd.inv_den[t + 1];
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
      icur = inext;
    }
    cl.sync();  // no CTA leaves while a peer may still read its partial sums
    if (rank == 0 && tid == 0) {
      if (DW && st == kStatusRedo) {
        bt.status[cd.cand] = kStatusRedo;  // the FP64 kernel rolls this candidate out again
      } else {
        if (bt.steps) bt.steps[cd.cand] = t_end;
        if (bt.metrics) {
          bt.status[cd.cand] = st;
          bt.train_err[cd.cand] = st == 0 ? sqrt(__longlong_as_double((long long)ratb)) : INFINITY;
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
  static const F tab[2][5][4] = {
      {{cols_kernel_ptr<1, 1, false>, cols_kernel_ptr<1, 2, false>, cols_kernel_ptr<1, 4, false>, cols_kernel_ptr<1, 8, false>},
       {cols_kernel_ptr<2, 1, false>, cols_kernel_ptr<2, 2, false>, cols_kernel_ptr<2, 4, false>, cols_kernel_ptr<2, 8, false>},
       {cols_kernel_ptr<3, 1, false>, cols_kernel_ptr<3, 2, false>, cols_kernel_ptr<3, 4, false>, cols_kernel_ptr<3, 8, false>},
       {cols_kernel_ptr<4, 1, false>, cols_kernel_ptr<4, 2, false>, cols_kernel_ptr<4, 4, false>, cols_kernel_ptr<4, 8, false>},
       {cols_kernel_ptr<5, 1, false>, cols_kernel_ptr<5, 2, false>, cols_kernel_ptr<5, 4, false>, cols_kernel_ptr<5, 8, false>}},
      {{cols_kernel_ptr<1, 1, true>, cols_kernel_ptr<1, 2, true>, cols_kernel_ptr<1, 4, true>, cols_kernel_ptr<1, 8, true>},
       {cols_kernel_ptr<2, 1, true>, cols_kernel_ptr<2, 2, true>, cols_kernel_ptr<2, 4, true>, cols_kernel_ptr<2, 8, true>},
       {cols_kernel_ptr<3, 1, true>, cols_kernel_ptr<3, 2, true>, cols_kernel_ptr<3, 4, true>, cols_kernel_ptr<3, 8, true>},
       {cols_kernel_ptr<4, 1, true>, cols_kernel_ptr<4, 2, true>, cols_kernel_ptr<4, 4, true>, cols_kernel_ptr<4, 8, true>},
       {cols_kernel_ptr<5, 1, true>, cols_kernel_ptr<5, 2, true>, cols_kernel_ptr<5, 4, true>, cols_kernel_ptr<5, 8, true>}},
  };
  const int ri = rc == 1 ? 0 : rc == 2 ? 1 : rc == 4 ? 2 : rc == 8 ? 3 : -1;
  if (nt < 1 || nt > 5 || ri < 0) return nullptr;
  return tab[dw ? 1 : 0][nt - 1][ri]();
}

int g_rows_want = 4;  // tunable: rows of O per CTA in the column-owned rollouts

// Whether a cluster of c CTAs of this kernel (threads per CTA, dynamic shared memory) can be
// resident (sizes above 8 need the non-portable attribute and enough SMs in one GPC); cached
// per kernel, size and shared memory.
bool cluster_fits(void* fn, int c, int threads = RB5, size_t smem = 0) {
  static std::mutex mu;
  static std::map<std::tuple<void*, int, size_t>, bool> cache;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(fn, c, smem);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  bool ok = true, refused = false;
  if (c > 8) {
    ok = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    refused = !ok;
  }
  if (ok && smem > 48 * 1024) {
    // the function's ceiling, not this launch's size: launches of the same kernel for other r
    // (other sizes) must stay valid, also inside a graph captured later
    ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCeiling) == cudaSuccess;
    refused = refused || !ok;
  }
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
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

// ---------------------------------------------------------------------------------------
// Column-owned rollouts for 32 < r <= 92 (the batched-learn workloads reach r = 80,
// d = 3321; at r = 92 six rows of d = 4371 fill the 227 KB of shared memory).  The operator no
// longer fits registers, so each CTA keeps its RC rows of O in
// shared memory (row rho at rho * d: a warp reads 32 consecutive entries of a row, free of
// bank conflicts), and 256 threads walk the d columns: thread tid forms phi_a for the
// columns a = tid + 256 j from the stage state and adds O[i][a] phi_a into its RC row sums.
//  * a transposed butterfly reduces the RC row sums of each warp (padded to 4 or 8 rows) to
//    one sum per row; the eight warp sums of a row are added in a fixed tree by a lane of
//    warp 1, which stores the row's value into the evaluation buffer of every CTA of the
//    cluster (distributed shared memory) before one cluster barrier (arrive.release ...
//    wait.acquire);
//  * the evaluation buffers alternate by evaluation parity, so a CTA that runs ahead never
//    writes into a buffer a slower peer is still reading;
//  * warp 0 owns the state (lane L: entries L, L + 32, L + 64), applies the RK4 stage
//    combination identically in every CTA and forms the metrics of state t between its
//    arrival at the first barrier of step t and its wait there.
// The row sums are the same trees over the same column partial sums whatever RC and the
// cluster size are, so the results do not depend on the launch shape.  Arithmetic: FP64, or
// double-word with the FP64 hand-back rules of the kernel for r <= 32.
constexpr int RBB = 256;
constexpr int NWB = RBB / 32;
constexpr int kMaxRB = 96;       // state entries: three per lane of warp 0
constexpr int kMaxRBig = 92;     // largest r whose rows fit shared memory in clusters of 16
constexpr size_t kSmemBig = kSmemCeiling;  // dynamic shared memory per CTA
constexpr int kMinRowsB = 3, kMaxRowsB = 8;

struct BigLayout {
  size_t o, pair, x, k, part, total;
};

// Shared memory of one CTA holding rc rows of an operator of width d (8 bytes per entry in
// both arithmetics: a double, or the (high, low) binary32 pair).
__host__ __device__ inline BigLayout big_layout(int rc, int d) {
  BigLayout L;
  size_t off = 0;
  L.o = off;
  off += (size_t)rc * d * 8;
  L.pair = off;
  off += ((size_t)d * 4 + 15) / 16 * 16;
  L.x = off;  // stage state, kMaxRB + 2 entries (x[r] = 1)
  off += (size_t)(kMaxRB + 2) * 8;
  L.k = off;  // evaluation results by parity
  off += (size_t)2 * kMaxRB * 8;
  L.part = off;  // warp sums [warp][row]
  off += (size_t)NWB * kMaxRowsB * 8;
  L.total = (off + 15) / 16 * 16;
  return L;
}

template <int RC, bool DW>
__global__ void __launch_bounds__(RBB, 2) rollout_big_kernel(RolloutBatch bt, int cand0) {
  using Part = typename std::conditional<DW, csum, double>::type;
  constexpr int RCP = RC <= 4 ? 4 : 8;  // rows of the transposed butterfly (zero-padded)
  extern __shared__ __align__(16) unsigned char smb[];
  __shared__ int s_stop, s_bad;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) pdl_trigger();
  const RolloutCand cd = bt.cands ? bt.cands[cand0 + (int)(blockIdx.x / C)] : bt.one;
  const int r = cd.r, d = cd.d, i0 = rank * RC;
  const int nrow = r - i0 < 0 ? 0 : (r - i0 < RC ? r - i0 : RC);  // rows this CTA owns
  const BigLayout L = big_layout(RC, d);
  double* Os = reinterpret_cast<double*>(smb + L.o);     // FP64 operator rows
  float2* Ow = reinterpret_cast<float2*>(smb + L.o);     // double-word operator rows
  unsigned* pair = reinterpret_cast<unsigned*>(smb + L.pair);
  double* xs = reinterpret_cast<double*>(smb + L.x);
  float2* xw = reinterpret_cast<float2*>(smb + L.x);
  double* kd = reinterpret_cast<double*>(smb + L.k);
  float2* kw = reinterpret_cast<float2*>(smb + L.k);
  Part* part = reinterpret_cast<Part*>(smb + L.part);

  const int want = (!DW && bt.redo) ? kStatusRedo : 0;
  bool run = !(bt.metrics && bt.status[cd.cand] != want);
  if (!run && !bt.redo && rank == 0 && tid == 0 && bt.status[cd.cand] != kStatusRedo) {
    bt.train_err[cd.cand] = INFINITY;
    bt.growth[cd.cand] = INFINITY;
    if (bt.steps) bt.steps[cd.cand] = 0;
  }
  if (!run) {
    if (blockIdx.x == gridDim.x - 1 && tid == 0) pdl_wait();
    return;
  }

  // operator rows (zero rows past r), the phi index pairs, the constant entry of the state
  bool bad = false;
  for (int e = tid; e < RC * d; e += RBB) {
    const int rho = e / d, a = e - rho * d, i = i0 + rho;
    const double v = i < r ? cd.O[i + (size_t)a * cd.ldo] : 0.0;
    if constexpr (DW) {
      bad = bad || !(fabs(v) <= kDwRange);
      const dw w = dw_of(v);
      Ow[e] = make_float2(w.h, w.l);
    } else {
      Os[e] = v;
    }
  }
  for (int i = tid; i < r; i += RBB) {
    const int off = r + i * r - i * (i - 1) / 2;  // column of x_i x_i
    for (int j = i; j < r; ++j) pair[off + j - i] = (unsigned)i | ((unsigned)j << 8);
    pair[i] = (unsigned)i | ((unsigned)r << 8);  // linear term x_i * 1
  }
  if (tid == 0) pair[d - 1] = (unsigned)r | ((unsigned)r << 8);  // constant term 1 * 1
  if constexpr (DW) {
    if (warp == 0)
      for (int j = 0; j < 3; ++j) {
        const int i = lane + 32 * j;
        if (i < r) bad = bad || !(fabs(bt.q0[i]) <= kDwRange);
      }
    const int any = __syncthreads_or(bad);
    if (tid == 0) s_bad = any;
  }
  cl.sync();  // every CTA has started and published its flag before any remote access
  if constexpr (DW) {
    int peer = 0;
    if (tid < C) peer = *cl.map_shared_rank(&s_bad, (unsigned)tid);
    if (__syncthreads_or(peer)) {
      if (rank == 0 && tid == 0) bt.status[cd.cand] = kStatusRedo;
      cl.sync();  // every CTA has read its peers' flags before any of them leaves
      if (blockIdx.x == gridDim.x - 1 && tid == 0) pdl_wait();
      return;
    }
  }

  // state: warp 0, lane L owns entries L, L + 32, L + 64
  double qv[3], mu[3], hcur[3];
  dw qw[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int i = lane + 32 * j;
    const bool own = warp == 0 && i < r;
    qv[j] = own ? bt.q0[i] : 0.0;
    qw[j] = dw_of(qv[j]);
    mu[j] = (own && bt.metrics) ? cd.mu[i] : 0.0;
    hcur[j] = (own && bt.metrics && bt.k > 0) ? bt.Qhat[i] : 0.0;
    if (own) {
      if constexpr (DW)
        xw[i] = make_float2(qw[j].h, qw[j].l);
      else
        xs[i] = qv[j];
    }
  }
  if (tid == 0) {
    if constexpr (DW)
      xw[r] = make_float2(1.0f, 0.0f);
    else
      xs[r] = 1.0;
  }
  const double dt = bt.dt, h2 = 0.5 * dt, h6 = dt / 6.0;
  const dw dtw = dw_of(dt), h2w = dw_of(h2), h6w = dw_of(h6);
  const double denom = bt.metrics ? *cd.denom : 1.0;
  unsigned long long ratb = 0ull;  // largest num_t / ||qhat_t||^2 (bits of a non-negative double)
  unsigned long long gnumb = 0ull;
  const double thr = bt.max_growth * denom;
  const bool band_ok = denom > 0.0 && isfinite(thr) && thr > 0.0;
  const double bw = DW ? 0x1p-20 : 0x1p-40;
  const unsigned long long band_lo = band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 - bw)) : 0ull;
  const unsigned long long band_hi = band_ok ? (unsigned long long)__double_as_longlong(thr * (1.0 + bw)) : ~0ull;
  int st = 0;
  double icur = (warp == 0 && lane == 0 && bt.metrics && bt.k > 0) ? cd.inv_den[0] : 0.0;

  // metrics of state t (warp 0, the same values in every CTA); lane 0 publishes the decision
  auto check = [&](int64_t t) {
    bool fin = true;
    unsigned long long devb = 0ull;
    double num = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i = lane + 32 * j;
      if (i >= r) continue;
      if constexpr (DW) qv[j] = dw_value(qw[j]);
      fin = fin && ((((unsigned long long)__double_as_longlong(qv[j])) >> 52) & 0x7ffull) != 0x7ffull;
      if (bt.metrics) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(qv[j] - mu[j]) & 0x7fffffffffffffffull;
        devb = b > devb ? b : devb;
        if (t < bt.k) num += (qv[j] - hcur[j]) * (qv[j] - hcur[j]);
      }
      if (bt.traj && rank == 0) bt.traj_out[t * r + i] = qv[j];
    }
    fin = __all_sync(kFull, fin);
    if (bt.metrics) {
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(kFull, devb, o2);
        devb = ob > devb ? ob : devb;
      }
      if (t < bt.k) {
        const double v1[1] = {num};
        num = warp_rows_sum<1>(v1, lane);
      }
      if (lane == 0 && fin) {
        gnumb = devb > gnumb ? devb : gnumb;
        if (t < bt.k) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(num * icur);
          ratb = b > ratb ? b : ratb;
        }
      }
    }
    if (lane == 0) {
      int stop = 0;
      if (!fin) {
        st = DW ? kStatusRedo : 2;
        stop = 1;
      } else if (bt.metrics && gnumb >= band_lo) {
        if constexpr (DW) {
          st = gnumb > band_hi ? 3 : kStatusRedo;
          stop = 1;
        } else if (gnumb > band_hi || __longlong_as_double((long long)gnumb) / denom >= bt.max_growth) {
          st = 3;
          stop = 1;
        }
      }
      if (t + 1 >= bt.n_steps) stop = 1;
      s_stop = stop;
    }
  };

  // one right-hand-side evaluation at the stage state; the r results land in this CTA's
  // evaluation buffer of parity e & 1 (and in every peer's)
  unsigned e = 0;
  auto eval = [&](bool with_check, int64_t t) {
    Part acc[RCP];
#pragma unroll
    for (int rho = 0; rho < RCP; ++rho) acc[rho] = Part{};
    for (int a = tid; a < d; a += RBB) {
      const unsigned p = pair[a];
      const int ia = (int)(p & 0xffu), ib = (int)(p >> 8);
      if constexpr (DW) {
        const float2 xa = xw[ia], xb = xw[ib];
        const float ph = __fmul_rn(xa.x, xb.x);
        const float pl = __fmaf_rn(xa.y, xb.x, __fmaf_rn(xa.x, xb.y, __fmaf_rn(xa.x, xb.x, -ph)));
#pragma unroll
        for (int rho = 0; rho < RC; ++rho) {
          const float2 ov = Ow[rho * d + a];
          const float pr = __fmul_rn(ov.x, ph);
          const float err = __fmaf_rn(ov.y, ph, __fmaf_rn(ov.x, pl, __fmaf_rn(ov.x, ph, -pr)));
          const dw u = two_sum(acc[rho].s, pr);
          acc[rho].s = u.h;
          acc[rho].c = __fadd_rn(acc[rho].c, __fadd_rn(u.l, err));
        }
      } else {
        const double ph = xs[ia] * xs[ib];
#pragma unroll
        for (int rho = 0; rho < RC; ++rho) acc[rho] = fma(Os[rho * d + a], ph, acc[rho]);
      }
    }
    const Part v = warp_rows_sum<RCP>(acc, lane);
    constexpr int per = 32 / RCP;  // lanes holding each row's sum
    if ((lane & (per - 1)) == 0 && lane / per < RC) part[warp * kMaxRowsB + lane / per] = v;
    __syncthreads();
    const int buf = (int)(e & 1u);
    if (warp == 1 && lane < nrow) {
      const Part* pp = part + lane;
      const Part s = add_v(add_v(add_v(pp[0 * kMaxRowsB], pp[1 * kMaxRowsB]), add_v(pp[2 * kMaxRowsB], pp[3 * kMaxRowsB])),
                           add_v(add_v(pp[4 * kMaxRowsB], pp[5 * kMaxRowsB]), add_v(pp[6 * kMaxRowsB], pp[7 * kMaxRowsB])));
      const int i = i0 + lane;
      if constexpr (DW) {
        const dw s2 = two_sum(s.s, s.c);
        const float2 val = make_float2(s2.h, s2.l);
        for (int j = 0; j < C; ++j) cl.map_shared_rank(kw + buf * kMaxRB, (unsigned)j)[i] = val;
      } else {
        for (int j = 0; j < C; ++j) cl.map_shared_rank(kd + buf * kMaxRB, (unsigned)j)[i] = s;
      }
    }
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    if (with_check && warp == 0) {
      check(t);
      __syncwarp();
    }
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    ++e;
    return buf;
  };

  __syncthreads();
  int64_t t_end = 0;
  double k1d[3], k2d[3], k3d[3];
  dw k1w[3], k2w[3], k3w[3];
  for (int64_t t = 0;; ++t) {
    t_end = t;
    double hnext[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i = lane + 32 * j;
      hnext[j] = (warp == 0 && i < r && bt.metrics && t + 1 < bt.k) ? bt.Qhat[i + (t + 1) * bt.ldqh] : 0.0;
    }
    const double inext = (warp == 0 && lane == 0 && bt.metrics && t + 1 < bt.k) ? cd.inv_den[t + 1] : 0.0;
    int b = eval(true, t);
    if (bt.mode == DOPINF_DISCRETE) {
      if (warp == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int i = lane + 32 * j;
          if (i >= r) continue;
          if constexpr (DW) {
            const float2 kv = kw[b * kMaxRB + i];
            k1w[j] = dw{kv.x, kv.y};
            xw[i] = kv;
          } else {
            k1d[j] = kd[b * kMaxRB + i];
            xs[i] = k1d[j];
          }
        }
      }
      __syncthreads();
      if (s_stop) break;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if constexpr (DW)
          qw[j] = k1w[j];
        else
          qv[j] = k1d[j];
      }
    } else {
      // RK4: stage s reads its evaluation, forms the next stage state (products and sums
      // rounded separately, q + (dt/6)(((k1 + 2 k2) + 2 k3) + k4) at the end)
      for (int s = 0; s < 4; ++s) {
        if (s > 0) b = eval(false, t);
        if (warp == 0) {
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const int i = lane + 32 * j;
            if (i >= r) continue;
            if constexpr (DW) {
              const float2 kv = kw[b * kMaxRB + i];
              const dw kk{kv.x, kv.y};
              dw x;
              if (s == 0) {
                k1w[j] = kk;
                x = dw_add(qw[j], dw_mul(h2w, kk));
              } else if (s == 1) {
                k2w[j] = kk;
                x = dw_add(qw[j], dw_mul(h2w, kk));
              } else if (s == 2) {
                k3w[j] = kk;
                x = dw_add(qw[j], dw_mul(dtw, kk));
              } else {
                const dw sum = dw_add(dw_add(dw_add(k1w[j], dw_twice(k2w[j])), dw_twice(k3w[j])), kk);
                qw[j] = dw_add(qw[j], dw_mul(h6w, sum));
                x = qw[j];
              }
              xw[i] = make_float2(x.h, x.l);
            } else {
              const double kk = kd[b * kMaxRB + i];
              double x;
              if (s == 0) {
                k1d[j] = kk;
                x = __dadd_rn(qv[j], __dmul_rn(h2, kk));
              } else if (s == 1) {
                k2d[j] = kk;
                x = __dadd_rn(qv[j], __dmul_rn(h2, kk));
              } else if (s == 2) {
                k3d[j] = kk;
                x = __dadd_rn(qv[j], __dmul_rn(dt, kk));
              } else {
                const double sum = __dadd_rn(__dadd_rn(__dadd_rn(k1d[j], 2.0 * k2d[j]), 2.0 * k3d[j]), kk);
                qv[j] = __dadd_rn(qv[j], __dmul_rn(h6, sum));
                x = qv[j];
              }
              xs[i] = x;
            }
          }
        }
        __syncthreads();
        if (s == 0 && s_stop) break;
      }
      if (s_stop) break;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) hcur[j] = hnext[j];
    icur = inext;
  }
  cl.sync();  // no CTA leaves while a peer may still store into its shared memory
  if (rank == 0 && tid == 0) {
    if (DW && st == kStatusRedo) {
      bt.status[cd.cand] = kStatusRedo;
    } else {
      if (bt.steps) bt.steps[cd.cand] = t_end;
      if (bt.metrics) {
        bt.status[cd.cand] = st;
        bt.train_err[cd.cand] = st == 0 ? sqrt(__longlong_as_double((long long)ratb)) : INFINITY;
        bt.growth[cd.cand] = st == 2 ? INFINITY : __longlong_as_double((long long)gnumb) / denom;
      }
      if (bt.traj && bt.finite) *bt.finite = st == 2 ? 0 : 1;
    }
  }
  if (blockIdx.x == gridDim.x - 1 && tid == 0) pdl_wait();
}

template <int RC, bool DW>
void* big_kernel_ptr() {
  return reinterpret_cast<void*>(&rollout_big_kernel<RC, DW>);
}

void* big_kernel(int rc, bool dw) {
  using F = void* (*)();
  static const F tab[2][kMaxRowsB - kMinRowsB + 1] = {
      {big_kernel_ptr<3, false>, big_kernel_ptr<4, false>, big_kernel_ptr<5, false>, big_kernel_ptr<6, false>,
       big_kernel_ptr<7, false>, big_kernel_ptr<8, false>},
      {big_kernel_ptr<3, true>, big_kernel_ptr<4, true>, big_kernel_ptr<5, true>, big_kernel_ptr<6, true>,
       big_kernel_ptr<7, true>, big_kernel_ptr<8, true>},
  };
  if (rc < kMinRowsB || rc > kMaxRowsB) return nullptr;
  return tab[dw ? 1 : 0][rc - kMinRowsB]();
}

int g_rows_big_want = 4;  // tunable: rows of O per CTA for r > 32

}  // namespace

bool rollout_cols_supported(int r) { return r >= 1 && r <= kMaxR5 && (dim_d(r) + RB5 - 1) / RB5 <= 5; }

// Rows per CTA and cluster size of the column-owned kernel for rank r (0 if none fits), for
// both arithmetics (the FP64 kernel re-runs what the double-word one hands back).
int rollout_cols_shape(int r, int* rows, int* cluster) {
  if (!rollout_cols_supported(r)) return 0;
  const int nt = (dim_d(r) + RB5 - 1) / RB5;
  for (int rc = g_rows_want; rc <= 8; rc *= 2) {
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

int g_arith = DOPINF_ROLLOUT_FP64;  // tunable: arithmetic of the learn rollouts (the paper's FP64)

int rollout_set_arith(int a) {
  const int prev = g_arith;
  if (a == DOPINF_ROLLOUT_FP64 || a == DOPINF_ROLLOUT_DW) g_arith = a;
  return prev;
}

int rollout_arith() { return g_arith; }

int rollout_set_rows(int rc) {
  const int prev = g_rows_want;
  if (rc == 1 || rc == 2 || rc == 4 || rc == 8) g_rows_want = rc;
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

bool rollout_big_supported(int r) { return r > kMaxR5 && r <= kMaxRBig; }

// Rows per CTA, cluster size and shared memory of the kernel for 32 < r <= 92 (0 if none
// fits): the preferred rows, raised until the cluster has at most 16 CTAs and both
// arithmetics' kernels can be resident.
int rollout_big_shape(int r, int* rows, int* cluster, size_t* smem) {
  if (!rollout_big_supported(r)) return 0;
  const int d = dim_d(r);
  int rc = g_rows_big_want;
  if (rc * 16 < r) rc = (r + 15) / 16;
  for (; rc <= kMaxRowsB; ++rc) {
    const int c = (r + rc - 1) / rc;
    const size_t sm = big_layout(rc, d).total;
    if (sm > kSmemBig) break;
    void* f64 = big_kernel(rc, false);
    void* fdw = big_kernel(rc, true);
    if (f64 && fdw && cluster_fits(f64, c, RBB, sm) && cluster_fits(fdw, c, RBB, sm)) {
      *rows = rc;
      *cluster = c;
      *smem = sm;
      return 1;
    }
  }
  return 0;
}

int rollout_set_rows_big(int rc) {
  const int prev = g_rows_big_want;
  if (rc >= kMinRowsB && rc <= kMaxRowsB) g_rows_big_want = rc;
  return prev;
}

// Candidates [cand0, cand0 + n) of one rank r > 32; chained as launch_rollouts_cols.
int launch_rollouts_big(RolloutBatch bt, int cand0, int n, int r, bool chained, cudaStream_t st) {
  int rc = 0, c = 0;
  size_t smem = 0;
  if (n < 1 || !rollout_big_shape(r, &rc, &c, &smem)) return DOPINF_E_UNSUPPORTED;
  void* fn = big_kernel(rc, bt.arith == DOPINF_ROLLOUT_DW);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * c), 1, 1);
  cfg.blockDim = dim3(RBB, 1, 1);
  cfg.dynamicSmemBytes = smem;
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

bool rollout_supported(int r) { return rollout_cols_supported(r) || rollout_big_supported(r); }

// Shape of the launch for rank r with either kernel (0 if none fits).
int rollout_shape(int r) {
  int rc = 0, c = 0;
  size_t sm = 0;
  return r <= kMaxR5 ? rollout_cols_shape(r, &rc, &c) : rollout_big_shape(r, &rc, &c, &sm);
}

int launch_rollouts_rank(RolloutBatch bt, int cand0, int n, int r, bool chained, cudaStream_t st) {
  return r <= kMaxR5 ? launch_rollouts_cols(bt, cand0, n, r, chained, st)
                     : launch_rollouts_big(bt, cand0, n, r, chained, st);
}

}  // namespace dopinf

using namespace dopinf;


using namespace dopinf;

DOPINF_API int dopinf_rollout(const double* O, int r, int64_t ldo, const double* q0, int64_t n_steps, int mode,
                              double dt, double* Qtilde, int* finite, void* stream) {
  if (!O || !q0 || !Qtilde || r < 1 || r > 255 || ldo < r || n_steps < 1) return DOPINF_E_ARG;
  if (mode != DOPINF_DISCRETE && mode != DOPINF_CONTINUOUS_RK4) return DOPINF_E_ARG;
  if (!rollout_supported(r) || !rollout_shape(r)) return DOPINF_E_UNSUPPORTED;
  const int d = dim_d(r);
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
  return launch_rollouts_rank(bt, 0, 1, r, false, as_stream(stream));
}
