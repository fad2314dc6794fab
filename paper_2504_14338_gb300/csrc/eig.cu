// Step III of dOpInf (Section 3.4): symmetric eigendecomposition of the Gram matrix
// (eq. mos_Sigma_W), the retained-energy rank (eq. ret_energy) and the basis-free
// projection T_r = U_r Lambda_r^{-1/2}, Qhat = T_r^T D (eqs. MoS_POD_basis, dOpInf_projection).
//
// Only the leading r_cap eigenpairs are formed (the paper notes that a partial eigensolve
// suffices when r is known; the energy rule needs only trace(D) besides them):
//  1. Householder reduction of D to tridiagonal form T = H^T D H, one reflector per column:
//     one cooperative launch with one grid barrier per column, or three launches per column;
//  2. the r_cap largest eigenvalues of T by Sturm-count multisection: a first round of 38912
//     points shared by all eigenvalues over the whole GPU, then one CTA of 8 warps per
//     eigenvalue, 256 trial points per round;
//  3. their eigenvectors by inverse iteration with the partially pivoted tridiagonal LU,
//     re-orthogonalised (classical Gram-Schmidt, twice) against earlier vectors whose
//     eigenvalues lie within 1e-3 ||T||;
//  4. back-transformation by the stored reflectors in blocks of 16 (compact WY form), sign
//     rule (largest-magnitude entry positive, lowest index on ties);
//  5. T_r and Qhat = T_r^T D with the FP64 TN product.
// All arithmetic is FP64; every reduction has a fixed order.
#include "common.cuh"
#include <cooperative_groups.h>
#include <math.h>
#include <float.h>

namespace dopinf {
namespace {

constexpr int EB = 256;  // threads per block for the reduction kernels
// block-reduction scratch: the warp partials (up to 32), the result, three broadcast scalars
constexpr int kShSlots = 36;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  // fixed-order tree: a butterfly in every warp, then one over the warp partials in warp 0
  // (lanes beyond the warp count add zeros), broadcast through sh[32].  FP64 additions issue
  // slowly here, so the second level runs in one warp only.
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = l < nw ? sh[l] : 0.0;
    int pw = 1;
    while (pw < nw) pw <<= 1;
    for (int o = pw >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

// The sums of the tridiagonalisation run over the first RW = 128 threads (one warp per
// scheduler: FP64 instructions issue slowly, and a warp pair on one scheduler would share its
// pipe): thread t < RW adds the entries t, t + RW, ... in order, each of the four warps sums its
// lanes by a butterfly, warp 0 adds the four warp sums by a butterfly, and the result is
// broadcast through sh[32].  block_sum_lo is called by all threads of the block (the others
// pass nothing and wait); block_sum_named by warps 0-3 only, which then synchronise among
// themselves on named barrier 1 while the other warps work on.
constexpr int RW = 128;
__device__ __forceinline__ void bar_lo() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ double warp_pair_sum4(double* sh) {
  const int l = threadIdx.x & 31;
  double s = l < 4 ? sh[l] : 0.0;
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}
__device__ __forceinline__ double block_sum_lo(double v, double* sh) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (w < 4) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[w] = v;
  }
  __syncthreads();
  if (w == 0) {
    const double s = warp_pair_sum4(sh);
    if (l == 0) sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}
__device__ __forceinline__ double block_sum_named(double v, double* sh) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  bar_lo();
  if (l == 0) sh[w] = v;
  bar_lo();
  if (w == 0) {
    const double s = warp_pair_sum4(sh);
    if (l == 0) sh[32] = s;
  }
  bar_lo();
  return sh[32];
}

// Reflector of column j: x = A[j+1:k, j] -> (I - tau v v^T) x = beta e1 with v[0] = 1.
// v overwrites A[j+1:k, j]; d[j] = A[j][j], e[j] = beta.
__global__ void __launch_bounds__(EB) hh_gen(double* A, int64_t k, int64_t j, double* d, double* e, double* tau) {
  __shared__ double sh[kShSlots];
  double* x = A + j * k;  // column j
  double part = 0.0;
  if (threadIdx.x < RW)
    for (int64_t i = j + 2 + threadIdx.x; i < k; i += RW) part += x[i] * x[i];
  const double sigma2 = block_sum_lo(part, sh);
  const double x0 = x[j + 1];
  double t, beta, scal;
  if (sigma2 == 0.0) {
    t = 0.0;
    beta = x0;
    scal = 0.0;
  } else {
    const double nrm = sqrt(x0 * x0 + sigma2);
    beta = x0 >= 0.0 ? -nrm : nrm;
    t = (beta - x0) / beta;
    scal = 1.0 / (x0 - beta);
  }
  __syncthreads();
  if (t != 0.0)
    for (int64_t i = j + 2 + threadIdx.x; i < k; i += blockDim.x) x[i] *= scal;
  if (threadIdx.x == 0) {
    d[j] = x[j];
    e[j] = beta;
    tau[j] = t;
    x[j + 1] = 1.0;
  }
}

// p = tau * A22 v with A22 = A[j+1:, j+1:], one warp per row (row i of A22 = column i).
__global__ void __launch_bounds__(EB) hh_symv(const double* A, int64_t k, int64_t j, const double* tau, double* p) {
  const double t = tau[j];
  if (t == 0.0) return;
  const int64_t m = k - j - 1;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const double* col = A + (j + 1 + row) * k + (j + 1);
  const double* v = A + j * k + (j + 1);
  double s = 0.0;
  for (int64_t l = lane; l < m; l += 32) s = fma(col[l], v[l], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) p[row] = t * s;
}

// A22 -= v w^T + w v^T with w = p - (tau/2)(p.v) v.  Each block recomputes p.v in a fixed
// order and updates a group of columns of A22 (full symmetric storage).
constexpr int R2_COLS = 16;
__global__ void __launch_bounds__(EB) hh_rank2(double* A, int64_t k, int64_t j, const double* tau, const double* p) {
  __shared__ double sh[kShSlots];
  const double t = tau[j];
  if (t == 0.0) return;
  const int64_t m = k - j - 1;
  const double* v = A + j * k + (j + 1);
  double part = 0.0;
  if (threadIdx.x < RW)
    for (int64_t l = threadIdx.x; l < m; l += RW) part = fma(p[l], v[l], part);
  const double alpha = -0.5 * t * block_sum_lo(part, sh);
  const int64_t c0 = (int64_t)blockIdx.x * R2_COLS;
  for (int cc = 0; cc < R2_COLS; ++cc) {
    const int64_t c = c0 + cc;
    if (c >= m) break;
    const double vc = v[c], wc = fma(alpha, vc, p[c]);
    double* col = A + (j + 1 + c) * k + (j + 1);
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
      const double wr = fma(alpha, v[r], p[r]);
      col[r] = fma(-wr, vc, fma(-v[r], wc, col[r]));
    }
  }
}

__global__ void hh_tail(const double* A, int64_t k, double* d, double* e, double* tau) {
  if (threadIdx.x != 0) return;
  if (k >= 2) {
    d[k - 2] = A[(k - 2) * k + (k - 2)];
    e[k - 2] = A[(k - 2) * k + (k - 1)];
    tau[k - 2] = 0.0;
  }
  d[k - 1] = A[(k - 1) * k + (k - 1)];
  e[k - 1] = 0.0;
  tau[k - 1] = 0.0;
}

// ---------------------------------------------------------------------------------------
// The same reduction in one cooperative launch.  The rank-2 update of step j and the row c of
// the next product p_{j+1} = tau_{j+1} A22 v_{j+1} (the matrix is symmetric, so row c is
// column c) are formed by the CTA that owns column c, and one grid barrier per column
// separates the steps.  Every CTA forms the next reflector redundantly from its own copy of
// the updated column j+1, with the reductions in the same fixed order as the three-launch
// version, so the results agree bit for bit.
// The barrier is a counter with a bounded wait: on expiry the kernel sets an error word and
// every CTA returns.
constexpr int TB = 256;
constexpr uint64_t kBarNs = 2000000000ull;
struct GridBar {
  unsigned count, err;
};

__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Arrival is one add on a counter that only grows (zeroed before the launch): the barrier of
// step s is passed once it reaches (s + 1) x grid, so the last arrival's add is all the others
// wait for.  stall = 1 (a test of the error path) raises every target by one: the count can
// never reach it, so every wait runs into its limit.
__device__ bool grid_sync(GridBar* b, unsigned& epoch, unsigned stall) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned target = (++epoch) * gridDim.x + stall;
    __threadfence();
    const unsigned prev = atomicAdd(&b->count, 1u);
    if (prev + 1u != target) {
      volatile unsigned* vcount = &b->count;
      volatile unsigned* verr = &b->err;
      const uint64_t t0 = gtimer_ns();
      while ((int)(*vcount - target) < 0) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (gtimer_ns() - t0 > kBarNs) {
          atomicOr(&b->err, 1u);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// Column c of the trailing matrix belongs to CTA c mod grid and is handled by warp
// 4 + (c div grid) mod 4 for the whole reduction.  With `resident`, a CTA keeps its columns in
// shared memory (slot c div grid) and writes to A only the columns that another CTA reads there
// (the next column, and the last one for the final 2 x 2 block); without, the columns live in A.
// Per step, after the barrier, each CTA fetches p_{j+1} and column j+2 together (one round
// trip to L2), forms w_j = p_j + alpha_j v_j once (in place of p_j) and the updated column
// j+1.  Then warps 0-3 form the reflector of that column while warps 4-7 apply update j to the
// CTA's trailing columns, and warps 4-7 form the CTA's entries of p_{j+1} = tau A22 v_{j+1}.
__global__ void __launch_bounds__(TB) hh_tridiag_coop(double* A, int64_t k, double* d, double* e, double* tau,
                                                      double* pg, GridBar* bar, int resident, unsigned stall) {
  extern __shared__ double smd[];
  double* vj = smd;          // v_j (rows j+1..k-1)
  double* pj = smd + k;      // p_j, then w_j
  double* vn = smd + 2 * k;  // column j+1 as update j-1 left it, after update j, then v_{j+1}
  double* own = smd + 3 * k; // resident: this CTA's columns
  __shared__ double sh[kShSlots];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t grid = gridDim.x;
  if (resident) {
    for (int64_t lc = 0; blockIdx.x + lc * grid < k; ++lc) {
      const double* src = A + (blockIdx.x + lc * grid) * k;
      for (int64_t r = threadIdx.x; r < k; r += blockDim.x) own[lc * k + r] = src[r];
    }
  }
  for (int64_t r = threadIdx.x; r < k; r += blockDim.x) vn[r] = __ldcg(A + r);  // column 0
  __syncthreads();
  double tj = 0.0;  // tau of the pending update (0: none)
  unsigned epoch = 0;
  for (int64_t j = -1; j + 2 < k; ++j) {
    const bool upd = j >= 0 && tj != 0.0;
    const int64_t c1 = j + 1;
    if (upd) {
      // (a) the pending update of step j: alpha = -tau_j/2 (p_j . v_j), w = p + alpha v
      const int64_t m = k - j - 1;
      double part = 0.0;
      if (threadIdx.x < RW)
        for (int64_t l = threadIdx.x; l < m; l += RW) part = fma(pj[j + 1 + l], vj[j + 1 + l], part);
      const double alpha = -0.5 * tj * block_sum_lo(part, sh);
      for (int64_t r = c1 + threadIdx.x; r < k; r += blockDim.x) pj[r] = fma(alpha, vj[r], pj[r]);
      __syncthreads();
      // (b) column j+1 after update j, rows j+1..k-1
      const double vc = vj[c1], wc = pj[c1];
      for (int64_t r = c1 + threadIdx.x; r < k; r += blockDim.x) vn[r] = fma(-pj[r], vc, fma(-vj[r], wc, vn[r]));
      __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d[c1] = vn[c1];
    // (c) the stored reflector of column j (nobody reads column j any more)
    if (blockIdx.x == 0 && j >= 0) {
      for (int64_t r = j + 1 + threadIdx.x; r < k; r += blockDim.x) A[r + j * k] = vj[r];
    }
    if (c1 + 2 >= k) {
      // last step: the trailing 2 x 2 block
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        e[c1] = vn[c1 + 1];
        tau[c1] = 0.0;
        const int64_t r = k - 1;
        double a = __ldcg(A + r + r * k);
        if (upd) {
          const double vc = vj[r], wc = pj[r];
          a = fma(-wc, vc, fma(-vj[r], wc, a));
        }
        d[r] = a;
        e[r] = 0.0;
        tau[r] = 0.0;
      }
      return;
    }
    const int64_t r0 = c1 + 1;
    if (warp < 4) {
      // (d) the reflector of column j+1 in place in vn (rows j+2..k-1, vn[j+2] = 1), the
      // scalars by threads 0 (tau, beta) and 32 (the scale) side by side
      double part = 0.0;
      for (int64_t i = c1 + 2 + threadIdx.x; i < k; i += RW) part += vn[i] * vn[i];
      const double sigma2 = block_sum_named(part, sh);
      if (threadIdx.x == 0 || threadIdx.x == 32) {
        const double x0 = vn[r0];
        double bb = x0, q = 0.0;
        if (sigma2 != 0.0) {
          const double nrm = sqrt(x0 * x0 + sigma2);
          bb = x0 >= 0.0 ? -nrm : nrm;
          q = threadIdx.x == 0 ? (bb - x0) / bb : 1.0 / (x0 - bb);
        }
        if (threadIdx.x == 0) {
          sh[33] = q;
          sh[34] = bb;
        } else {
          sh[35] = q;
        }
      }
      bar_lo();
      if (sh[33] != 0.0) {
        const double scal = sh[35];
        for (int64_t i = c1 + 2 + threadIdx.x; i < k; i += RW) vn[i] *= scal;
      }
      bar_lo();
      if (threadIdx.x == 0) vn[r0] = 1.0;
    } else if (upd) {
      // (e) update j on the trailing columns c >= j+2 (rows >= j+2)
      for (int64_t lc = warp - 4; blockIdx.x + lc * grid < k; lc += 4) {
        const int64_t c = blockIdx.x + lc * grid;
        if (c < r0) continue;
        double* col = A + c * k;
        double* cs = resident ? own + lc * k : col;
        const bool through = !resident || c == r0 || c == k - 1;
        const double vc = vj[c], wc = pj[c];
        for (int64_t l = lane; l < k - r0; l += 32) {
          const int64_t r = r0 + l;
          double a = resident ? cs[r] : __ldcg(col + r);
          a = fma(-pj[r], vc, fma(-vj[r], wc, a));
          if (resident) cs[r] = a;
          if (through) col[r] = a;
        }
      }
    }
    __syncthreads();
    const double tn = sh[33];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      e[c1] = sh[34];
      tau[c1] = tn;
    }
    // (f) this CTA's entries of p_{j+1} (warps 4-7, one column per warp at a time)
    if (warp >= 4 && tn != 0.0) {
      for (int64_t lc = warp - 4; blockIdx.x + lc * grid < k; lc += 4) {
        const int64_t c = blockIdx.x + lc * grid;
        if (c < r0) continue;
        const double* cs = resident ? own + lc * k : A + c * k;
        double s = 0.0;
        for (int64_t l = lane; l < k - r0; l += 32) {
          const int64_t r = r0 + l;
          s = fma(resident ? cs[r] : __ldcg(cs + r), vn[r], s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) pg[c] = tn * s;
      }
    }
    if (!grid_sync(bar, epoch, stall)) return;
    // (g) v_{j+1} becomes the pending reflector; p_{j+1} and column j+2 (rows j+2..k-1, as
    // update j left it) from global memory, both loads issued before either is stored
    const double* cn = A + (c1 + 1) * k;
    for (int64_t r = c1 + threadIdx.x; r < k; r += blockDim.x) {
      const double v = vn[r];
      const double pv = r > c1 && tn != 0.0 ? __ldcg(pg + r) : 0.0;
      const double cv = r > c1 ? __ldcg(cn + r) : 0.0;
      vj[r] = v;
      if (r > c1) {
        pj[r] = pv;
        vn[r] = cv;
      }
    }
    tj = tn;
    __syncthreads();
  }
}

// Number of eigenvalues of T below x, without a division: the signs of the leading principal
// minors p_i = det(T_i - x I), p_0 = 1, p_1 = d_0 - x, p_i = (d_{i-1} - x) p_{i-1} - e_{i-2}^2 p_{i-2},
// change sign exactly as often (Sturm).  The quotient form q_i = p_i / p_{i-1} puts an FP64
// division on the chain of every step; here the chain is one FMA.  The pair (p_{i-1}, p_i) is
// rescaled by one exact power of two (exponent-field arithmetic) whenever p_i leaves
// [2^-300, 2^300], and a p_i that vanishes against p_{i-1} (ratio below 2^-1000, or zero) is
// replaced by -2^-1000 p_{i-1} (after bringing p_{i-1} near 1), the zero-pivot rule of the
// quotient form.  e2[i] = e_i^2; T is scaled beforehand so that its norm is near 1
// (tri_prep), which keeps every product of the recurrence far from overflow.
__device__ __forceinline__ int exp_field(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}
__device__ __forceinline__ double pow2(int s) { return __longlong_as_double((long long)(1023 + s) << 52); }

__device__ int64_t sturm_count_poly(const double* d, const double* e2, int64_t k, double x) {
  double pm2 = 1.0, pm1 = d[0] - x;
  if (exp_field(pm1) < 1023 - 1000) pm1 = -pow2(-1000);  // p_1 vanishes against p_0 = 1
  int64_t cnt = pm1 < 0.0;
#pragma unroll 4
  for (int64_t i = 1; i < k; ++i) {
    double p = fma(d[i] - x, pm1, -(e2[i - 1] * pm2));
    const int ep = exp_field(p);
    if (ep < 1023 - 300 || ep > 1023 + 300) {
      const int em = exp_field(pm1);
      if (ep == 0 || ep < em - 1000) {
        // vanishing minor (counts as a sign change): p_{i-1} to [1, 2), p_i = -2^-1000 p_{i-1}
        pm1 *= pow2(1023 - em);
        p = -pm1 * pow2(-1000);
      } else {
        int sh = 1023 - ep;  // p to [1, 2) and p_{i-1} by the same factor
        sh = sh > 1023 ? 1023 : (sh < -1022 ? -1022 : sh);
        const double f = pow2(sh);
        p *= f;
        pm1 *= f;
      }
    }
    cnt += (__double_as_longlong(p) ^ __double_as_longlong(pm1)) < 0;  // signs differ
    pm2 = pm1;
    pm1 = p;
  }
  return cnt;
}

// T scaled by an exact power of two 2^-E with max(|d_i|, |e_i|) in [1, 2) (nothing to scale for
// T = 0): ds, es and e2s = es^2, and the factor 2^E in *sc.  Counts and bisection run on the
// scaled matrix; its eigenvalues times 2^E are those of T exactly.  Then the Gershgorin
// interval of the scaled matrix and the pivot floor of the Sturm count, bnd = {lo, hi, pivmin,
// ||T||} (minima and maxima are exact, so the parallel reduction gives the serial loop's values).
__global__ void __launch_bounds__(256) tri_prep(const double* d, const double* e, int64_t k, double* ds, double* es,
                                                double* e2s, double* sc, double* bnd) {
  __shared__ unsigned long long sh[256];
  __shared__ double shl[8], shh[8], she[8];
  unsigned long long mb = 0;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(d[i]) & 0x7fffffffffffffffull;
    const unsigned long long b =
        i + 1 < k ? (unsigned long long)__double_as_longlong(e[i]) & 0x7fffffffffffffffull : 0ull;
    mb = a > mb ? a : mb;
    mb = b > mb ? b : mb;
  }
  sh[threadIdx.x] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long mx = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) mx = sh[i] > mx ? sh[i] : mx;
    int ex = (int)(mx >> 52) - 1023;  // max in [2^ex, 2^(ex + 1)) (normal numbers)
    if (mx == 0 || (mx >> 52) == 0 || (mx >> 52) == 0x7ff) ex = 0;
    sh[0] = (unsigned long long)(long long)ex;
  }
  __syncthreads();
  const int ex = (int)(long long)sh[0];
  // 2^-ex in two factors so that neither leaves the normal range
  const double f1 = pow2(-ex / 2), f2 = pow2(-ex - (-ex / 2));
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
    ds[i] = d[i] * f1 * f2;
    const double v = i + 1 < k ? e[i] * f1 * f2 : 0.0;
    es[i] = v;
    e2s[i] = v * v;
  }
  if (threadIdx.x == 0) *sc = pow2(ex / 2) * pow2(ex - ex / 2);
  __syncthreads();
  double lo = DBL_MAX, hi = -DBL_MAX, emax2 = 0.0;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
    const double el = i > 0 ? fabs(es[i - 1]) : 0.0, er = i + 1 < k ? fabs(es[i]) : 0.0;
    lo = fmin(lo, ds[i] - el - er);
    hi = fmax(hi, ds[i] + el + er);
    if (i + 1 < k) emax2 = fmax(emax2, es[i] * es[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    shl[threadIdx.x >> 5] = lo;
    shh[threadIdx.x >> 5] = hi;
    she[threadIdx.x >> 5] = emax2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      lo = fmin(lo, shl[i]);
      hi = fmax(hi, shh[i]);
      emax2 = fmax(emax2, she[i]);
    }
    const double pivmin = DBL_MIN * fmax(1.0, emax2);
    const double w = fmax(fabs(lo), fabs(hi));
    lo -= 4.0 * DBL_EPSILON * w + 2.0 * pivmin;
    hi += 4.0 * DBL_EPSILON * w + 2.0 * pivmin;
    bnd[0] = lo;
    bnd[1] = hi;
    bnd[2] = pivmin;
    bnd[3] = fmax(fabs(lo), fabs(hi));
  }
}

// The first multisection round is shared by all eigenvalues: NGP points of the Gershgorin
// interval [lo, hi] (x_t = lo + (hi - lo)(t + 1)/(NGP + 1)), one Sturm count per thread over the
// whole GPU, about 15 bits of every eigenvalue in the time of one count.
constexpr int NGP = 152 * 256;
__global__ void __launch_bounds__(256) tri_count_grid(const double* d, const double* e2, const double* bnd, int64_t k,
                                                      int* cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NGP) return;
  const double lo = bnd[0], hi = bnd[1];
  const double x = lo + (hi - lo) * (double)(t + 1) / (double)(NGP + 1);
  cnt[t] = (int)sturm_count_poly(d, e2, k, x);
}

// One CTA of MS_W warps per wanted eigenvalue (index idx in descending order = ascending index
// k-1-idx) of the scaled matrix (tri_prep).  It starts from the sub-interval the shared round
// (tri_count_grid) left; each further round evaluates 32 MS_W interior points of [lo, hi], one
// per thread, and keeps the sub-interval that holds the eigenvalue: a (32 MS_W + 1)-fold
// reduction per round.  The count is a chain of dependent FP64 operations, so two warps share
// each scheduler at little cost and a round takes about one count.
constexpr int MS_W = 8;
__global__ void __launch_bounds__(32 * MS_W) tri_multisect(const double* d, const double* e2, const double* sc,
                                                           const double* bnd, const int* cnt, int64_t k, int r_cap,
                                                           double* lam, double* tnorm) {
  __shared__ unsigned s_above[MS_W];
  __shared__ double s_x[32 * MS_W];
  __shared__ int s_first;
  const int idx = blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5;
  constexpr int np = 32 * MS_W;
  if (idx >= r_cap) return;
  double lo = bnd[0], hi = bnd[1];
  const double pivmin = bnd[2], tn = bnd[3];
  const double f = *sc;
  if (idx == 0 && t == 0) *tnorm = tn * f;
  const int64_t a = k - 1 - idx;  // ascending index
  {
    // the shared round: the first of its points above the eigenvalue (count > a)
    if (t == 0) s_first = NGP;
    __syncthreads();
    int first = NGP;  // independent loads, no early exit: the scan costs about one L2 round trip
    for (int u = t; u < NGP; u += blockDim.x)
      if (__ldg(cnt + u) > a && u < first) first = u;
    if (first < NGP) atomicMin(&s_first, first);
    __syncthreads();
    const int g = s_first;
    const double width = hi - lo;
    const double nlo = g == 0 ? lo : lo + width * (double)g / (double)(NGP + 1);
    const double nhi = g == NGP ? hi : lo + width * (double)(g + 1) / (double)(NGP + 1);
    lo = nlo;
    hi = nhi;
  }
  for (int round = 0; round < 64; ++round) {
    const double width = hi - lo;
    if (width <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + DBL_EPSILON * tn + 4.0 * pivmin) break;
    const double x = lo + width * (double)(t + 1) / (double)(np + 1);
    const int64_t c = sturm_count_poly(d, e2, k, x);
    // the eigenvalue lies below x iff count(x) > a
    const unsigned above = __ballot_sync(0xffffffffu, c > a);
    if ((t & 31) == 0) s_above[warp] = above;
    s_x[t] = x;
    __syncthreads();
    int first = np;  // first trial point above the eigenvalue
    for (int w = 0; w < MS_W; ++w)
      if (s_above[w]) {
        first = w * 32 + __ffs(s_above[w]) - 1;
        break;
      }
    const double nlo = first == 0 ? lo : s_x[first - 1];
    const double nhi = first == np ? hi : s_x[first];
    __syncthreads();
    if (nlo == lo && nhi == hi) break;
    lo = nlo;
    hi = nhi;
  }
  if (t == 0) lam[idx] = 0.5 * (lo + hi) * f;
}

__device__ __forceinline__ double start_value(int64_t i, int j) {
  // deterministic pseudo-random start vector in (-1, 1): a 64-bit integer hash of (i, j)
  unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull ^ ((unsigned long long)j << 32 | 0x5bd1e995u);
  h ^= h >> 31;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 29;
  return ((double)(h >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

// Inverse iteration, one warp per eigenvector, its working arrays in shared memory (k <= 4000;
// above, in the per-vector slice of `scratch`, 6 k doubles each): lane 0 factors
// T - lambda I = P L U (partial pivoting by rows) and runs the triangular sweeps, the warp forms
// the start vector, the reciprocals of U's diagonal (so that the backward sweep multiplies
// instead of dividing) and the norms.  Three iterations, then Z (element i of vector j at
// [i * r_cap + j]).
constexpr int64_t kInvitSmemK = 4000;
__global__ void __launch_bounds__(32) tri_invit(const double* d, const double* e, int64_t k, int r_cap,
                                                const double* lam, const double* tnorm, double* scratch, double* Z) {
  extern __shared__ double smv[];
  double* sm = k <= kInvitSmemK ? smv : scratch + (size_t)blockIdx.x * 6 * k;
  double* Dg = sm;           // U diagonal, then its reciprocals
  double* Du = sm + k;       // U first superdiagonal
  double* Du2 = sm + 2 * k;  // U second superdiagonal (from row swaps)
  double* Dl = sm + 3 * k;   // L multipliers
  double* z = sm + 4 * k;
  unsigned char* piv = reinterpret_cast<unsigned char*>(sm + 5 * k);
  const int j = blockIdx.x, lane = threadIdx.x;
  if (j >= r_cap) return;
  const double lj = lam[j];
  const double eps_piv = DBL_EPSILON * fmax(*tnorm, DBL_MIN);
  for (int64_t i = lane; i < k; i += 32) {
    Dg[i] = d[i] - lj;
    Du[i] = i + 1 < k ? e[i] : 0.0;
    Dl[i] = i + 1 < k ? e[i] : 0.0;
    Du2[i] = 0.0;
    z[i] = start_value(i, j);
  }
  __syncwarp();
  if (lane == 0) {
    for (int64_t i = 0; i + 1 < k; ++i) {
      const double di = Dg[i], li = Dl[i];
      if (fabs(di) >= fabs(li)) {
        piv[i] = 0;
        const double f = di != 0.0 ? li / di : 0.0;
        Dl[i] = f;
        Dg[i + 1] = Dg[i + 1] - f * Du[i];
      } else {
        piv[i] = 1;
        const double f = di / li;
        Dg[i] = li;
        Dl[i] = f;
        const double tmp = Du[i];
        const double dn = Dg[i + 1];
        Du[i] = dn;
        Dg[i + 1] = tmp - f * dn;
        if (i + 2 < k) {
          const double un = Du[i + 1];
          Du2[i] = un;
          Du[i + 1] = -f * un;
        }
      }
    }
  }
  __syncwarp();
  for (int64_t i = lane; i < k; i += 32) {
    double g = Dg[i];
    if (fabs(g) < eps_piv) g = g < 0.0 ? -eps_piv : eps_piv;
    const double rg = 1.0 / g;
    Dg[i] = rg;
    // the backward sweep's coefficients scaled by the reciprocal pivot, so that its dependent
    // chain is one FMA per row: s_i = z_i/U_ii - (U_i,i+1/U_ii) s_{i+1} - (U_i,i+2/U_ii) s_{i+2}
    Du[i] *= rg;
    Du2[i] *= rg;
  }
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    if (lane == 0) {
      // forward: L^{-1} P b
      double zi = z[0];
      for (int64_t i = 0; i + 1 < k; ++i) {
        const double f = Dl[i], zn = z[i + 1];
        if (piv[i]) {
          z[i] = zn;
          zi = zi - f * zn;
        } else {
          z[i] = zi;
          zi = zn - f * zi;
        }
      }
      z[k - 1] = zi;
      // backward: U^{-1}, by the reciprocal pivots (the term of s_{i+2} is off the chain)
      double z1 = 0.0, z2 = 0.0;  // z[i + 1], z[i + 2]
      for (int64_t i = k - 1; i >= 0; --i) {
        const double b = fma(-Du2[i], z2, z[i] * Dg[i]);
        const double s = fma(-Du[i], z1, b);
        z[i] = s;
        z2 = z1;
        z1 = s;
      }
    }
    __syncwarp();
    double mx = 0.0;
    for (int64_t i = lane; i < k; i += 32) mx = fmax(mx, fabs(z[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double inv_mx = 1.0 / mx;
    double nrm2 = 0.0;
    for (int64_t i = lane; i < k; i += 32) {
      const double v = z[i] * inv_mx;
      nrm2 = fma(v, v, nrm2);
      z[i] = v;
    }
    for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
    const double inv = 1.0 / sqrt(nrm2);
    __syncwarp();
    for (int64_t i = lane; i < k; i += 32) z[i] *= inv;
    __syncwarp();
  }
  for (int64_t i = lane; i < k; i += 32) Z[(size_t)i * r_cap + j] = z[i];
}

// Re-orthogonalisation of each vector against the earlier vectors of its group
// (|lambda_i - lambda_j| <= 1e-3 ||T||), twice, then normalisation, on a cluster of OC CTAs:
// CTA q owns rows [q k / OC, (q + 1) k / OC) of Z.  Classical Gram-Schmidt: the CTAs' partial
// dot products of their rows land in shared memory; after a cluster barrier every CTA adds the
// OC partials in rank order, so all apply the same coefficients to their own rows.  The
// partials alternate between two buffers, so a buffer is rewritten only after a later barrier
// that every reader of its previous contents has passed.  Vectors in order; the FP64 work is
// spread over OC SMs.
constexpr int OC = 8;
__global__ void __launch_bounds__(EB) tri_orth(int64_t k, int r_cap, const double* lam, const double* tnorm, double* Z) {
  extern __shared__ double orth_sm[];
  double* part0 = orth_sm;                 // two buffers of r_cap + 1 partials
  double* coef = orth_sm + 2 * (r_cap + 1);
  __shared__ double sh[kShSlots];
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned q = cl.block_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = k * q / OC, r1 = k * (q + 1) / OC;
  const double tol = 1e-3 * (*tnorm);
  int par = 0;
#define ZZ(i, j) Z[(size_t)(i) * r_cap + (j)]
  auto exchange = [&]() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  };
  for (int j = 1; j < r_cap; ++j) {
    int first = j;
    while (first > 0 && fabs(lam[first - 1] - lam[j]) <= tol) --first;
    if (first == j) continue;
    for (int pass = 0; pass < 2; ++pass) {
      double* pp = part0 + par * (r_cap + 1);
      for (int i = first + warp; i < j; i += EB / 32) {
        double s = 0.0;
        for (int64_t r = r0 + lane; r < r1; r += 32) s = fma(ZZ(r, i), ZZ(r, j), s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) pp[i] = s;
      }
      exchange();
      for (int i = first + threadIdx.x; i < j; i += blockDim.x) {
        double c = 0.0;
        for (unsigned o = 0; o < OC; ++o) c += cl.map_shared_rank(pp, o)[i];
        coef[i] = c;
      }
      __syncthreads();
      for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double z = ZZ(r, j);
        for (int i = first; i < j; ++i) z = fma(-coef[i], ZZ(r, i), z);
        ZZ(r, j) = z;
      }
      __syncthreads();
      par ^= 1;
    }
    double* pp = part0 + par * (r_cap + 1);
    double part = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) part = fma(ZZ(r, j), ZZ(r, j), part);
    const double nq = block_sum(part, sh);
    if (threadIdx.x == 0) pp[r_cap] = nq;
    exchange();
    double nrm2 = 0.0;
    for (unsigned o = 0; o < OC; ++o) nrm2 += cl.map_shared_rank(pp, o)[r_cap];
    const double inv = 1.0 / sqrt(nrm2);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) ZZ(r, j) *= inv;
    __syncthreads();
    par ^= 1;
  }
#undef ZZ
  exchange();  // no CTA leaves while a peer may still read its shared memory
}

// Back-transformation in blocks of NBW reflectors, in the compact WY form (Schreiber and Van
// Loan, SIAM J. Sci. Stat. Comput. 10 (1989)): H_{j0} H_{j0+1} ... H_{j0+nb-1} = I - V T V^T,
// V the block's reflectors (zero above their leading 1) and T upper triangular with
// T_ii = tau_i and T[0:l, l] = -tau_l T[0:l, 0:l] V[:, 0:l]^T v_l.  T is formed once per block
// (wy_gram, wy_tfactor); each eigenvector then takes z -= V (T (V^T z)) per block, NBW
// independent dot products instead of NBW dependent ones.
constexpr int NBW = 16;

// G[b][i][l] = v_{j0+i} . v_{j0+l} for i < l: block b = blockIdx.x, column l = blockIdx.y, one
// warp per product, over the rows where v_{j0+l} is nonzero (j0+l+1..k-1).
__global__ void __launch_bounds__(EB) wy_gram(const double* A, int64_t k, int64_t nrefl, double* G) {
  const int64_t j0 = (int64_t)blockIdx.x * NBW;
  const int l = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j0 + l >= nrefl) return;
  const double* vl = A + (j0 + l) * k;
  double* g = G + (size_t)blockIdx.x * NBW * NBW;
  for (int i = warp; i < l; i += EB / 32) {
    const double* vi = A + (j0 + i) * k;
    double s = 0.0;
    for (int64_t r = j0 + l + 1 + lane; r < k; r += 32) s = fma(vi[r], vl[r], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g[i * NBW + l] = s;
  }
}

// T of block b = blockIdx.x (one warp, lane i forms row i), written over G's block.
__global__ void __launch_bounds__(32) wy_tfactor(const double* tau, int64_t nrefl, double* G) {
  __shared__ double T[NBW][NBW];
  const int64_t j0 = (int64_t)blockIdx.x * NBW;
  const int nb = (int)(nrefl - j0 < NBW ? nrefl - j0 : NBW);
  const int i = threadIdx.x;
  double* g = G + (size_t)blockIdx.x * NBW * NBW;
  if (i < NBW)
    for (int c = 0; c < NBW; ++c) T[i][c] = 0.0;
  __syncwarp();
  for (int l = 0; l < nb; ++l) {
    const double tl = tau[j0 + l];
    double s = 0.0;
    if (i < l)
      for (int m = i; m < l; ++m) s = fma(T[i][m], g[m * NBW + l], s);
    __syncwarp();
    if (i < l) T[i][l] = -tl * s;
    if (i == l) T[i][l] = tl;
    __syncwarp();
  }
  if (i < NBW)
    for (int c = 0; c < NBW; ++c) g[i * NBW + c] = T[i][c];
}

// U[:, j] = H_0 H_1 ... H_{k-3} z_j (nrefl = k - 2 reflectors, the last block first), then the
// sign rule and T_r = U_r Lambda^{-1/2}.  One block per eigenvector; the vector lives in
// shared memory.
__global__ void __launch_bounds__(EB) hh_back(const double* A, int64_t k, int r_cap, int64_t nrefl,
                                              const double* Tw, const double* lam, const double* Z, double* U,
                                              double* Tr) {
  extern __shared__ double z[];
  __shared__ double y[NBW], yt[NBW];
  __shared__ int s_arg;
  const int j = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) z[i] = Z[(size_t)i * r_cap + j];
  __syncthreads();
  const int64_t nblk = nrefl > 0 ? (nrefl + NBW - 1) / NBW : 0;
  for (int64_t b = nblk - 1; b >= 0; --b) {
    const int64_t j0 = b * NBW;
    const int nb = (int)(nrefl - j0 < NBW ? nrefl - j0 : NBW);
    // y = V^T z
    for (int i = warp; i < nb; i += EB / 32) {
      const double* vi = A + (j0 + i) * k;
      double s = 0.0;
      for (int64_t r = j0 + i + 1 + lane; r < k; r += 32) s = fma(vi[r], z[r], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) y[i] = s;
    }
    __syncthreads();
    // yt = T y
    if (threadIdx.x < nb) {
      const double* T = Tw + (size_t)b * NBW * NBW;
      const int i = threadIdx.x;
      double s = 0.0;
      for (int m = i; m < nb; ++m) s = fma(T[i * NBW + m], y[m], s);
      yt[i] = s;
    }
    __syncthreads();
    // z -= V yt: row r meets the reflectors i with j0 + i + 1 <= r
    for (int64_t r = j0 + 1 + threadIdx.x; r < k; r += blockDim.x) {
      const int ilim = (int)(r - j0 < nb ? r - j0 : nb);
      double acc = z[r];
      for (int i = 0; i < ilim; ++i) acc = fma(-A[r + (j0 + i) * k], yt[i], acc);
      z[r] = acc;
    }
    __syncthreads();
  }
  // sign rule: the entry of largest magnitude is positive (lowest index on ties)
  if (threadIdx.x == 0) {
    double best = -1.0;
    int arg = 0;
    for (int64_t i = 0; i < k; ++i) {
      const double a = fabs(z[i]);
      if (a > best) {
        best = a;
        arg = (int)i;
      }
    }
    s_arg = arg;
  }
  __syncthreads();
  const double sgn = z[s_arg] < 0.0 ? -1.0 : 1.0;
  const double l = lam[j];
  const double sc = l > 0.0 ? 1.0 / sqrt(l) : 0.0;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
    const double u = sgn * z[i];
    U[i + (size_t)j * k] = u;
    Tr[i + (size_t)j * k] = u * sc;
  }
}

// One warp: trace(D) as lane sums (lane l adds D_ii for i = l mod 32 in order) and a butterfly.
__global__ void finalize_rank(const double* D, int64_t k, int64_t ldd, const double* lam, int r_cap, double tau,
                              int r_fixed, double* out_eig, int* r_dev, double* trace_dev) {
  double tr = 0.0;
  for (int64_t i = threadIdx.x; i < k; i += 32) tr += D[i + i * ldd];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (threadIdx.x != 0) return;
  int r = 0;
  if (r_fixed > 0) {
    r = r_fixed;
  } else {
    double cum = 0.0;
    for (int i = 0; i < r_cap; ++i) {
      cum += lam[i];
      if (cum / tr > tau) {
        r = i + 1;
        break;
      }
    }
  }
  for (int i = 0; i < r_cap; ++i) out_eig[i] = lam[i];
  if (r > 0 && !(lam[r - 1] > 0.0)) r = -r;  // lambda_r <= 0
  *r_dev = r;
  *trace_dev = tr;
}

struct ReduceWs {
  double *A, *d, *e, *tau, *p, *lam, *tnorm, *Z, *U, *iv, *trace, *ds, *es, *e2s, *sc, *bnd, *wy;
  int *r, *cnt;
  GridBar* bar;
  void* tn;
  size_t tn_bytes, used;
};

// One layout for the size query (base == nullptr) and the entry point.
ReduceWs carve_reduce(void* base, int64_t k, int r_cap) {
  Carver c(base);
  ReduceWs w;
  w.A = c.take<double>((size_t)k * k);
  w.d = c.take<double>(k);
  w.e = c.take<double>(k);
  w.tau = c.take<double>(k);
  w.p = c.take<double>(k);
  w.lam = c.take<double>(r_cap);
  w.tnorm = c.take<double>(1);
  w.trace = c.take<double>(1);
  w.r = c.take<int>(1);
  w.bar = c.take<GridBar>(1);
  w.Z = c.take<double>((size_t)k * r_cap);
  w.U = c.take<double>((size_t)k * r_cap);
  w.iv = c.take<double>(k > kInvitSmemK ? (size_t)6 * k * r_cap : 1);  // inverse iteration, large k
  w.ds = c.take<double>(k);  // the scaled tridiagonal of the bisection
  w.es = c.take<double>(k);
  w.e2s = c.take<double>(k);
  w.sc = c.take<double>(1);
  w.bnd = c.take<double>(4);
  w.cnt = c.take<int>(NGP);  // the counts of the shared multisection round
  const int64_t nblk = k > 2 ? (k - 2 + NBW - 1) / NBW : 1;
  w.wy = c.take<double>((size_t)nblk * NBW * NBW);  // the T factors of the back-transformation
  w.tn_bytes = tn_workspace(k, r_cap, k, 0);
  w.tn = c.take<char>(w.tn_bytes);
  w.used = c.used;
  return w;
}

// Householder tridiagonalisation of w.A: one cooperative launch (grid barrier per column)
// where 3 k doubles of shared memory fit, else three launches per column.
int g_reduce_coop = 1;

int tridiagonalise(const ReduceWs& w, int64_t k, cudaStream_t st) {
  size_t smem = (size_t)3 * k * sizeof(double);
  DOPINF_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(GridBar), st));
  int dev = 0, sms = 0, coop = 0;
  DOPINF_CUDA(cudaGetDevice(&dev));
  DOPINF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DOPINF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (g_reduce_coop && k >= 3 && coop && smem <= 200 * 1024) {
    // FP64 throughput per SM binds: about four trailing columns per CTA (one warp on each
    // of the SM's four schedulers), at most one CTA per SM (a cheap barrier)
    int64_t grid = (k - 1 + 3) / 4;
    if (grid > sms) grid = sms;
    if (grid < 1) grid = 1;
    // the CTA's columns in shared memory where they fit
    const int64_t ncl = (k + grid - 1) / grid;
    const size_t smem_res = (size_t)(3 + ncl) * k * sizeof(double);
    int resident = smem_res <= 200 * 1024 ? 1 : 0;
    if (resident) smem = smem_res;
    DOPINF_CUDA(cudaFuncSetAttribute(hh_tridiag_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DOPINF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hh_tridiag_coop, TB, smem));
    if (per_sm >= 1) {
      double* A = w.A;
      double *d = w.d, *e = w.e, *tau = w.tau, *p = w.p;
      GridBar* bar = w.bar;
      int64_t kk = k;
      unsigned stall = (test_stall() & kStallGridBarrier) ? 1u : 0u;
      void* args[] = {&A, &kk, &d, &e, &tau, &p, &bar, &resident, &stall};
      DOPINF_CUDA(cudaLaunchCooperativeKernel((const void*)hh_tridiag_coop, dim3((unsigned)grid), dim3(TB), args, smem, st));
      return launch_status();  // the barrier's error word is read with the results
    }
  }
  for (int64_t j = 0; j + 2 < k; ++j) {
    const int64_t m = k - j - 1;
    hh_gen<<<1, EB, 0, st>>>(w.A, k, j, w.d, w.e, w.tau);
    hh_symv<<<(unsigned)((m + 7) / 8), EB, 0, st>>>(w.A, k, j, w.tau, w.p);
    hh_rank2<<<(unsigned)((m + R2_COLS - 1) / R2_COLS), EB, 0, st>>>(w.A, k, j, w.tau, w.p);
  }
  hh_tail<<<1, 32, 0, st>>>(w.A, k, w.d, w.e, w.tau);
  return launch_status();
}

}  // namespace
}  // namespace dopinf

using namespace dopinf;

DOPINF_API int dopinf_tune_reduce_coop(int on) {
  const int prev = g_reduce_coop;
  if (on == 0 || on == 1) g_reduce_coop = on;
  return prev;
}

DOPINF_API size_t dopinf_reduce_workspace(int64_t k, int r_cap) {
  if (k < 1 || r_cap < 1) return 0;
  return carve_reduce(nullptr, k, r_cap).used;
}

namespace dopinf {
namespace {
// r <= 0 (rank or energy failure) and an expired grid barrier as flag bits (asynchronous path).
__global__ void reduce_flags(const int* r, const unsigned* bar_err, unsigned* flags) {
  unsigned b = 0;
  if (*r <= 0) b |= DOPINF_FLAG_RANK;
  if (*bar_err) b |= DOPINF_FLAG_TIMEOUT;
  if (b) atomicOr(flags, b);
}

// The re-orthogonalisation as one cluster of OC CTAs; its shared memory holds 3 (r_cap + 1)
// doubles (r_cap is at most k, and k is bounded by the back-transformation's shared memory).
int launch_orth(int64_t k, int r_cap, const double* lam, const double* tnorm, double* Z, cudaStream_t st) {
  const size_t smem = (size_t)3 * (r_cap + 1) * sizeof(double);
  if (smem > 48 * 1024)
    DOPINF_CUDA(cudaFuncSetAttribute(tri_orth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(OC, 1, 1);
  cfg.blockDim = dim3(EB, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = OC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DOPINF_CUDA(cudaLaunchKernelEx(&cfg, tri_orth, k, r_cap, lam, tnorm, Z));
  return DOPINF_OK;
}

// Everything but the read-back: r and trace(D) land in r_dev / trace_dev (device).
int reduce_launch(const double* D, int64_t k, int64_t ldd, double energy_target, int r_fixed, int r_cap,
                  int* r_dev, double* trace_dev, double* eigvals, double* Tr, double* Qhat, const ReduceWs& w,
                  cudaStream_t st) {
  DOPINF_CUDA(cudaMemcpy2DAsync(w.A, k * sizeof(double), D, ldd * sizeof(double), k * sizeof(double), k,
                                cudaMemcpyDeviceToDevice, st));
  DOPINF_TRY(tridiagonalise(w, k, st));
  // one eigenvalue (8 warps) and one eigenvector (a warp) per CTA: both are chains of dependent
  // FP64 operations, so they are spread over the SMs rather than packed into a few
  tri_prep<<<1, 256, 0, st>>>(w.d, w.e, k, w.ds, w.es, w.e2s, w.sc, w.bnd);
  tri_count_grid<<<(NGP + 255) / 256, 256, 0, st>>>(w.ds, w.e2s, w.bnd, k, w.cnt);
  tri_multisect<<<r_cap, 32 * MS_W, 0, st>>>(w.ds, w.e2s, w.sc, w.bnd, w.cnt, k, r_cap, w.lam, w.tnorm);
  DOPINF_TRY(launch_status());
  const size_t iv_smem = k <= kInvitSmemK ? (size_t)k * (5 * sizeof(double) + 1) : 0;
  if (iv_smem > 48 * 1024)
    DOPINF_CUDA(cudaFuncSetAttribute(tri_invit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)iv_smem));
  tri_invit<<<r_cap, 32, iv_smem, st>>>(w.d, w.e, k, r_cap, w.lam, w.tnorm, w.iv, w.Z);
  DOPINF_TRY(launch_orth(k, r_cap, w.lam, w.tnorm, w.Z, st));
  const int64_t nrefl = k > 2 ? k - 2 : 0;
  if (nrefl > 0) {
    const unsigned nblk = (unsigned)((nrefl + NBW - 1) / NBW);
    wy_gram<<<dim3(nblk, NBW), EB, 0, st>>>(w.A, k, nrefl, w.wy);
    wy_tfactor<<<nblk, 32, 0, st>>>(w.tau, nrefl, w.wy);
  }
  const size_t smem = (size_t)k * sizeof(double);
  if (smem > 48 * 1024) DOPINF_CUDA(cudaFuncSetAttribute(hh_back, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  hh_back<<<r_cap, EB, smem, st>>>(w.A, k, r_cap, nrefl, w.wy, w.lam, w.Z, w.U, Tr);
  DOPINF_TRY(launch_status());
  DOPINF_TRY(tn_product(Tr, k, D, ldd, DOPINF_F64, k, r_cap, k, 0, 0, Qhat, r_cap, w.tn, w.tn_bytes, st));
  finalize_rank<<<1, 32, 0, st>>>(D, k, ldd, w.lam, r_cap, energy_target, r_fixed, eigvals, r_dev, trace_dev);
  return launch_status();
}

int reduce_check(const double* D, int64_t k, int64_t ldd, double energy_target, int r_fixed, int r_cap,
                 const double* eigvals, const double* Tr, const double* Qhat, void* ws, size_t ws_bytes) {
  if (!D || k < 1 || ldd < k || r_cap < 1 || r_cap > k || r_fixed > r_cap || !eigvals || !Tr || !Qhat)
    return DOPINF_E_ARG;
  if (r_fixed <= 0 && !(energy_target >= 0.0 && energy_target < 1.0)) return DOPINF_E_ARG;
  if (!ws || ws_bytes < dopinf_reduce_workspace(k, r_cap) || misaligned(ws)) return DOPINF_E_ARG;
  if ((size_t)k * sizeof(double) > 200 * 1024) return DOPINF_E_UNSUPPORTED;  // back-transform keeps z in smem
  if ((size_t)3 * (r_cap + 1) * sizeof(double) > 200 * 1024) return DOPINF_E_UNSUPPORTED;  // orthogonalisation
  return DOPINF_OK;
}
}  // namespace
}  // namespace dopinf

DOPINF_API int dopinf_reduce_async(const double* D, int64_t k, int64_t ldd, double energy_target, int r_fixed,
                                   int r_cap, int* r_dev, double* trace_dev, double* eigvals, double* Tr,
                                   double* Qhat, unsigned* dev_flags, void* ws, size_t ws_bytes, void* stream) {
  if (!r_dev || !trace_dev || !dev_flags) return DOPINF_E_ARG;
  DOPINF_TRY(reduce_check(D, k, ldd, energy_target, r_fixed, r_cap, eigvals, Tr, Qhat, ws, ws_bytes));
  cudaStream_t st = as_stream(stream);
  ReduceWs w = carve_reduce(ws, k, r_cap);
  DOPINF_TRY(reduce_launch(D, k, ldd, energy_target, r_fixed, r_cap, r_dev, trace_dev, eigvals, Tr, Qhat, w, st));
  reduce_flags<<<1, 1, 0, st>>>(r_dev, &w.bar->err, dev_flags);
  return launch_status();
}

DOPINF_API int dopinf_reduce(const double* D, int64_t k, int64_t ldd, double energy_target, int r_fixed, int r_cap,
                             int* r_out, double* trace_out, double* eigvals, double* Tr, double* Qhat, void* ws,
                             size_t ws_bytes, void* stream) {
  if (!r_out || !trace_out) return DOPINF_E_ARG;
  DOPINF_TRY(reduce_check(D, k, ldd, energy_target, r_fixed, r_cap, eigvals, Tr, Qhat, ws, ws_bytes));
  cudaStream_t st = as_stream(stream);
  ReduceWs w = carve_reduce(ws, k, r_cap);
  DOPINF_TRY(reduce_launch(D, k, ldd, energy_target, r_fixed, r_cap, w.r, w.trace, eigvals, Tr, Qhat, w, st));
  int r_host = 0;
  double tr_host = 0.0;
  DOPINF_CUDA(cudaMemcpyAsync(&r_host, w.r, sizeof(int), cudaMemcpyDeviceToHost, st));
  DOPINF_CUDA(cudaMemcpyAsync(&tr_host, w.trace, sizeof(double), cudaMemcpyDeviceToHost, st));
  unsigned bar_err = 0;
  DOPINF_CUDA(cudaMemcpyAsync(&bar_err, &w.bar->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  DOPINF_CUDA(cudaStreamSynchronize(st));
  if (bar_err) {
    set_last_error("dopinf_reduce: grid barrier of the tridiagonalisation", cudaErrorTimeout);
    return DOPINF_E_TIMEOUT;
  }
  *trace_out = tr_host;
  if (r_host == 0) {
    *r_out = 0;
    return DOPINF_E_RANK;
  }
  if (r_host < 0) {
    *r_out = -r_host;
    return DOPINF_E_RANK;
  }
  *r_out = r_host;
  return DOPINF_OK;
}
