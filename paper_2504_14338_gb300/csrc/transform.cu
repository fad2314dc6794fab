// Step II of dOpInf (Section 3.3): per-row temporal centering and per-variable max-abs
// scaling of the snapshot matrix, as two streaming passes over Q (a third one for the
// standard-deviation scaling, the other strategy the section names).
//
//  pass 1 (stats):  per row i, the FP64 sum over t in time order, the min and the max.
//                   mean_i = sum / k.  Because rounding to nearest is monotone,
//                   max_t |fl(Q[i,t] - mean_i)| = max(|fl(max_i - mean_i)|, |fl(min_i - mean_i)|),
//                   so the per-variable scale is reduced from the row extremes with an
//                   order-independent atomic max on the (non-negative) FP64 bit patterns.
//  pass 2 (apply):  Q[i,t] = (Q[i,t] - mean_i) / scale_var(i), each operation IEEE-rounded.
//
// Q is column-major (snapshot t contiguous), so one thread per row walks its row with
// warp-coalesced loads.
#include "common.cuh"
#include <math.h>

namespace dopinf {
namespace {

struct VarTable {
  int n_vars;
  int64_t off[kMaxVars + 1];
};

__device__ __forceinline__ int var_of(const VarTable& vt, int64_t i) {
  int v = 0;
  while (v + 1 < vt.n_vars && i >= vt.off[v + 1]) ++v;
  return v;
}

// Order-preserving map of a double's bits to a signed integer (valid for non-NaN values),
// so that min/max of FP64 data run on the integer pipe instead of the narrow FP64 pipe.
__device__ __forceinline__ long long ord64(double x) {
  long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double unord64(long long o) {
  return __longlong_as_double(o ^ ((o >> 63) & 0x7fffffffffffffffLL));
}

__device__ __forceinline__ void warp_max_atomic(unsigned long long* dst, double a, bool valid, int v) {
  const unsigned full = 0xffffffffu;
  int v0 = __shfl_sync(full, v, 0);
  unsigned long long bits = valid ? (unsigned long long)__double_as_longlong(a) : 0ull;
  if (__all_sync(full, v == v0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long b2 = __shfl_xor_sync(full, bits, o);
      bits = b2 > bits ? b2 : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(dst + v0, bits);
  } else if (valid) {
    atomicMax(dst + v, bits);
  }
}

__global__ void __launch_bounds__(256) stats_f64(const double* __restrict__ Q, int64_t n, int64_t k,
                                                 int64_t ldq, VarTable vt, double* __restrict__ mean,
                                                 unsigned long long* __restrict__ vmax,
                                                 unsigned* __restrict__ flags, int center, int scale) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = i < n;
  int64_t ii = valid ? i : n - 1;
  const double* p = Q + ii;
  double s = 0.0;
  long long mn = LLONG_MAX, mx = LLONG_MIN;
  int64_t t = 0;
  for (; t + 8 <= k; t += 8) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = __ldcs(p + (t + u) * ldq);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s += x[u];
      long long o = ord64(x[u]);
      mn = o < mn ? o : mn;
      mx = o > mx ? o : mx;
    }
  }
  for (; t < k; ++t) {
    double x = __ldcs(p + t * ldq);
    s += x;
    long long o = ord64(x);
    mn = o < mn ? o : mn;
    mx = o > mx ? o : mx;
  }
  double m = s / (double)k;
  if (valid) {
    mean[i] = m;
    if (!isfinite(s)) atomicOr(flags, DOPINF_FLAG_NONFINITE);
  }
  if (scale) {
    double mc = center ? m : 0.0;
    double a = fmax(fabs(unord64(mx) - mc), fabs(unord64(mn) - mc));
    if (isnan(s)) a = __longlong_as_double(0x7ff8000000000000LL);
    warp_max_atomic(vmax, a, valid, var_of(vt, ii));
  }
}

__global__ void __launch_bounds__(256) stats_f32(const float* __restrict__ Q, int64_t n, int64_t k,
                                                 int64_t ldq, VarTable vt, double* __restrict__ mean,
                                                 unsigned long long* __restrict__ vmax,
                                                 unsigned* __restrict__ flags, int center, int scale) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = i < n;
  int64_t ii = valid ? i : n - 1;
  const float* p = Q + ii;
  double s = 0.0;
  float mn = INFINITY, mx = -INFINITY;
  int64_t t = 0;
  for (; t + 8 <= k; t += 8) {
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = __ldcs(p + (t + u) * ldq);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s += (double)x[u];
      mn = fminf(mn, x[u]);
      mx = fmaxf(mx, x[u]);
    }
  }
  for (; t < k; ++t) {
    float x = __ldcs(p + t * ldq);
    s += (double)x;
    mn = fminf(mn, x);
    mx = fmaxf(mx, x);
  }
  double m = s / (double)k;
  if (valid) {
    mean[i] = m;
    if (!isfinite(s)) atomicOr(flags, DOPINF_FLAG_NONFINITE);
  }
  if (scale) {
    double mc = center ? m : 0.0;
    float chi = (float)((double)mx - mc);
    float clo = (float)((double)mn - mc);
    double a = (double)fmaxf(fabsf(chi), fabsf(clo));
    if (isnan(s)) a = __longlong_as_double(0x7ff8000000000000LL);
    warp_max_atomic(vmax, a, valid, var_of(vt, ii));
  }
}

__global__ void finalize_scale(double* var_scale, int n_vars, int scale, unsigned* flags) {
  int v = threadIdx.x + blockIdx.x * blockDim.x;
  if (v >= n_vars) return;
  if (!scale) {
    var_scale[v] = 1.0;
    return;
  }
  double s = var_scale[v];  // holds the max bits written by the stats pass
  if (!isfinite(s)) {
    atomicOr(flags, DOPINF_FLAG_NONFINITE);
  } else if (s == 0.0) {
    atomicOr(flags, DOPINF_FLAG_ZERO_SCALE);
    s = 1.0;
  }
  var_scale[v] = s;
}

// c / s rounded to nearest from y = RN(1/s), by Markstein's correction (P. Markstein, "Computation
// of elementary functions on the IBM RISC System/6000 processor", IBM J. Res. Dev. 34(1), 1990):
// q0 = RN(c y) lies within one ulp of c / s, the remainder c - s q0 is exact as one FMA, and
// RN(q0 + rem y) is the correctly rounded quotient.  Three FP64 operations instead of a full
// division; operands near the ends of the exponent range (zero, subnormal, huge, non-finite)
// take the IEEE division, so the result equals c / s bit for bit everywhere.
__device__ __forceinline__ double div_by(double c, double s, double y, bool s_ok) {
  // |c| in [2^-900, 2^900), read from the exponent field: an integer test, where a
  // floating-point compare would take GB300's FP64 pipe (an issue slot per compare)
  const int ec = (int)(((unsigned long long)__double_as_longlong(c) >> 52) & 0x7ff);
  if (!s_ok || ec < 1023 - 900 || ec >= 1023 + 900) return __ddiv_rn(c, s);
  const double q0 = __dmul_rn(c, y);
  const double rem = __fma_rn(-q0, s, c);
  return __fma_rn(rem, y, q0);
}

// One thread per row and a chunk of columns; grid.y walks the columns.
template <typename T>
__global__ void __launch_bounds__(256) apply_kernel(T* __restrict__ Q, int64_t n, int64_t k, int64_t ldq,
                                                    VarTable vt, const double* __restrict__ mean,
                                                    const double* __restrict__ var_scale, int center,
                                                    int scale, int cols_per_block) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double m = center ? mean[i] : 0.0;
  double s = var_scale[var_of(vt, i)];
  const double y = __ddiv_rn(1.0, s);
  const bool s_ok = fabs(s) >= 0x1p-500 && fabs(s) <= 0x1p+500;
  int64_t t0 = (int64_t)blockIdx.y * cols_per_block;
  int64_t t1 = t0 + cols_per_block < k ? t0 + cols_per_block : k;
  T* p = Q + i;
  for (int64_t t = t0; t < t1; ++t) {
    T x = p[t * ldq];
    if constexpr (sizeof(T) == 8) {
      double c = center ? __dsub_rn((double)x, m) : (double)x;
      if (scale) c = div_by(c, s, y, s_ok);
      p[t * ldq] = (T)c;
    } else {
      float c = center ? (float)((double)x - m) : (float)x;
      if (scale) c = c / (float)s;
      p[t * ldq] = (T)c;
    }
  }
}

// Standard-deviation scaling (DOPINF_SCALE_STD): per row the sum over t, in time order, of the
// squared centred values (centred exactly as the apply pass centres them).
template <typename T>
__global__ void __launch_bounds__(256) rowsq_kernel(const T* __restrict__ Q, int64_t n, int64_t k, int64_t ldq,
                                                    const double* __restrict__ mean, int center,
                                                    double* __restrict__ rowsq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m = center ? mean[i] : 0.0;
  double s = 0.0;
  for (int64_t t = 0; t < k; ++t) {
    const T x = Q[i + t * ldq];
    double c;
    if constexpr (sizeof(T) == 8)
      c = center ? __dsub_rn(x, m) : x;
    else
      c = center ? (double)(float)((double)x - m) : (double)x;
    s = __dadd_rn(s, __dmul_rn(c, c));
  }
  rowsq[i] = s;
}

// One CTA per variable: the rows' sums in a fixed order (each thread a strided sequence, then a
// fixed tree), s_j = sqrt(total / (rows * k)), rounded to FP32 for FP32 data; a zero scale
// becomes 1 (flagged), a non-finite one is flagged.
__global__ void __launch_bounds__(256) var_std_kernel(const double* __restrict__ rowsq, VarTable vt, int64_t k,
                                                      int f32, double* __restrict__ var_scale,
                                                      unsigned* __restrict__ flags) {
  __shared__ double sh[256];
  const int v = blockIdx.x;
  const int64_t a = vt.off[v], b = vt.off[v + 1];
  double s = 0.0;
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) s += rowsq[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double cnt = (double)(b - a) * (double)k;
    double sd = cnt > 0.0 ? sqrt(sh[0] / cnt) : 0.0;
    if (f32) sd = (double)(float)sd;
    if (!isfinite(sd)) {
      atomicOr(flags, DOPINF_FLAG_NONFINITE);
    } else if (sd == 0.0) {
      atomicOr(flags, DOPINF_FLAG_ZERO_SCALE);
      sd = 1.0;
    }
    var_scale[v] = sd;
  }
}

}  // namespace

}  // namespace dopinf

using namespace dopinf;

DOPINF_API size_t dopinf_transform_workspace(int64_t n, int n_vars) {
  (void)n_vars;
  Carver c(nullptr);
  c.take<unsigned>(1);
  c.take<double>(n > 0 ? (size_t)n : 1);  // per-row sums of squares (standard-deviation scaling)
  return c.used;
}

DOPINF_API int dopinf_transform(void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int n_vars,
                                const int64_t* var_row_offsets, unsigned flags, double* row_mean,
                                double* var_scale, unsigned* dev_flags, void* ws, size_t ws_bytes,
                                void* stream) {
  if (dtype != DOPINF_F64 && dtype != DOPINF_F32) return DOPINF_E_ARG;
  if (n < 0 || k < 1 || ldq < (n > 1 ? n : 1) || n_vars < 1 || n_vars > kMaxVars) return DOPINF_E_ARG;
  if (!var_row_offsets || !row_mean || !var_scale || (n > 0 && !Q)) return DOPINF_E_ARG;
  if (flags & ~(DOPINF_CENTER | DOPINF_SCALE | DOPINF_SCALE_STD)) return DOPINF_E_ARG;
  if ((flags & DOPINF_SCALE) && (flags & DOPINF_SCALE_STD)) return DOPINF_E_ARG;
  const int std_scale = (flags & DOPINF_SCALE_STD) != 0;
  VarTable vt;
  vt.n_vars = n_vars;
  for (int v = 0; v <= n_vars; ++v) {
    vt.off[v] = var_row_offsets[v];
    if (v > 0 && vt.off[v] < vt.off[v - 1]) return DOPINF_E_ARG;
  }
  if (vt.off[0] != 0 || vt.off[n_vars] != n) return DOPINF_E_ARG;
  if (!dev_flags || std_scale) {
    if (!ws || ws_bytes < dopinf_transform_workspace(n, n_vars) || misaligned(ws)) return DOPINF_E_ARG;
  }
  cudaStream_t st = as_stream(stream);
  Carver cv(ws);
  unsigned* fl_ws = cv.take<unsigned>(1);
  double* rowsq = cv.take<double>(n > 0 ? (size_t)n : 1);
  unsigned* fl = dev_flags;
  if (!fl) {
    fl = fl_ws;
    DOPINF_CUDA(cudaMemsetAsync(fl, 0, sizeof(unsigned), st));
  }
  int center = (flags & DOPINF_CENTER) != 0, scale = (flags & DOPINF_SCALE) != 0;
  DOPINF_CUDA(cudaMemsetAsync(var_scale, 0, sizeof(double) * n_vars, st));
  if (n > 0) {
    unsigned blocks = (unsigned)((n + 255) / 256);
    auto* vmax = reinterpret_cast<unsigned long long*>(var_scale);
    if (dtype == DOPINF_F64)
      stats_f64<<<blocks, 256, 0, st>>>(static_cast<const double*>(Q), n, k, ldq, vt, row_mean, vmax, fl, center, scale);
    else
      stats_f32<<<blocks, 256, 0, st>>>(static_cast<const float*>(Q), n, k, ldq, vt, row_mean, vmax, fl, center, scale);
    DOPINF_TRY(launch_status());
  }
  finalize_scale<<<(n_vars + 63) / 64, 64, 0, st>>>(var_scale, n_vars, scale, fl);
  DOPINF_TRY(launch_status());
  if (std_scale) {
    if (n > 0) {
      const unsigned blocks = (unsigned)((n + 255) / 256);
      if (dtype == DOPINF_F64)
        rowsq_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(Q), n, k, ldq, row_mean, center, rowsq);
      else
        rowsq_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(Q), n, k, ldq, row_mean, center, rowsq);
      DOPINF_TRY(launch_status());
    }
    var_std_kernel<<<n_vars, 256, 0, st>>>(rowsq, vt, k, dtype == DOPINF_F32, var_scale, fl);
    DOPINF_TRY(launch_status());
    scale = 1;
  }
  if (n > 0 && (center || scale)) {
    int cols = 16;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)((k + cols - 1) / cols));
    if (dtype == DOPINF_F64)
      apply_kernel<double><<<grid, 256, 0, st>>>(static_cast<double*>(Q), n, k, ldq, vt, row_mean,
                                                  var_scale, center, scale, cols);
    else
      apply_kernel<float><<<grid, 256, 0, st>>>(static_cast<float*>(Q), n, k, ldq, vt, row_mean,
                                                 var_scale, center, scale, cols);
    DOPINF_TRY(launch_status());
  }
  return DOPINF_OK;
}
