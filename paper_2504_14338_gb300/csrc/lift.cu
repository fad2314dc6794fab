// Step V of dOpInf (Section 3.6): the reduced solution mapped back to the original
// coordinates at chosen rows (probe locations, or every row), in two FP64 products and the
// inverse of Step II's transform:
//   basis_rows   V[j, a] = sum_s Q[row_j, s] T_r[s, a]         (rows of the POD basis,
//                eq. MoS_POD_basis: V_r = Q T_r, from the transformed snapshots)
//   lift_rows    X[j, t] = scale(row_j) * sum_a V[j, a] Qtilde[a, t] + mean(row_j)
// The paper's ranks each lift their own rows with no communication; here the rows are the
// grid's blocks.  Both products are FP64 FMA chains in a fixed order.
#include "common.cuh"

namespace dopinf {
namespace {

constexpr int BR = 128;  // rows per CTA of basis_rows
constexpr int AC = 8;    // POD modes per thread
constexpr int TS = 64;   // snapshots per staged tile of T_r

// One thread per row j and a chunk of AC modes (blockIdx.y); T_r staged in shared memory one
// tile of TS snapshots at a time.  rows == nullptr: row j is row j.  A row index outside
// [0, n) gives a NaN row (nothing is read for it).
template <typename T>
__global__ void __launch_bounds__(BR) basis_rows(const T* __restrict__ Q, int64_t n, int64_t k, int64_t ldq,
                                                 const double* __restrict__ Tr, int64_t ldt, int r,
                                                 const int64_t* __restrict__ rows, int64_t n_rows,
                                                 double* __restrict__ V, int64_t ldv) {
  __shared__ double ts[TS][AC];
  const int64_t j = (int64_t)blockIdx.x * BR + threadIdx.x;
  const int a0 = blockIdx.y * AC;
  int64_t row = j;
  if (rows && j < n_rows) row = rows[j];
  const bool ok = j < n_rows && row >= 0 && row < n;
  double acc[AC];
#pragma unroll
  for (int c = 0; c < AC; ++c) acc[c] = 0.0;
  for (int64_t s0 = 0; s0 < k; s0 += TS) {
    __syncthreads();
    for (int e = threadIdx.x; e < TS * AC; e += BR) {
      const int s = e % TS, c = e / TS;
      ts[s][c] = (s0 + s < k && a0 + c < r) ? Tr[(s0 + s) + (int64_t)(a0 + c) * ldt] : 0.0;
    }
    __syncthreads();
    if (ok) {
      const int smax = k - s0 < TS ? (int)(k - s0) : TS;
      for (int s = 0; s < smax; ++s) {
        const double q = (double)Q[row + (s0 + s) * ldq];
#pragma unroll
        for (int c = 0; c < AC; ++c) acc[c] = fma(q, ts[s][c], acc[c]);
      }
    }
  }
  if (j < n_rows)
#pragma unroll
    for (int c = 0; c < AC; ++c)
      if (a0 + c < r) V[j + (int64_t)(a0 + c) * ldv] = ok ? acc[c] : NAN;
}

struct InvTransform {
  int n_vars;
  int64_t off[kMaxVars + 1];  // variable row offsets
};

// X[j, t] = scale * (sum_a V[j, a] Qtilde[a, t]) + mean, each operation rounded separately.
// threadIdx.x walks rows (coalesced V and X), threadIdx.y times.
__global__ void __launch_bounds__(256) lift_rows(const double* __restrict__ V, int64_t ldv, int r,
                                                 const double* __restrict__ Qt, int64_t ldqt, int64_t n_t,
                                                 const int64_t* __restrict__ rows, int64_t n_rows,
                                                 const double* __restrict__ row_mean,
                                                 const double* __restrict__ var_scale, const InvTransform inv,
                                                 double* __restrict__ X, int64_t ldx) {
  const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
  if (j >= n_rows) return;
  const int64_t row = rows ? rows[j] : j;
  double scale = 1.0;
  if (var_scale) {
    int v = 0;
    while (v + 1 < inv.n_vars && row >= inv.off[v + 1]) ++v;
    scale = var_scale[v];
  }
  const double mean = (row_mean && row >= 0 && row < inv.off[inv.n_vars]) ? row_mean[row] : 0.0;
  for (int64_t t = (int64_t)blockIdx.y * 8 + threadIdx.y; t < n_t; t += (int64_t)gridDim.y * 8) {
    double y = 0.0;
    for (int a = 0; a < r; ++a) y = fma(V[j + (int64_t)a * ldv], Qt[a + t * ldqt], y);
    if (var_scale) y = __dmul_rn(scale, y);
    if (row_mean) y = __dadd_rn(y, mean);
    X[j + t * ldx] = y;
  }
}

}  // namespace
}  // namespace dopinf

using namespace dopinf;

DOPINF_API size_t dopinf_lift_workspace(int64_t n_rows, int r) {
  if (n_rows < 1 || r < 1) return 0;
  return align_up((size_t)n_rows * r * sizeof(double));
}

DOPINF_API int dopinf_lift(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, const double* Tr,
                           int64_t ldt, int r, const double* Qtilde, int64_t ldqt, int64_t n_t, const int64_t* rows,
                           int64_t n_rows, const double* row_mean, const double* var_scale, int n_vars,
                           const int64_t* var_row_offsets, double* X, int64_t ldx, void* ws, size_t ws_bytes,
                           void* stream) {
  if (!Q || !Tr || !Qtilde || !X || n < 1 || k < 1 || ldq < n || r < 1 || ldt < k || ldqt < r || n_t < 1 ||
      n_rows < 1 || ldx < n_rows)
    return DOPINF_E_ARG;
  if (!rows && n_rows > n) return DOPINF_E_ARG;
  if (dtype != DOPINF_F64 && dtype != DOPINF_F32) return DOPINF_E_ARG;
  if (r > 65535 * AC) return DOPINF_E_UNSUPPORTED;
  InvTransform inv = {};
  inv.n_vars = 1;
  inv.off[1] = n;
  if (var_scale || row_mean) {
    if (var_scale && (!var_row_offsets || n_vars < 1 || n_vars > kMaxVars)) return DOPINF_E_ARG;
    if (var_row_offsets && n_vars >= 1 && n_vars <= kMaxVars) {
      if (var_row_offsets[0] != 0 || var_row_offsets[n_vars] != n) return DOPINF_E_ARG;
      for (int v = 0; v < n_vars; ++v)
        if (var_row_offsets[v + 1] < var_row_offsets[v]) return DOPINF_E_ARG;
      inv.n_vars = n_vars;
      for (int v = 0; v <= n_vars; ++v) inv.off[v] = var_row_offsets[v];
    }
  }
  if (!ws || ws_bytes < dopinf_lift_workspace(n_rows, r) || misaligned(ws)) return DOPINF_E_ARG;
  double* V = static_cast<double*>(ws);
  cudaStream_t st = as_stream(stream);
  if ((n_rows + BR - 1) / BR > (int64_t)0x7fffffff || (n_rows + 31) / 32 > (int64_t)0x7fffffff)
    return DOPINF_E_UNSUPPORTED;
  const dim3 g1((unsigned)((n_rows + BR - 1) / BR), (unsigned)((r + AC - 1) / AC));
  if (dtype == DOPINF_F64)
    basis_rows<double><<<g1, BR, 0, st>>>(static_cast<const double*>(Q), n, k, ldq, Tr, ldt, r, rows, n_rows, V,
                                          n_rows);
  else
    basis_rows<float><<<g1, BR, 0, st>>>(static_cast<const float*>(Q), n, k, ldq, Tr, ldt, r, rows, n_rows, V,
                                         n_rows);
  DOPINF_TRY(launch_status());
  const int64_t tb = (n_t + 7) / 8;
  const dim3 g2((unsigned)((n_rows + 31) / 32), (unsigned)(tb < 65535 ? tb : 65535));
  lift_rows<<<g2, dim3(32, 8), 0, st>>>(V, n_rows, r, Qtilde, ldqt, n_t, rows, n_rows, row_mean, var_scale, inv, X,
                                        ldx);
  return launch_status();
}
