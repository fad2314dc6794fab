// FP64 "TN" product C = A^T B over a long contraction dimension K (the rows of the
// snapshot matrix), used for the method-of-snapshots Gram D = Q^T Q (Section 3.4,
// eq. mos_partitioned) and for the OpInf normal equations Dhat^T Dhat, Dhat^T Y (Section 3.5,
// eq. OpInf_reg).
//
// Design: 64 x 64 output tiles, 256 threads with 4 x 4 FP64 accumulators each, K staged
// through shared memory 16 rows at a time.  K is split across CTAs (the partitioned sum
// D = sum_i Q_i^T Q_i of the paper, with row blocks as the partitions); every CTA writes its
// partial tile to the workspace and a second kernel adds the partials in split order, so the
// result does not depend on scheduling.  With sym = 1 only tiles on or above the diagonal are
// computed and mirrored.  On GB300 the FP64 pipe (about 1.1 TFLOP/s for the whole chip) and
// not HBM bounds this kernel: every staged element feeds 64 FMAs.
#include "common.cuh"

namespace dopinf {
namespace {

constexpr int TM = 64, TN = 64, BK = 16, NT = 256;
// Resident CTAs on GB300: 152 SMs x 3 (the register limit of this kernel).  The plan targets
// this count independently of the device queried, so results do not depend on the device.
constexpr int kSlots = 152 * 3;

struct TnPlan {
  int tiles_m, tiles_n, ntiles, splits, units, grid;
  int64_t rows_per_split;
};

// Units = (tile, row split) pairs; a persistent grid walks them.  The split count is chosen so
// that the units fill whole waves of the resident slots (every unit costs the same).
TnPlan make_plan(int64_t K, int64_t M, int64_t N, int sym) {
  TnPlan p;
  p.tiles_m = (int)((M + TM - 1) / TM);
  p.tiles_n = (int)((N + TN - 1) / TN);
  p.ntiles = sym ? p.tiles_n * (p.tiles_n + 1) / 2 : p.tiles_m * p.tiles_n;
  if (p.ntiles < 1) p.ntiles = 1;
  int64_t max_splits = (K + BK * 8 - 1) / (BK * 8);  // at least 128 rows per split
  if (max_splits < 1) max_splits = 1;
  int best = 1;
  double best_eff = -1.0;
  for (int sp = 1; sp <= 4 * kSlots && sp <= max_splits; ++sp) {
    const int64_t units = (int64_t)p.ntiles * sp;
    const int64_t waves = (units + kSlots - 1) / kSlots;
    const double eff = (double)units / (double)(waves * kSlots) - 0.0005 * sp;
    if (eff > best_eff) {
      best_eff = eff;
      best = sp;
    }
    if (units >= 8 * kSlots) break;
  }
  int64_t rps = (K + best - 1) / best;
  rps = (rps + BK - 1) / BK * BK;
  if (rps < BK) rps = BK;
  p.rows_per_split = rps;
  p.splits = (int)((K + rps - 1) / rps);
  if (p.splits < 1) p.splits = 1;
  p.units = p.ntiles * p.splits;
  p.grid = p.units < kSlots ? p.units : kSlots;
  return p;
}

__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int sym, int& bi, int& bj) {
  if (sym) {
    int t = tile, row = 0, len = tiles_n;
    while (t >= len) {
      t -= len;
      ++row;
      --len;
    }
    bi = row;
    bj = row + t;
  } else {
    bi = tile % tiles_m;
    bj = tile / tiles_m;
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) tn_partial(const T* __restrict__ A, int64_t lda,
                                                 const T* __restrict__ B, int64_t ldb, int64_t K,
                                                 int64_t M, int64_t N, int64_t rows_per_split,
                                                 int tiles_m, int tiles_n, int sym, int ntiles, int units,
                                                 double* __restrict__ part) {
  __shared__ double As[BK][TM + 1];
  __shared__ double Bs[BK][TN + 1];
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
  const int tile = u % ntiles, split = u / ntiles;
  int bi, bj;
  tile_coords(tile, tiles_m, tiles_n, sym, bi, bj);
  const int64_t m0 = (int64_t)bi * TM, n0 = (int64_t)bj * TN;
  const int64_t k0 = (int64_t)split * rows_per_split;
  const int64_t k1 = k0 + rows_per_split < K ? k0 + rows_per_split : K;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lr = tid & 15, lc = tid >> 4;  // loader: row within the chunk, column group
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t kk = k0; kk < k1; kk += BK) {
    const int64_t row = kk + lr;
    const bool rv = row < k1;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int c = lc + 16 * p;
      const int64_t gm = m0 + c, gn = n0 + c;
      As[lr][c] = (rv && gm < M) ? (double)A[row + gm * lda] : 0.0;
      Bs[lr][c] = (rv && gn < N) ? (double)B[row + gn * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < BK; ++r) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[r][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[r][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* out = part + (size_t)u * (TM * TN);  // u = split * ntiles + tile
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) out[(ty + 16 * j) * TM + tx + 16 * i] = acc[i][j];
  }
}

__global__ void __launch_bounds__(NT) tn_reduce(const double* __restrict__ part, int splits, int ntiles,
                                                int tiles_m, int tiles_n, int sym, int64_t M, int64_t N,
                                                int accumulate, double* __restrict__ C, int64_t ldc) {
  int bi, bj;
  tile_coords(blockIdx.x, tiles_m, tiles_n, sym, bi, bj);
  const int e = blockIdx.y * NT + threadIdx.x;  // element of the tile, column-major
  const int m = e % TM, nn = e / TM;
  const int64_t gm = (int64_t)bi * TM + m, gn = (int64_t)bj * TN + nn;
  if (gm >= M || gn >= N) return;
  double s = 0.0;
  for (int sp = 0; sp < splits; ++sp) s += part[((size_t)sp * ntiles + blockIdx.x) * (TM * TN) + e];
  if (accumulate) s += C[gm + gn * ldc];
  C[gm + gn * ldc] = s;
  if (sym && bi != bj) C[gn + gm * ldc] = s;
}

}  // namespace

size_t tn_workspace(int64_t K, int64_t M, int64_t N, int sym) {
  TnPlan p = make_plan(K, M, N, sym);
  Carver c(nullptr);
  c.take<double>((size_t)p.splits * p.ntiles * TM * TN);
  return c.used;
}

int tn_product(const void* A, int64_t lda, const void* B, int64_t ldb, int dtype, int64_t K, int64_t M,
               int64_t N, int sym, int accumulate, double* C, int64_t ldc, void* ws, size_t ws_bytes,
               cudaStream_t st) {
  if (M <= 0 || N <= 0) return DOPINF_OK;
  if (K < 0 || !C || ldc < M || (K > 0 && (!A || !B || lda < K || ldb < K))) return DOPINF_E_ARG;
  if (sym && (A != B || M != N || lda != ldb)) return DOPINF_E_ARG;
  TnPlan p = make_plan(K, M, N, sym);
  if (!ws || ws_bytes < tn_workspace(K, M, N, sym) || misaligned(ws)) return DOPINF_E_ARG;
  Carver cv(ws);
  double* part = cv.take<double>((size_t)p.splits * p.ntiles * TM * TN);
  if (dtype == DOPINF_F64)
    tn_partial<double><<<p.grid, NT, 0, st>>>(static_cast<const double*>(A), lda, static_cast<const double*>(B),
                                              ldb, K, M, N, p.rows_per_split, p.tiles_m, p.tiles_n, sym,
                                              p.ntiles, p.units, part);
  else if (dtype == DOPINF_F32)
    tn_partial<float><<<p.grid, NT, 0, st>>>(static_cast<const float*>(A), lda, static_cast<const float*>(B),
                                             ldb, K, M, N, p.rows_per_split, p.tiles_m, p.tiles_n, sym,
                                             p.ntiles, p.units, part);
  else
    return DOPINF_E_ARG;
  DOPINF_TRY(launch_status());
  tn_reduce<<<dim3(p.ntiles, TM * TN / NT), NT, 0, st>>>(part, p.splits, p.ntiles, p.tiles_m, p.tiles_n,
                                                         sym, M, N, accumulate, C, ldc);
  return launch_status();
}

}  // namespace dopinf

using namespace dopinf;

DOPINF_API size_t dopinf_gram_workspace(int64_t n, int64_t k, int dtype, int mode) {
  (void)dtype;
  if (n < 0 || k < 1) return 0;
  if (mode == DOPINF_GRAM_BF16X4) return gram_tc_workspace(n, k);
  if (mode == DOPINF_GRAM_OZAKI_FP64) return gram_ozaki_workspace(n, k);
  if (mode != DOPINF_GRAM_FP64) return 0;
  return tn_workspace(n, k, k, 1);
}

static int gram_impl(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int mode, int accumulate,
                     double* D, int64_t ldd, unsigned* dev_flags, void* ws, size_t ws_bytes, void* stream) {
  if (n < 0 || k < 1 || ldq < (n > 1 ? n : 1) || ldd < k || !D || (n > 0 && !Q)) return DOPINF_E_ARG;
  if (dtype != DOPINF_F64 && dtype != DOPINF_F32) return DOPINF_E_ARG;
  if (mode != DOPINF_GRAM_FP64 && mode != DOPINF_GRAM_BF16X4 && mode != DOPINF_GRAM_OZAKI_FP64)
    return DOPINF_E_UNSUPPORTED;
  if (n == 0) {
    if (accumulate) return DOPINF_OK;
    return cuda_status(cudaMemset2DAsync(D, ldd * sizeof(double), 0, k * sizeof(double), k,
                                         as_stream(stream)));
  }
  if (mode == DOPINF_GRAM_BF16X4)
    return gram_tc(Q, dtype, n, k, ldq, accumulate, D, ldd, dev_flags, ws, ws_bytes, as_stream(stream));
  if (mode == DOPINF_GRAM_OZAKI_FP64)
    return gram_ozaki(Q, dtype, n, k, ldq, accumulate, D, ldd, dev_flags, ws, ws_bytes, as_stream(stream));
  return tn_product(Q, ldq, Q, ldq, dtype, n, k, k, 1, accumulate, D, ldd, ws, ws_bytes, as_stream(stream));
}

DOPINF_API int dopinf_gram(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int mode,
                           int accumulate, double* D, int64_t ldd, void* ws, size_t ws_bytes,
                           void* stream) {
  return gram_impl(Q, dtype, n, k, ldq, mode, accumulate, D, ldd, nullptr, ws, ws_bytes, stream);
}

DOPINF_API int dopinf_gram_async(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int mode,
                                 int accumulate, double* D, int64_t ldd, unsigned* dev_flags, void* ws,
                                 size_t ws_bytes, void* stream) {
  if (!dev_flags) return DOPINF_E_ARG;
  return gram_impl(Q, dtype, n, k, ldq, mode, accumulate, D, ldd, dev_flags, ws, ws_bytes, stream);
}

// ------------------------------------------------------------------------------------------
// Allocation-free FP64 Gram: the same kernels with their split-K partials in a fixed
// file-scope device array instead of a caller workspace.  For callers that cannot allocate
// device memory: code running inside a memory pool or an allocator callback, plugins that
// must not touch the device allocator, and code that runs while a CUDA graph is being
// built by someone else.  The array (kNoAllocScratchBytes) lives on every GPU that loads
// this library until the process exits.
// ------------------------------------------------------------------------------------------
namespace dopinf {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB per device
constexpr int kNoAllocMaxUnits = (int)(kNoAllocScratchBytes / (TM * TN * sizeof(double)));
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

constexpr int kNoAllocMaxDevices = 128;
constexpr int kNoAllocMaxK = 2816;  // 44 x 44 tiles of 64: 990 upper tiles of 32 KB fit the array
static_assert((kNoAllocMaxK / TM) * (kNoAllocMaxK / TM + 1) / 2 <= kNoAllocMaxUnits, "k limit");

// Device address of g_noalloc_scratch per device ordinal, with the id of the context it was
// resolved in.  In host code the symbol name is a host-side stand-in, not a device address,
// so it is resolved with cudaGetSymbolAddress while the device is current, and again whenever
// the device's context has changed (after a cudaDeviceReset the array may sit elsewhere).
struct NoAllocAddr {
  void* addr;
  unsigned long long ctx_id;
};
NoAllocAddr g_noalloc_addr[kNoAllocMaxDevices];

// Id of the calling thread's current context (0 if none is current yet), through the driver
// entry points the runtime hands out, so that the library does not link libcuda itself.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();  // a missing entry point only disables the check
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

}  // namespace
}  // namespace dopinf

DOPINF_API size_t dopinf_gram_noalloc_scratch_bytes(void) { return dopinf::kNoAllocScratchBytes; }

DOPINF_API int dopinf_gram_fp64_noalloc(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int accumulate,
                                        double* D, int64_t ldd, void* stream) {
  using namespace dopinf;
  if (n < 1 || k < 1 || ldq < n || ldd < k || !D || !Q) return DOPINF_E_ARG;
  if (dtype != DOPINF_F64 && dtype != DOPINF_F32) return DOPINF_E_ARG;
  if (k > kNoAllocMaxK) return DOPINF_E_UNSUPPORTED;  // before any tile count is formed
  // plan: as the workspace path, with the row split reduced until the partials fit the array
  TnPlan p = make_plan(n, k, k, 1);
  if (p.ntiles > kNoAllocMaxUnits) return DOPINF_E_UNSUPPORTED;
  if (p.units > kNoAllocMaxUnits) {
    const int splits = kNoAllocMaxUnits / p.ntiles;
    int64_t rps = (n + splits - 1) / splits;
    rps = (rps + BK - 1) / BK * BK;
    p.rows_per_split = rps;
    p.splits = (int)((n + rps - 1) / rps);
    p.units = p.ntiles * p.splits;
    p.grid = p.units < kSlots ? p.units : kSlots;
  }
  int dev = 0;
  DOPINF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return DOPINF_E_UNSUPPORTED;
  // first call on this device, or a new context since the address was taken: resolve it
  NoAllocAddr& slot = g_noalloc_addr[dev];
  const unsigned long long ctx = current_ctx_id();
  if (!slot.addr || ctx == 0 || ctx != slot.ctx_id) {
    void* addr = nullptr;
    DOPINF_CUDA(cudaGetSymbolAddress(&addr, g_noalloc_scratch));
    slot.addr = addr;
    slot.ctx_id = ctx ? ctx : current_ctx_id();  // the lookup above made the context current
  }
  double* part = static_cast<double*>(slot.addr);
  cudaStream_t st = as_stream(stream);
  if (dtype == DOPINF_F64)
    tn_partial<double><<<p.grid, NT, 0, st>>>(static_cast<const double*>(Q), ldq, static_cast<const double*>(Q), ldq,
                                              n, k, k, p.rows_per_split, p.tiles_m, p.tiles_n, 1, p.ntiles, p.units,
                                              part);
  else
    tn_partial<float><<<p.grid, NT, 0, st>>>(static_cast<const float*>(Q), ldq, static_cast<const float*>(Q), ldq, n,
                                             k, k, p.rows_per_split, p.tiles_m, p.tiles_n, 1, p.ntiles, p.units,
                                             part);
  DOPINF_TRY(launch_status());
  tn_reduce<<<dim3(p.ntiles, TM * TN / NT), NT, 0, st>>>(part, p.splits, p.ntiles, p.tiles_m, p.tiles_n, 1, k, k,
                                                         accumulate, D, ldd);
  return launch_status();
}
