// Split-precision method-of-snapshots Gram D = Q^T Q (Section 3.4, eq. mos_partitioned) on
// the tcgen05 tensor cores.
//
// Each value is split into two BF16 slices, x = h + l + e with h = bf16(x) and
// l = bf16(x - h) (x - h is exact in the source precision), |e| <= 2^-17 |x|.  Then
// Q^T Q ~= H^T H + H^T L + L^T H + L^T L: four BF16 products per 128 x 128 output tile.  The
// terms left out (those with e) change sign from row to row and grow like sqrt(n) against
// the n-fold sum.
//
// Accumulation.  The tensor core's FP32 accumulation rounds toward zero by about half an ulp
// per MMA (measured on GB300: the diagonal of a long sum drifts low in proportion to the number
// of MMAs).  So the MMA accumulator is restarted for every drain chunk (default: two stages of
// 64 rows), the small slice products of a stage are issued before the large ones, and each
// chunk sum is added to an FP32 (hi, lo) pair with Knuth's TwoSum, which carries the running
// sum to about 2^-44.  A final kernel adds the units of a tile in a fixed order and mirrors the
// upper triangle, so D is exactly symmetric and reproducible run to run.
//
// The large product gets columns of its own.  The accumulator is 256 columns wide: one MMA with
// the B operand [H_b; L_b] (the two slice tiles lie next to each other in shared memory) gives
//     D_left = H_a^T H_b,  D_right = H_a^T L_b,
// and two 128-column MMAs add L_a^T H_b and L_a^T L_b to D_right; the drain adds the halves.
// Nothing small is ever added to the large H^T H sum, so the chunks can span two stages (the
// per-chunk hand-off and drain cost as much as the MMAs at one stage) with the accuracy of
// one-stage chunks, and 12 MMA instructions per stage instead of 16 (with 128-column MMAs only,
// the issue loop, not the tensor pipe, set the pace).
//
// Kernel structure (one persistent CTA per SM, 576 threads):
//   warp 0    TMA producer: H and L tiles of the a-block and of the b-block (128 snapshots x
//             64 rows each, one contiguous 16 KB block of the tiled slice planes, 128-byte
//             swizzle) into a 3-stage shared ring;
//   warp 1    TMEM allocator and single-thread MMA issuer: tcgen05.mma M = 128, N = 256,
//             K = 16 into one of two 256-column TMEM accumulators;
//   warps 2-17 drain (four per TMEM lane quadrant, 32 columns each): tcgen05.ld of both halves
//             of the finished accumulator, their sum added by
//             TwoSum into (hi, lo) kept in registers for the whole work unit (tile, row range);
//             at its end hi + lo is written in FP64.
// Work units are ordered split-major, so the CTAs running together read the same rows and
// the slices come from HBM about once.  Every mbarrier wait is bounded in time; on expiry the
// kernel records an error, lets its copies and MMAs finish (again with bounded waits), frees
// TMEM and returns.
#include "common.cuh"
#include "sm100.cuh"
#include <cuda_bf16.h>

namespace dopinf {
namespace {

using namespace sm100;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int STAGES = 3;
constexpr uint32_t TILE = BM * BK * 2;         // 16 KB: one slice of one block
constexpr uint32_t STAGE_BYTES = 4 * TILE;     // Ah, Al, Bh, Bl
constexpr size_t SMEM_BYTES = STAGES * (size_t)STAGE_BYTES + 1024;
constexpr int NDRAIN = 16;
constexpr int NTHREADS = 64 + 32 * NDRAIN;
constexpr uint32_t TMEM_COLS = 512;
constexpr int NACC = 2;        // TMEM accumulators of 256 columns (left: H_b, right: L_b products)
constexpr int ACC_COLS = 2 * BN;
int64_t g_chunk_rows = 128;  // rows summed by one MMA accumulator before the TwoSum drain (tunable)
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kSmTarget = 152;  // the work split targets GB300's SM count, independent of the device queried

struct TcShape {
  int64_t n, nrb;  // nrb: 64-row blocks of the tiled slice planes
  int k, tn, ntiles, splits, units;
  int64_t rows_per_split, chunk_rows;
  int stall;  // test of the error path: the MMA issuer never releases a stage, so waits expire
};

// upper-triangle tiles (ta <= tb) of a tn x tn tile grid, row-major
__host__ __device__ inline void tile_of(int t, int tn, int& ta, int& tb) {
  ta = 0;
  while (t >= tn - ta) {
    t -= tn - ta;
    ++ta;
  }
  tb = ta + t;
}
__host__ __device__ inline int tile_index(int ta, int tb, int tn) { return ta * tn - ta * (ta - 1) / 2 + (tb - ta); }

__device__ __forceinline__ float two_sum_hi(float hi, float a, float& err) {
  const float s = __fadd_rn(hi, a);
  const float z = __fsub_rn(s, hi);
  err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(a, z));
  return s;
}

// 18 warps put 5 on two of the schedulers: 96 registers keep them inside one scheduler's file
__global__ void __maxnreg__(96)
    gram_bf16x4_kernel(const __grid_constant__ CUtensorMap mapH, const __grid_constant__ CUtensorMap mapL, TcShape sh,
                       double* __restrict__ part, unsigned* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[NACC], acce_bar[NACC], drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], NDRAIN);
    }
    mbar_init(&drain_bar, 1);
    abort_sh = 0;
    fence_mbar_init();
    tma_prefetch_desc(&mapH);
    tma_prefetch_desc(&mapL);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_sh, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  auto fail = [&](unsigned code) {
    atomicOr(err, code);
    abort_sh = 1;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------- TMA producer
      int stage = 0;
      int64_t it = 0;
      for (int u = blockIdx.x; u < sh.units && !abort_sh; u += gridDim.x) {
        int ta, tb;
        tile_of(u % sh.ntiles, sh.tn, ta, tb);
        const int64_t k0 = (int64_t)(u / sh.ntiles) * sh.rows_per_split;
        const int64_t k1 = k0 + sh.rows_per_split < sh.n ? k0 + sh.rows_per_split : sh.n;
        for (int64_t row = k0; row < k1 && !abort_sh; row += BK) {
          if (it >= STAGES && !mbar_wait(&empty_bar[stage], (uint32_t)((it / STAGES) - 1) & 1u, kWaitNs)) {
            fail(1u);
            break;
          }
          uint8_t* base = smem + (size_t)stage * STAGE_BYTES;
          mbar_arrive_expect_tx(&full_bar[stage], STAGE_BYTES);
          const int za = (int)(ta * sh.nrb + row / BK), zb = (int)(tb * sh.nrb + row / BK);
          tma_load_3d(base, &mapH, &full_bar[stage], 0, 0, za);
          tma_load_3d(base + TILE, &mapL, &full_bar[stage], 0, 0, za);
          tma_load_3d(base + 2 * TILE, &mapH, &full_bar[stage], 0, 0, zb);
          tma_load_3d(base + 3 * TILE, &mapL, &full_bar[stage], 0, 0, zb);
          stage = (stage + 1) % STAGES;
          ++it;
        }
      }
      // let the last copies land before the CTA can exit (bounded)
      for (int64_t j = it - STAGES > 0 ? it - STAGES : 0; j < it; ++j)
        mbar_wait(&full_bar[j % STAGES], (uint32_t)(j / STAGES) & 1u, kWaitNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA issuer
      const uint32_t idesc = idesc_bf16_f32(BM, ACC_COLS), idesc_half = idesc_bf16_f32(BM, BN);
      int stage = 0;
      int64_t it = 0, chunk = 0;
      bool issued = false;
      for (int u = blockIdx.x; u < sh.units && !abort_sh; u += gridDim.x) {
        const int64_t k0 = (int64_t)(u / sh.ntiles) * sh.rows_per_split;
        const int64_t k1 = k0 + sh.rows_per_split < sh.n ? k0 + sh.rows_per_split : sh.n;
        for (int64_t c0 = k0; c0 < k1 && !abort_sh; c0 += sh.chunk_rows) {
          const int buf = (int)(chunk % NACC);
          if (chunk >= NACC && !mbar_wait(&acce_bar[buf], (uint32_t)((chunk / NACC) - 1) & 1u, kWaitNs)) {
            fail(2u);
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tmem + (uint32_t)(buf * ACC_COLS);
          const int64_t c1 = c0 + sh.chunk_rows < k1 ? c0 + sh.chunk_rows : k1;
          bool first = true;
          for (int64_t row = c0; row < c1; row += BK) {
            if (!mbar_wait(&full_bar[stage], (uint32_t)(it / STAGES) & 1u, kWaitNs)) {
              fail(4u);
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + (size_t)stage * STAGE_BYTES);
            const uint32_t ah = sa, al = sa + TILE, bh = sa + 2 * TILE;  // L_b at bh + TILE
            // H_a^T [H_b; L_b] -> [H^T H | H^T L] first (it starts the chunk's accumulator), then
            // L_a^T H_b and L_a^T L_b into the right half only: the H^T H columns never receive a
            // small addend, so their truncation is that of the H^T H products alone
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t o = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzled row
              mma_bf16(dacc, sdesc_k_sw128(ah + o), sdesc_k_sw128(bh + o), idesc, first && kk == 0 ? 0u : 1u);
            }
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t o = kk * 32;
              mma_bf16(dacc + BN, sdesc_k_sw128(al + o), sdesc_k_sw128(bh + o), idesc_half, 1u);
              mma_bf16(dacc + BN, sdesc_k_sw128(al + o), sdesc_k_sw128(bh + TILE + o), idesc_half, 1u);
            }
            issued = true;
            first = false;
            if (!sh.stall) mma_commit(&empty_bar[stage]);
            stage = (stage + 1) % STAGES;
            ++it;
          }
          if (abort_sh) break;
          mma_commit(&accf_bar[buf]);
          ++chunk;
        }
      }
      if (issued) {  // every MMA of this thread complete before TMEM is released
        mma_commit(&drain_bar);
        mbar_wait(&drain_bar, 0u, kWaitNs);
      }
    }
  } else {
    // --------------------------------------------------------------- drain (warps 2-17)
    const int q = warp & 3;                  // TMEM lane quadrant this warp may access
    const int c0w = ((warp - 2) >> 2) * 32;  // this warp's 32 output columns
    const int row = q * 32 + lane;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    int64_t chunk = 0;
    for (int u = blockIdx.x; u < sh.units && !abort_sh; u += gridDim.x) {
      const int64_t k0 = (int64_t)(u / sh.ntiles) * sh.rows_per_split;
      const int64_t k1 = k0 + sh.rows_per_split < sh.n ? k0 + sh.rows_per_split : sh.n;
      float hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        hi[j] = 0.f;
        lo[j] = 0.f;
      }
      bool ok = true;
      for (int64_t c0 = k0; c0 < k1; c0 += sh.chunk_rows) {
        const int buf = (int)(chunk % NACC);
        ok = mbar_wait(&accf_bar[buf], (uint32_t)(chunk / NACC) & 1u, kWaitNs);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (lane == 0) fail(8u);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + lane_off + (uint32_t)(buf * ACC_COLS) + (uint32_t)c0w;
        // four columns at a time: left half (H_b products) + right half (L_b products)
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          uint32_t a[4], b[4];
          tmem_ld_32x32b_x4(acc + (uint32_t)(g * 4), a);
          tmem_ld_32x32b_x4(acc + (uint32_t)(BN + g * 4), b);
          tmem_wait_ld();
          if (g == 7) {  // the accumulator is free once every column is loaded
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce_bar[buf]);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float e;
            const float v = __fadd_rn(__uint_as_float(a[j]), __uint_as_float(b[j]));
            hi[g * 4 + j] = two_sum_hi(hi[g * 4 + j], v, e);
            lo[g * 4 + j] = __fadd_rn(lo[g * 4 + j], e);
          }
        }
        ++chunk;
      }
      if (!ok) break;
      // unit finished: hi + lo of this warp's columns, in FP64, to the unit's partial tile
      double* P = part + (size_t)u * BM * BN;
#pragma unroll
      for (int j = 0; j < 32; ++j) P[(size_t)(c0w + j) * BM + row] = (double)hi[j] + (double)lo[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// D[a, b] = D[b, a] = sum over the row splits (in order) of the unit partials, a <= b.
__global__ void gram_tc_reduce(const double* __restrict__ part, TcShape sh, int accumulate, double* __restrict__ D,
                               int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t kk = sh.k;
  if (e >= kk * kk) return;
  const int a = (int)(e % kk), b = (int)(e / kk);
  if (a > b) return;
  const int ta = a / BM, tb = b / BN;
  const int t = tile_index(ta, tb, sh.tn);
  const size_t off = (size_t)(b - tb * BN) * BM + (a - ta * BM);
  double s = 0.0;
  for (int sp = 0; sp < sh.splits; ++sp) s += part[((size_t)sp * sh.ntiles + t) * BM * BN + off];
  if (accumulate) s += D[a + (int64_t)b * ldd];
  D[a + (int64_t)b * ldd] = s;
  D[b + (int64_t)a * ldd] = s;
}

// h = bf16(x), l = bf16(x - h) in the tiled slice layout: the plane is a sequence of
// 64-row x 128-column blocks, block (column block cb, row block rb) at index cb * nrb + rb,
// each 16 KB contiguous with its 128 columns one after the other (64 rows = 128 bytes each).
// One TMA box is then one contiguous read.  Rows >= n and columns >= k are written as zeros.
template <typename T>
__global__ void split_bf16(const T* __restrict__ Q, int64_t n, int64_t k, int64_t ldq, __nv_bfloat16* __restrict__ H,
                           __nv_bfloat16* __restrict__ L, int64_t nrb, int64_t ncb, unsigned* __restrict__ err) {
  const int64_t rows = nrb * BK, cols = ncb * BM;
  const int64_t total = rows * cols;
  bool bad = false;  // NaN or Inf met: reported through the error word, D is then not valid
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, t = e / rows;
    __nv_bfloat16 h = __float2bfloat16_rn(0.0f), l = h;
    if (i < n && t < k) {
      const T x = Q[i + t * ldq];
      bad = bad || !isfinite(x);
      if constexpr (sizeof(T) == 8) {
        h = __double2bfloat16(x);
        l = __double2bfloat16(x - (double)__bfloat162float(h));
      } else {
        h = __float2bfloat16_rn(x);
        l = __float2bfloat16_rn(x - __bfloat162float(h));
      }
    }
    const int64_t off = ((t / BM) * nrb + i / BK) * (BM * BK) + (t % BM) * BK + (i % BK);
    H[off] = h;
    L[off] = l;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrNonfinite);
}

TcShape make_shape(int64_t n, int64_t k) {
  const int sms = kSmTarget;
  TcShape s;
  s.n = n;
  s.nrb = (n + BK - 1) / BK;
  s.k = (int)k;
  s.tn = (int)((k + BM - 1) / BM);
  s.ntiles = s.tn * (s.tn + 1) / 2;
  // choose the row split so that the units fill whole waves of SMs as evenly as possible
  const int64_t max_split = (n + 4 * BK - 1) / (4 * BK) > 0 ? (n + 4 * BK - 1) / (4 * BK) : 1;
  int best = 1;
  double best_eff = -1.0;
  for (int sp = 1; sp <= 256 && sp <= max_split; ++sp) {
    const int64_t units = (int64_t)s.ntiles * sp;
    const int64_t waves = (units + sms - 1) / sms;
    const double eff = (double)units / (double)(waves * sms) - 0.0005 * sp;  // prefer fewer splits on ties
    if (eff > best_eff) {
      best_eff = eff;
      best = sp;
    }
    if (units >= 16 * sms) break;
  }
  int64_t rps = (n + best - 1) / best;
  rps = (rps + BK - 1) / BK * BK;
  s.rows_per_split = rps;
  s.splits = (int)((n + rps - 1) / rps);
  if (s.splits < 1) s.splits = 1;
  s.units = s.ntiles * s.splits;
  s.chunk_rows = rps < g_chunk_rows ? rps : g_chunk_rows;
  s.stall = 0;
  return s;
}

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3-D map over a tiled BF16 plane: (64 rows, 128 columns, blocks), box = one block, 128-byte
// swizzle.  The box lands in shared memory as 128 rows (columns of Q) of 128 bytes.
bool make_map(CUtensorMap* map, void* base, int64_t nblocks) {
  EncodeTiledFn f = encode_fn();
  if (!f) return false;
  cuuint64_t dims[3] = {(cuuint64_t)BK, (cuuint64_t)BM, (cuuint64_t)nblocks};
  cuuint64_t strides[2] = {(cuuint64_t)(BK * 2), (cuuint64_t)(BK * BM * 2)};
  cuuint32_t box[3] = {BK, BM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return f(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcWs {
  __nv_bfloat16 *H, *L;
  double* part;
  unsigned* err;
  int64_t nrb, ncb;
  size_t used;
};

TcWs carve_tc(void* base, int64_t n, int64_t k) {
  const TcShape s = make_shape(n, k);
  Carver c(base);
  TcWs w;
  w.nrb = (n + BK - 1) / BK;
  w.ncb = (k + BM - 1) / BM;
  w.H = c.take<__nv_bfloat16>((size_t)w.nrb * w.ncb * BK * BM);
  w.L = c.take<__nv_bfloat16>((size_t)w.nrb * w.ncb * BK * BM);
  w.part = c.take<double>((size_t)s.units * BM * BN);
  w.err = c.take<unsigned>(1);
  w.used = c.used;
  return w;
}

}  // namespace

size_t gram_tc_workspace(int64_t n, int64_t k) { return carve_tc(nullptr, n, k).used; }

int64_t gram_tc_set_chunk_rows(int64_t rows) {
  const int64_t prev = g_chunk_rows;
  if (rows > 0) g_chunk_rows = (rows + BK - 1) / BK * BK;
  return prev;
}

int gram_tc(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int accumulate, double* D, int64_t ldd,
            unsigned* dev_flags, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (n > ((int64_t)1 << 31) - BK || k > 65535) return DOPINF_E_UNSUPPORTED;
  if (((n + BK - 1) / BK) * ((k + BM - 1) / BM) > (int64_t)INT32_MAX) return DOPINF_E_UNSUPPORTED;
  if (!ws || ws_bytes < gram_tc_workspace(n, k) || misaligned(ws)) return DOPINF_E_ARG;
  TcWs w = carve_tc(ws, n, k);
  TcShape sh = make_shape(n, k);
  sh.stall = (test_stall() & kStallTensorGram) ? 1 : 0;
  DOPINF_CUDA(cudaMemsetAsync(w.err, 0, sizeof(unsigned), st));
  const int64_t total = w.nrb * BK * w.ncb * BM;
  const unsigned sblocks = (unsigned)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
  if (dtype == DOPINF_F64)
    split_bf16<double><<<sblocks, 256, 0, st>>>(static_cast<const double*>(Q), n, k, ldq, w.H, w.L, w.nrb, w.ncb, w.err);
  else
    split_bf16<float><<<sblocks, 256, 0, st>>>(static_cast<const float*>(Q), n, k, ldq, w.H, w.L, w.nrb, w.ncb, w.err);
  DOPINF_TRY(launch_status());
  CUtensorMap mh, ml;
  if (!make_map(&mh, w.H, w.nrb * w.ncb) || !make_map(&ml, w.L, w.nrb * w.ncb)) return DOPINF_E_CUDA;
  DOPINF_CUDA(cudaFuncSetAttribute(gram_bf16x4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
  {
    int per_sm = 0;  // the kernel needs one resident CTA per SM (registers, shared memory)
    DOPINF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram_bf16x4_kernel, NTHREADS, SMEM_BYTES));
    if (per_sm < 1) {
      set_last_error("gram_bf16x4_kernel does not fit on an SM", cudaErrorLaunchOutOfResources);
      return DOPINF_E_CUDA;
    }
  }
  const int grid = sh.units < num_sms() ? sh.units : num_sms();
  gram_bf16x4_kernel<<<grid, NTHREADS, SMEM_BYTES, st>>>(mh, ml, sh, w.part, w.err);
  DOPINF_TRY(launch_status());
  const int64_t kk = k * k;
  gram_tc_reduce<<<(unsigned)((kk + 255) / 256), 256, 0, st>>>(w.part, sh, accumulate, D, ldd);
  DOPINF_TRY(launch_status());
  return finish_timeout(w.err, dev_flags, st);
}

}  // namespace dopinf
