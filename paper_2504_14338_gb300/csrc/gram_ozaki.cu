// FP64-accurate method-of-snapshots Gram D = Q^T Q (Section 3.4, eq. mos_partitioned) on the
// BF16 tensor cores, by an error-free split into integer digits (the splitting idea of Ozaki,
// Ogita, Oishi and Rump, "Error-free transformations of matrix multiplication", 2012).
//
// GB300 has about 1.1 TFLOP/s of FP64 but ~2 PFLOP/s of BF16 tensor throughput.  Each column a
// of Q is scaled by 2^-s_a (s_a = 1 + the exponent bounding its max-abs, so |x| < 2^(s_a - 1))
// and rounded to a 55-bit fixed-point integer V = round(x 2^(56 - s_a)), which is cut into
// S = 7 balanced base-256 digits (integer arithmetic on the IEEE encoding; the FP64 pipe is not
// used):
//     x = 2^s_a * sum_i d_i 2^(-8 i) + e,  |e| <= 2^(s_a - 57),
// with |d_i| <= 128, integers exact in BF16.  Then
//     D_ab = 2^(s_a + s_b) * sum_w 2^(-8 w) S_w,   S_w = sum_{i + j = w} D_i^T D_j,
// keeping the weights w = 2..8 (28 digit products; the dropped ones weigh below 2^-55 of
// 2^(s_a + s_b), as does the rounding of V).
// Each S_w is formed in a pass of its own: a product of two digits is at most 2^14, so a
// chunk of L rows of the m_w products of a weight is at most L m_w 2^14 < 2^24 when
// L = 64 * floor(16 / m_w): every partial sum in the FP32 tensor accumulator is an integer
// below 2^24 and therefore exact, whatever the accumulator's rounding.  Chunk sums go into an
// FP32 (hi, lo) pair in tensor memory by TwoSum, exact while |lo| < 2^24 (at most 2^19 rows per
// work unit); at the end of a unit hi + lo is weighted by 2^(-8 w) and stored in FP64 as the
// unit's partial tile of that weight (the drain threads keep hi of their 64 columns in
// registers, lo in tensor memory).  A final kernel sums weights and units of a tile in a fixed order, applies
// 2^(s_a + s_b) and mirrors the upper triangle.
//
// Kernel structure per pass (one persistent CTA per SM, 320 threads), as the BF16x4 kernel:
// TMA producer warp (one 16 KB contiguous block per tile from the tiled digit planes), single-
// thread tcgen05.mma issuer (M = N = 128, K = 16), 8 drain warps; TMEM: three 128-column
// accumulators and lo.  Every wait is bounded in time.
#include "common.cuh"
#include "sm100.cuh"
#include <cuda_bf16.h>

namespace dopinf {
namespace {

using namespace sm100;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int NDIG = 7;            // digits per value
constexpr int DIG_BITS = 8;
constexpr int W_MIN = 2, W_MAX = NDIG + 1;
constexpr int STAGES = 6;
constexpr uint32_t TILE = BM * BK * 2;     // 16 KB
constexpr uint32_t STAGE_BYTES = 2 * TILE;  // one digit block of the a-block and one of the b-block
constexpr size_t SMEM_BYTES = STAGES * (size_t)STAGE_BYTES + 1024;
constexpr int NDRAIN = 8;
constexpr int NTHREADS = 64 + 32 * NDRAIN;
constexpr uint32_t TMEM_COLS = 512;
constexpr int NACC = 3;  // TMEM accumulators of 128 columns; the fourth block holds lo
constexpr uint32_t COL_LO = 384;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kSmTarget = 152;
constexpr int64_t kMaxUnitRows = (int64_t)1 << 19;  // keeps |lo| < 2^24 (exact TwoSum carry)

struct OzShape {
  int64_t n, nrb, ncb;
  int k, tn, ntiles, splits, units;
  int64_t rows_per_split;
  int stall;  // test of the error path: the MMA issuer of the first pass never releases a stage
};

__host__ __device__ inline void tile_of(int t, int tn, int& ta, int& tb) {
  ta = 0;
  while (t >= tn - ta) {
    t -= tn - ta;
    ++ta;
  }
  tb = ta + t;
}
__host__ __device__ inline int tile_index(int ta, int tb, int tn) { return ta * tn - ta * (ta - 1) / 2 + (tb - ta); }

// digit pairs (i, j), i + j = w, 1 <= i, j <= NDIG
__host__ __device__ inline int pair_lo(int w) { return w - NDIG > 1 ? w - NDIG : 1; }
__host__ __device__ inline int pair_hi(int w) { return w - 1 < NDIG ? w - 1 : NDIG; }
__host__ __device__ inline int pairs_of(int w) { return pair_hi(w) - pair_lo(w) + 1; }
// rows per exact chunk of weight w: L m_w 2^14 < 2^24
__host__ __device__ inline int64_t chunk_rows_of(int w) { return (int64_t)BK * (16 / pairs_of(w)); }

__device__ __forceinline__ float two_sum_hi(float hi, float a, float& err) {
  const float s = __fadd_rn(hi, a);
  const float z = __fsub_rn(s, hi);
  err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(a, z));
  return s;
}

// Sign and magnitude bits of a value: x = sign * m * 2^(e - bias) with an integer significand m
// (implicit bit included), read from the IEEE encoding with integer operations only.
__device__ __forceinline__ void decode(double x, bool& neg, unsigned long long& m, int& e2) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  neg = (b >> 63) != 0;
  const int ef = (int)((b >> 52) & 0x7ff);
  m = b & 0xfffffffffffffull;
  if (ef) m |= 1ull << 52;
  e2 = (ef ? ef : 1) - 1075;  // x = m * 2^e2
}
__device__ __forceinline__ void decode(float x, bool& neg, unsigned long long& m, int& e2) {
  const unsigned b = __float_as_uint(x);
  neg = (b >> 31) != 0;
  const int ef = (int)((b >> 23) & 0xff);
  m = b & 0x7fffffu;
  if (ef) m |= 1u << 23;
  e2 = (ef ? ef : 1) - 150;
}

// max |Q[:, a]| per column, as s_a = 1 + the exponent e with max < 2^e (0 for an all-zero column).
// Magnitudes compare as integers of their encodings.
template <typename T>
__global__ void __launch_bounds__(256) colmax_kernel(const T* __restrict__ Q, int64_t n, int64_t ldq, int* __restrict__ sexp,
                                                     unsigned* __restrict__ err) {
  __shared__ unsigned long long sh[256];
  const int64_t a = blockIdx.x;
  const T* q = Q + a * ldq;
  auto mag = [](T x) -> unsigned long long {
    if constexpr (sizeof(T) == 8)
      return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    else
      return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
  };
  unsigned long long mb = 0, mb1 = 0, mb2 = 0, mb3 = 0;
  const int64_t step = blockDim.x;
  int64_t i = threadIdx.x;
  for (; i + 3 * step < n; i += 4 * step) {  // four independent loads in flight per thread
    const unsigned long long b0 = mag(q[i]), b1 = mag(q[i + step]), b2 = mag(q[i + 2 * step]), b3 = mag(q[i + 3 * step]);
    mb = b0 > mb ? b0 : mb;
    mb1 = b1 > mb1 ? b1 : mb1;
    mb2 = b2 > mb2 ? b2 : mb2;
    mb3 = b3 > mb3 ? b3 : mb3;
  }
  for (; i < n; i += step) {
    const unsigned long long b = mag(q[i]);
    mb = b > mb ? b : mb;
  }
  mb = mb1 > mb ? mb1 : mb;
  mb = mb2 > mb ? mb2 : mb;
  mb = mb3 > mb ? mb3 : mb;
  sh[threadIdx.x] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long mx = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) mx = sh[i] > mx ? sh[i] : mx;
    int e = 0;
    // NaN or Inf (an all-ones exponent field): reported through the error word, and the column
    // is digitised as if it were zero (D is then not valid)
    const unsigned long long inf_bits = sizeof(T) == 8 ? 0x7ff0000000000000ull : 0x7f800000ull;
    if (mx >= inf_bits) {
      atomicOr(err, kErrNonfinite);
      mx = 0;
    }
    if (mx) {
      bool neg;
      unsigned long long m;
      int e2;
      if constexpr (sizeof(T) == 8)
        decode(__longlong_as_double((long long)mx), neg, m, e2);
      else
        decode(__uint_as_float((unsigned)mx), neg, m, e2);
      e = e2 + 64 - __clzll((long long)m) + 1;  // m 2^e2 < 2^(e - 1)
    }
    sexp[a] = e;
  }
}

// V = round(x 2^(56 - s)) as a signed integer (|V| <= 2^55 for |x| < 2^(s - 1), error <= 1/2).
template <typename T>
__device__ __forceinline__ long long fixed56(T x, int s) {
  bool neg;
  unsigned long long m;
  int e2;
  decode(x, neg, m, e2);
  const int sh = e2 + 56 - s;  // V = m 2^sh
  unsigned long long u;
  if (sh >= 0)
    u = m << sh;  // |x| < 2^(s - 1) keeps this below 2^55
  else if (sh > -64)
    u = (m + (1ull << (-sh - 1))) >> (-sh);  // round half up in magnitude
  else
    u = 0;
  return neg ? -(long long)u : (long long)u;
}

// Digits into the tiled planes (plane p at p * nrb * ncb * 8192, block (cb, rb) inside it), by
// integer arithmetic: V = round(x 2^(56 - s_a)) (error <= 2^(s_a - 57) in x), then balanced
// base-256 digits from the low end, d_7 .. d_2 in [-128, 127], and the rest d_1 with
// |d_1| <= 128 (|V| <= 2^55), so that V = sum_i d_i 2^(8 (7 - i)).  A thread takes 4 consecutive
// rows of one column and writes 8 bytes per plane; blockIdx.y walks the (padded) columns.
constexpr int DIG_ROWS = 4;
template <typename T>
__global__ void __launch_bounds__(256) digits_kernel(const T* __restrict__ Q, int64_t n, int64_t k, int64_t ldq,
                                                     const int* __restrict__ sexp, __nv_bfloat16* __restrict__ planes,
                                                     int64_t nrb, int64_t ncb) {
  const int64_t rows = nrb * BK, cols = ncb * BM;
  const size_t plane = (size_t)nrb * ncb * BM * BK;
  for (int64_t t = blockIdx.y; t < cols; t += gridDim.y) {
    const T* q = Q + t * ldq;
    const int s = t < k ? sexp[t] : 0;
    const size_t cbase = (size_t)(t / BM) * nrb * (BM * BK) + (size_t)(t % BM) * BK;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * DIG_ROWS; i0 < rows;
         i0 += (int64_t)gridDim.x * blockDim.x * DIG_ROWS) {
      long long V[DIG_ROWS];
#pragma unroll
      for (int u = 0; u < DIG_ROWS; ++u) V[u] = (t < k && i0 + u < n) ? fixed56(q[i0 + u], s) : 0;
      // i0 is a multiple of 4 and BK of 64: the 4 rows sit in one block, 8-byte aligned
      __nv_bfloat16* dst = planes + cbase + (size_t)(i0 / BK) * (BM * BK) + (i0 % BK);
#pragma unroll
      for (int p = NDIG - 1; p >= 0; --p) {
        __nv_bfloat16 h[DIG_ROWS];
#pragma unroll
        for (int u = 0; u < DIG_ROWS; ++u) {
          long long d = V[u];
          if (p > 0) {
            d = ((V[u] + 128) & 255) - 128;
            V[u] = (V[u] - d) >> DIG_BITS;
          }
          // |d| <= 128: through a 32-bit integer (a 64-bit integer conversion runs on the FP64 pipe)
          h[u] = __float2bfloat16_rn((float)(int)d);
        }
        uint2 pk;
        pk.x = (unsigned)__bfloat16_as_ushort(h[0]) | ((unsigned)__bfloat16_as_ushort(h[1]) << 16);
        pk.y = (unsigned)__bfloat16_as_ushort(h[2]) | ((unsigned)__bfloat16_as_ushort(h[3]) << 16);
        *reinterpret_cast<uint2*>(dst + p * plane) = pk;
      }
    }
  }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_pass_kernel(const __grid_constant__ CUtensorMap map, OzShape sh, int w, double* __restrict__ part,
                      unsigned* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[NACC], acce_bar[NACC], drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int plo = pair_lo(w), phi = pair_hi(w);
  const int64_t chunk_rows = chunk_rows_of(w);
  const int64_t plane_blocks = sh.nrb * sh.ncb;
  __shared__ int skip_sh;
  // a bounded wait of an earlier pass expired: D is not valid, the later passes stop at once
  if (threadIdx.x == 0) skip_sh = (w > W_MIN && (*reinterpret_cast<volatile unsigned*>(err) & ~kErrNonfinite)) ? 1 : 0;
  __syncthreads();
  if (skip_sh) return;

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
    tma_prefetch_desc(&map);
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
          const int64_t rb = row / BK;
          for (int i = plo; i <= phi && !abort_sh; ++i) {
            const int j = w - i;
            if (it >= STAGES && !mbar_wait(&empty_bar[stage], (uint32_t)((it / STAGES) - 1) & 1u, kWaitNs)) {
              fail(1u);
              break;
            }
            uint8_t* base = smem + (size_t)stage * STAGE_BYTES;
            mbar_arrive_expect_tx(&full_bar[stage], STAGE_BYTES);
            const int za = (int)((i - 1) * plane_blocks + ta * sh.nrb + rb);
            const int zb = (int)((j - 1) * plane_blocks + tb * sh.nrb + rb);
            tma_load_3d(base, &map, &full_bar[stage], 0, 0, za);
            tma_load_3d(base + TILE, &map, &full_bar[stage], 0, 0, zb);
            stage = (stage + 1) % STAGES;
            ++it;
          }
        }
      }
      for (int64_t jj = it - STAGES > 0 ? it - STAGES : 0; jj < it; ++jj)
        mbar_wait(&full_bar[jj % STAGES], (uint32_t)(jj / STAGES) & 1u, kWaitNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA issuer
      const uint32_t idesc = idesc_bf16_f32(BM, BN);
      int stage = 0;
      int64_t it = 0, chunk = 0;
      bool issued = false;
      for (int u = blockIdx.x; u < sh.units && !abort_sh; u += gridDim.x) {
        const int64_t k0 = (int64_t)(u / sh.ntiles) * sh.rows_per_split;
        const int64_t k1 = k0 + sh.rows_per_split < sh.n ? k0 + sh.rows_per_split : sh.n;
        for (int64_t c0 = k0; c0 < k1 && !abort_sh; c0 += chunk_rows) {
          const int buf = (int)(chunk % NACC);
          if (chunk >= NACC && !mbar_wait(&acce_bar[buf], (uint32_t)((chunk / NACC) - 1) & 1u, kWaitNs)) {
            fail(2u);
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tmem + (uint32_t)(buf * BN);
          const int64_t c1 = c0 + chunk_rows < k1 ? c0 + chunk_rows : k1;
          bool first = true;
          for (int64_t row = c0; row < c1 && !abort_sh; row += BK) {
            for (int i = plo; i <= phi; ++i) {
              if (!mbar_wait(&full_bar[stage], (uint32_t)(it / STAGES) & 1u, kWaitNs)) {
                fail(4u);
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + (size_t)stage * STAGE_BYTES);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t o = kk * 32;
                mma_bf16(dacc, sdesc_k_sw128(sa + o), sdesc_k_sw128(sa + TILE + o), idesc, first && kk == 0 ? 0u : 1u);
              }
              issued = true;
              first = false;
              if (!(sh.stall && w == W_MIN)) mma_commit(&empty_bar[stage]);
              stage = (stage + 1) % STAGES;
              ++it;
            }
          }
          if (abort_sh) break;
          mma_commit(&accf_bar[buf]);
          ++chunk;
        }
      }
      if (issued) {
        mma_commit(&drain_bar);
        mbar_wait(&drain_bar, 0u, kWaitNs);
      }
    }
  } else {
    // --------------------------------------------------------------- drain (warps 2-9)
    const int q = warp & 3;
    const int c0w = ((warp - 2) >> 2) * 64;
    const int row = q * 32 + lane;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const double weight = ldexp(1.0, -DIG_BITS * w);
    int64_t chunk = 0;
    for (int u = blockIdx.x; u < sh.units && !abort_sh; u += gridDim.x) {
      const int64_t k0 = (int64_t)(u / sh.ntiles) * sh.rows_per_split;
      const int64_t k1 = k0 + sh.rows_per_split < sh.n ? k0 + sh.rows_per_split : sh.n;
      float hi[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) hi[j] = 0.f;
      bool ok = true;
      for (int64_t c0 = k0; c0 < k1; c0 += chunk_rows) {
        const int buf = (int)(chunk % NACC);
        ok = mbar_wait(&accf_bar[buf], (uint32_t)(chunk / NACC) & 1u, kWaitNs);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (lane == 0) fail(8u);
          break;
        }
        tc_fence_after();
        const bool first = c0 == k0;
        // a 16-column quarter at a time: hi in registers, lo in tensor memory
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const uint32_t col = (uint32_t)(c0w + g * 16);
          uint32_t a[16], lo[16];
          tmem_ld_32x32b_x16(tmem + lane_off + (uint32_t)(buf * BN) + col, a);
          if (!first) tmem_ld_32x32b_x16(tmem + lane_off + COL_LO + col, lo);
          tmem_wait_ld();
          if (g == 3) {  // the accumulator is free once all quarters are loaded
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce_bar[buf]);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float e;
            hi[g * 16 + j] = two_sum_hi(hi[g * 16 + j], __uint_as_float(a[j]), e);
            lo[j] = first ? __float_as_uint(e) : __float_as_uint(__fadd_rn(__uint_as_float(lo[j]), e));
          }
          tmem_st_32x32b_x16(tmem + lane_off + COL_LO + col, lo);
        }
        tmem_wait_st();
        ++chunk;
      }
      if (!ok) break;
      double* P = part + ((size_t)(w - W_MIN) * sh.units + u) * BM * BN;  // one slice per weight
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        uint32_t lo[32];
        tmem_ld_32x32b_x32(tmem + lane_off + COL_LO + (uint32_t)(c0w + g * 32), lo);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j)
          P[(size_t)(c0w + g * 32 + j) * BM + row] =
              weight * ((double)hi[g * 32 + j] + (double)__uint_as_float(lo[j]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// D[a, b] = D[b, a] = 2^(s_a + s_b) * sum over splits of the unit partials, a <= b
__global__ void ozaki_reduce(const double* __restrict__ part, OzShape sh, const int* __restrict__ sexp, int accumulate,
                             double* __restrict__ D, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t kk = sh.k;
  if (e >= kk * kk) return;
  const int a = (int)(e % kk), b = (int)(e / kk);
  if (a > b) return;
  const int ta = a / BM, tb = b / BN;
  const int t = tile_index(ta, tb, sh.tn);
  const size_t off = (size_t)(b - tb * BN) * BM + (a - ta * BM);
  double s = 0.0;
  for (int wi = 0; wi <= W_MAX - W_MIN; ++wi)
    for (int sp = 0; sp < sh.splits; ++sp)
      s += part[((size_t)wi * sh.units + (size_t)sp * sh.ntiles + t) * BM * BN + off];
  s = ldexp(s, sexp[a] + sexp[b]);
  if (accumulate) s += D[a + (int64_t)b * ldd];
  D[a + (int64_t)b * ldd] = s;
  D[b + (int64_t)a * ldd] = s;
}

OzShape make_oz_shape(int64_t n, int64_t k) {
  OzShape s;
  s.n = n;
  s.nrb = (n + BK - 1) / BK;
  s.ncb = (k + BM - 1) / BM;
  s.k = (int)k;
  s.tn = (int)s.ncb;
  s.ntiles = s.tn * (s.tn + 1) / 2;
  const int64_t min_split = (n + kMaxUnitRows - 1) / kMaxUnitRows;
  const int64_t max_split = (n + 4 * BK - 1) / (4 * BK) > 0 ? (n + 4 * BK - 1) / (4 * BK) : 1;
  int best = (int)min_split;
  double best_eff = -1.0;
  for (int64_t sp = min_split; sp <= min_split + 256 && sp <= (max_split > min_split ? max_split : min_split); ++sp) {
    const int64_t units = (int64_t)s.ntiles * sp;
    const int64_t waves = (units + kSmTarget - 1) / kSmTarget;
    const double eff = (double)units / (double)(waves * kSmTarget) - 0.0005 * (double)sp;
    if (eff > best_eff) {
      best_eff = eff;
      best = (int)sp;
    }
    if (units >= 16 * kSmTarget) break;
  }
  int64_t rps = (n + best - 1) / best;
  rps = (rps + BK - 1) / BK * BK;
  s.rows_per_split = rps;
  s.splits = (int)((n + rps - 1) / rps);
  s.units = s.ntiles * s.splits;
  s.stall = 0;
  return s;
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

struct OzWs {
  __nv_bfloat16* planes;
  double* part;
  int* sexp;
  unsigned* err;
  size_t used;
};

OzWs carve_oz(void* base, int64_t n, int64_t k) {
  const OzShape s = make_oz_shape(n, k);
  Carver c(base);
  OzWs w;
  w.planes = c.take<__nv_bfloat16>((size_t)NDIG * s.nrb * s.ncb * BK * BM);
  w.part = c.take<double>((size_t)(W_MAX - W_MIN + 1) * s.units * BM * BN);
  w.sexp = c.take<int>(k);
  w.err = c.take<unsigned>(1);
  w.used = c.used;
  return w;
}

}  // namespace

size_t gram_ozaki_workspace(int64_t n, int64_t k) { return carve_oz(nullptr, n, k).used; }

int gram_ozaki(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int accumulate, double* D, int64_t ldd,
               unsigned* dev_flags, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (k > 65535 || n > ((int64_t)1 << 40)) return DOPINF_E_UNSUPPORTED;
  OzShape sh = make_oz_shape(n, k);
  sh.stall = (test_stall() & kStallTensorGram) ? 1 : 0;
  if ((int64_t)NDIG * sh.nrb * sh.ncb > (int64_t)INT32_MAX) return DOPINF_E_UNSUPPORTED;
  if (!ws || ws_bytes < gram_ozaki_workspace(n, k) || misaligned(ws)) return DOPINF_E_ARG;
  OzWs w = carve_oz(ws, n, k);
  DOPINF_CUDA(cudaMemsetAsync(w.err, 0, sizeof(unsigned), st));
  if (dtype == DOPINF_F64)
    colmax_kernel<double><<<(unsigned)k, 256, 0, st>>>(static_cast<const double*>(Q), n, ldq, w.sexp, w.err);
  else
    colmax_kernel<float><<<(unsigned)k, 256, 0, st>>>(static_cast<const float*>(Q), n, ldq, w.sexp, w.err);
  DOPINF_TRY(launch_status());
  {
    // rows split in chunks of 256 threads x 4 rows, enough CTAs for ~32 per SM over all columns
    const int64_t rows = sh.nrb * BK, cols = sh.ncb * BM;
    const int64_t xb_need = (rows + 1023) / 1024;
    const int64_t ycols = cols < 65535 ? cols : 65535;
    int64_t xb = (152 * 32 + ycols - 1) / ycols;
    xb = xb < 1 ? 1 : (xb > xb_need ? xb_need : xb);
    const dim3 grid((unsigned)xb, (unsigned)ycols);
    if (dtype == DOPINF_F64)
      digits_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(Q), n, k, ldq, w.sexp, w.planes, sh.nrb,
                                                  sh.ncb);
    else
      digits_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(Q), n, k, ldq, w.sexp, w.planes, sh.nrb,
                                                 sh.ncb);
  }
  DOPINF_TRY(launch_status());
  CUtensorMap map;
  if (!make_map(&map, w.planes, (int64_t)NDIG * sh.nrb * sh.ncb)) return DOPINF_E_CUDA;
  DOPINF_CUDA(cudaFuncSetAttribute(ozaki_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
  {
    int per_sm = 0;  // the kernel needs one resident CTA per SM (registers, shared memory)
    DOPINF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ozaki_pass_kernel, NTHREADS, SMEM_BYTES));
    if (per_sm < 1) {
      set_last_error("ozaki_pass_kernel does not fit on an SM", cudaErrorLaunchOutOfResources);
      return DOPINF_E_CUDA;
    }
  }
  int sms = 0, dev = 0;
  DOPINF_CUDA(cudaGetDevice(&dev));
  DOPINF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sh.units < sms ? sh.units : sms;
  for (int wgt = W_MIN; wgt <= W_MAX; ++wgt) {
    ozaki_pass_kernel<<<grid, NTHREADS, SMEM_BYTES, st>>>(map, sh, wgt, w.part, w.err);
    DOPINF_TRY(launch_status());
  }
  const int64_t kk = k * k;
  ozaki_reduce<<<(unsigned)((kk + 255) / 256), 256, 0, st>>>(w.part, sh, w.sexp, accumulate, D, ldd);
  DOPINF_TRY(launch_status());
  return finish_timeout(w.err, dev_flags, st);
}

}  // namespace dopinf
