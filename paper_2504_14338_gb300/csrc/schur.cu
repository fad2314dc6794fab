// Regularised normal equations of Step IV, (G + diag(reg)) O^T = B (Section 3.5, eq. OpInf_reg;
// the Step IV code solves one system per (beta1, beta2)), for every candidate of a grid by
// block elimination of the quadratic unknowns.
//
// Order the d unknowns as S (the s = r(r+1)/2 quadratic terms, regularised by beta2) and L
// (the r linear terms and the constant, m = r + 1 of them, regularised by beta1):
//     [ G_SS + beta2 I   G_SL           ] [x_S]   [B_S]
//     [ G_LS             G_LL + beta1 I ] [x_L] = [B_L].
// The S block does not depend on beta1.  So, per (r, beta2) "unit", a Cholesky of the
// symmetric matrix E = [[G_SS + beta2 I, G_SL, B_S], [G_LS, G_LL, B_L], [B_S^T, B_L^T, *]]
// (size N = s + m + r) is run over its first s columns only.  That leaves
//     L_S (the factor of G_SS + beta2 I),  W = G_LS L_S^-T,  V^T = B_S^T L_S^-T,
//     C0 = G_LL - W W^T and B'_L = B_L - W V  in the trailing block,
// and a blocked back substitution L_S^T [Z | Y] = [W^T | V] gives Z = (G_SS + beta2 I)^-1 G_SL
// and Y = (G_SS + beta2 I)^-1 B_S.  Per candidate (r, beta1, beta2) what is left is small:
//     (C0 + beta1 I) x_L = B'_L   (Cholesky of order m),   x_S = Y - Z x_L.
// This is the Cholesky factorisation of the symmetrically permuted matrix, so it is exact in
// exact arithmetic and backward stable like the plain one; a non-positive pivot (in the unit
// or in the candidate's block) marks the candidate invalid.
//
// Work: one unit costs ~s^3/3 + 2 s^2 (m + r) flop and is shared by the n_b1 candidates of its
// beta2; a candidate costs ~m^3/3 + s m r.  Everything is FP64 (the FP64 pipe binds).  Units run
// in parallel: per 32-column panel, a diagonal-block factorisation (one warp per unit), a
// triangular solve of the rows below (a thread per row) and a tile update of the trailing
// matrix (64 x 64 tiles), each one launch over all units; the back substitution runs by panels
// in the same way.
#include "common.cuh"
#include <math.h>

namespace dopinf {
namespace {

constexpr int NB = 32;  // panel width
constexpr int TT = 64;  // update tile
constexpr int SB = 256;

__device__ __forceinline__ int panel_width(int s, int p0) { return s - p0 < NB ? s - p0 : NB; }

// natural index (0..d-1, order [linear r | quadratic s | constant]) of permuted position p
__device__ __forceinline__ int natural(int p, int r, int s) {
  if (p < s) return r + p;
  const int q = p - s;
  return q < r ? q : r + s;
}

__global__ void __launch_bounds__(SB) schur_build(const SchurUnit* __restrict__ units, int* __restrict__ fail) {
  const SchurUnit U = units[blockIdx.y];
  const int r = U.r, s = U.s, m = U.m, N = U.N, d = U.d;
  if (blockIdx.x == 0 && threadIdx.x == 0) fail[U.unit] = 0;
  const int64_t total = (int64_t)N * (s + m);  // columns 0..s+m-1, rows j..N-1
  for (int64_t e = (int64_t)blockIdx.x * SB + threadIdx.x; e < total; e += (int64_t)gridDim.x * SB) {
    const int j = (int)(e / N), i = (int)(e % N);
    if (i < j) continue;
    const int nj = natural(j, r, s);
    double v;
    if (i < s + m) {
      v = U.G[natural(i, r, s) + (int64_t)nj * d];
      if (i == j && i < s) v += U.b2;
    } else {
      v = U.B[nj + (int64_t)(i - s - m) * d];
    }
    U.E[i + (int64_t)j * N] = v;
  }
}

// Cholesky of the diagonal block of panel p0, one warp per unit (lane = row of the block).
__global__ void schur_potrf(const SchurUnit* __restrict__ units, int p0, int* __restrict__ fail) {
  __shared__ double a[NB][NB + 1];
  const SchurUnit U = units[blockIdx.x];
  if (p0 >= U.s || fail[U.unit]) return;
  const int pw = panel_width(U.s, p0), N = U.N, lane = threadIdx.x;
  double* E = U.E;
  if (lane < pw)
    for (int j = 0; j <= lane; ++j) a[lane][j] = E[(p0 + lane) + (int64_t)(p0 + j) * N];
  __syncwarp();
  bool bad = false;
  for (int j = 0; j < pw; ++j) {
    const double piv = a[j][j];
    if (!(piv > 0.0) || !isfinite(piv)) {
      bad = true;
      break;
    }
    const double ljj = sqrt(piv), inv = 1.0 / ljj;
    if (lane > j && lane < pw) a[lane][j] *= inv;
    __syncwarp();
    if (lane == j) a[j][j] = ljj;
    if (lane > j && lane < pw) {
      const double lij = a[lane][j];
      for (int c = j + 1; c <= lane; ++c) a[lane][c] = fma(-lij, a[c][j], a[lane][c]);
    }
    __syncwarp();
  }
  if (bad) {
    if (lane == 0) fail[U.unit] = 1;
    return;
  }
  if (lane < pw)
    for (int j = 0; j <= lane; ++j) E[(p0 + lane) + (int64_t)(p0 + j) * N] = a[lane][j];
}

// Rows below the diagonal block: E[i, panel] <- E[i, panel] L_pp^-T, one thread per row.
__global__ void __launch_bounds__(SB) schur_trsm(const SchurUnit* __restrict__ units, int p0,
                                                 const int* __restrict__ fail) {
  __shared__ double Lp[NB][NB + 1];
  __shared__ double invd[NB];  // reciprocals of the diagonal: the sweep multiplies, no division on its chain
  const SchurUnit U = units[blockIdx.y];
  if (p0 >= U.s || fail[U.unit]) return;
  const int pw = panel_width(U.s, p0), N = U.N, q0 = p0 + pw;
  if (q0 + (int)blockIdx.x * SB >= N) return;
  double* E = U.E;
  for (int e = threadIdx.x; e < NB * NB; e += SB) {
    const int i = e % NB, j = e / NB;
    if (i < pw && j <= i) Lp[i][j] = E[(p0 + i) + (int64_t)(p0 + j) * N];
  }
  __syncthreads();
  if (threadIdx.x < pw) invd[threadIdx.x] = 1.0 / Lp[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int row = q0 + (int)blockIdx.x * SB + threadIdx.x;
  if (row >= N) return;
  double x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < pw) {
      double v = E[row + (int64_t)(p0 + j) * N];
#pragma unroll
      for (int l = 0; l < j; ++l) v = fma(-x[l], Lp[j][l], v);
      x[j] = v * invd[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < pw) E[row + (int64_t)(p0 + j) * N] = x[j];
}

__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
  ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  tj = t - ti * (ti + 1) / 2;
}

// Trailing update E[i][j] -= sum_l E[i][p0+l] E[j][p0+l] over the lower 64 x 64 tiles of rows
// and columns >= p0 + pw, columns < s + m (the right-hand-side block against itself is never
// needed).
__global__ void __launch_bounds__(SB) schur_update(const SchurUnit* __restrict__ units, int p0,
                                                   const int* __restrict__ fail) {
  __shared__ double As[NB][TT], Bs[NB][TT];
  const SchurUnit U = units[blockIdx.y];
  if (p0 >= U.s || fail[U.unit]) return;
  const int pw = panel_width(U.s, p0), N = U.N, q0 = p0 + pw, cols = U.s + U.m;
  const int T = (N - q0 + TT - 1) / TT;
  if ((int)blockIdx.x >= T * (T + 1) / 2) return;
  int ti, tj;
  tri_tile((int)blockIdx.x, ti, tj);
  const int R0 = q0 + ti * TT, C0 = q0 + tj * TT;
  if (C0 >= cols) return;
  double* E = U.E;
  for (int e = threadIdx.x; e < NB * TT; e += SB) {
    const int x = e % TT, l = e / TT;
    const int ra = R0 + x, cb = C0 + x;
    As[l][x] = (l < pw && ra < N) ? E[ra + (int64_t)(p0 + l) * N] : 0.0;
    Bs[l][x] = (l < pw && cb < N) ? E[cb + (int64_t)(p0 + l) * N] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int l = 0; l < pw; ++l) {
    double av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[l][tx + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[l][ty + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = R0 + tx + 16 * a, j = C0 + ty + 16 * b;
      if (i < N && j < cols && i >= j) E[i + (int64_t)j * N] -= acc[a][b];
    }
}

// Back substitution L_S^T X = R on panel [p0, p0 + pw), R[p][c] = E[(s + c) + p N] for the
// m + r columns c; one thread per column.
__global__ void schur_back_diag(const SchurUnit* __restrict__ units, int p0, const int* __restrict__ fail) {
  __shared__ double Lp[NB][NB + 1];
  __shared__ double invd[NB];  // reciprocals of the diagonal: the sweep multiplies
  const SchurUnit U = units[blockIdx.x];
  if (p0 >= U.s || fail[U.unit]) return;
  const int pw = panel_width(U.s, p0), N = U.N, s = U.s, nc = U.m + U.r;
  double* E = U.E;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    if (i < pw && j <= i) Lp[i][j] = E[(p0 + i) + (int64_t)(p0 + j) * N];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < pw; j += blockDim.x) invd[j] = 1.0 / Lp[j][j];
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    double x[NB];
#pragma unroll
    for (int jj = NB - 1; jj >= 0; --jj) {
      if (jj < pw) {
        double v = E[(s + c) + (int64_t)(p0 + jj) * N];
#pragma unroll
        for (int l = jj + 1; l < NB; ++l)
          if (l < pw) v = fma(-Lp[l][jj], x[l], v);
        x[jj] = v * invd[jj];
      }
    }
#pragma unroll
    for (int jj = 0; jj < NB; ++jj)
      if (jj < pw) E[(s + c) + (int64_t)(p0 + jj) * N] = x[jj];
  }
}

// Rows above the panel: R[q][c] -= sum_l L[p0 + l][q] X[p0 + l][c], tiles of 64 q x 64 c.
__global__ void __launch_bounds__(SB) schur_back_update(const SchurUnit* __restrict__ units, int p0,
                                                        const int* __restrict__ fail) {
  __shared__ double Ls[NB][TT], Xs[NB][TT];
  const SchurUnit U = units[blockIdx.y];
  if (p0 >= U.s || fail[U.unit] || p0 == 0) return;
  const int pw = panel_width(U.s, p0), N = U.N, s = U.s, nc = U.m + U.r;
  const int nq = (p0 + TT - 1) / TT, ncb = (nc + TT - 1) / TT;
  if ((int)blockIdx.x >= nq * ncb) return;
  const int q0 = ((int)blockIdx.x % nq) * TT, c0 = ((int)blockIdx.x / nq) * TT;
  double* E = U.E;
  for (int e = threadIdx.x; e < NB * TT; e += SB) {
    const int l = e % NB, x = e / NB;  // l fastest: column q of L is contiguous in l
    const int q = q0 + x;
    Ls[l][x] = (l < pw && q < p0) ? E[(p0 + l) + (int64_t)q * N] : 0.0;
  }
  for (int e = threadIdx.x; e < NB * TT; e += SB) {
    const int x = e % TT, l = e / TT;
    const int c = c0 + x;
    Xs[l][x] = (l < pw && c < nc) ? E[(s + c) + (int64_t)(p0 + l) * N] : 0.0;
  }
  __syncthreads();
  const int tc = threadIdx.x & 15, tq = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int l = 0; l < pw; ++l) {
    double lv[4], xv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) lv[a] = Ls[l][tq + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) xv[b] = Xs[l][tc + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(lv[a], xv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int q = q0 + tq + 16 * a, c = c0 + tc + 16 * b;
      if (q < p0 && c < nc) E[(s + c) + (int64_t)q * N] -= acc[a][b];
    }
}

// One CTA per candidate: (C0 + beta1 I) x_L = B'_L by Cholesky (in the candidate's scratch),
// x_S = Y - Z x_L, written as the operator O (r x d, ld r) in the natural order.
__global__ void __launch_bounds__(SB) schur_candidate(const SchurCand* __restrict__ cands,
                                                      const int* __restrict__ fail, int* __restrict__ status) {
  __shared__ int s_fail;
  const SchurCand cc = cands[blockIdx.x];
  const int r = cc.r, s = cc.s, m = cc.m, N = cc.N;
  const double* E = cc.E;
  double* C = cc.scratch;                 // m x m, ld m
  double* X = cc.scratch + (size_t)m * m;  // m x r, ld m
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = SB / 32;
  if (fail[cc.unit]) {
    if (tid == 0) status[cc.cand] = 1;
    return;
  }
  for (int e = tid; e < m * m; e += SB) {
    const int i = e % m, j = e / m;
    if (i >= j) C[e] = E[(s + i) + (int64_t)(s + j) * N] + (i == j ? cc.b1 : 0.0);
  }
  for (int e = tid; e < m * r; e += SB) {
    const int a = e % m, c = e / m;
    X[e] = E[(s + m + c) + (int64_t)(s + a) * N];
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    const double piv = C[j + j * m];
    if (!(piv > 0.0) || !isfinite(piv)) {
      if (tid == 0) s_fail = 1;
      break;
    }
    const double ljj = sqrt(piv), inv = 1.0 / ljj;
    for (int i = j + 1 + tid; i < m; i += SB) C[i + j * m] *= inv;
    __syncthreads();
    if (tid == 0) C[j + j * m] = ljj;
    for (int c = j + 1 + w; c < m; c += nw) {
      const double lc = C[c + j * m];
      for (int i = c + lane; i < m; i += 32) C[i + c * m] = fma(-C[i + j * m], lc, C[i + c * m]);
    }
    __syncthreads();
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) status[cc.cand] = 1;
    return;
  }
  for (int j = 0; j < m; ++j) {  // L z = b
    const double inv = 1.0 / C[j + j * m];
    for (int c = tid; c < r; c += SB) X[j + c * m] *= inv;
    __syncthreads();
    const int rows = m - j - 1;
    for (int e = tid; e < rows * r; e += SB) {
      const int i = j + 1 + e % rows, c = e / rows;
      X[i + c * m] = fma(-C[i + j * m], X[j + c * m], X[i + c * m]);
    }
    __syncthreads();
  }
  for (int j = m - 1; j >= 0; --j) {  // L^T x = z
    const double inv = 1.0 / C[j + j * m];
    for (int c = tid; c < r; c += SB) X[j + c * m] *= inv;
    __syncthreads();
    for (int e = tid; e < j * r; e += SB) {
      const int i = e % j, c = e / j;
      X[i + c * m] = fma(-C[j + i * m], X[j + c * m], X[i + c * m]);
    }
    __syncthreads();
  }
  // O[:, a] for the linear terms (a < r) and the constant (a = r + s): x_L
  for (int e = tid; e < r * m; e += SB) {
    const int i = e % r, a = e / r;
    const int nat = a < r ? a : r + s;
    cc.O[i + (int64_t)nat * r] = X[a + i * m];
  }
  // quadratic terms: x_S[p][c] = Y[p][c] - sum_a Z[p][a] x_L[a][c], a warp per p, lanes over c
  for (int p = w; p < s; p += nw) {
    const double* Zp = E + s + (int64_t)p * N;  // Z[p][a] = Zp[a], Y[p][c] = Zp[m + c]
    for (int c = lane; c < r; c += 32) {
      double v = Zp[m + c];
      for (int a = 0; a < m; ++a) v = fma(-Zp[a], X[a + c * m], v);
      cc.O[c + (int64_t)(r + p) * r] = v;
    }
  }
  if (tid == 0) status[cc.cand] = 0;
}

}  // namespace

size_t schur_unit_doubles(int r) {
  const int64_t s = (int64_t)r * (r + 1) / 2, N = s + 2 * r + 1;
  return (size_t)(N * N);
}
size_t schur_cand_doubles(int r) { return (size_t)(r + 1) * (r + 1) + (size_t)(r + 1) * r; }

int schur_solve(const SchurUnit* units_dev, const SchurUnit* units_host, int n_units, const SchurCand* cands_dev,
                int n_cand, int* unit_fail, int* cand_status, cudaStream_t st) {
  int s_max = 0, N_max = 0, nc_max = 0;
  for (int u = 0; u < n_units; ++u) {
    s_max = units_host[u].s > s_max ? units_host[u].s : s_max;
    N_max = units_host[u].N > N_max ? units_host[u].N : N_max;
    nc_max = units_host[u].m + units_host[u].r > nc_max ? units_host[u].m + units_host[u].r : nc_max;
  }
  {
    const int64_t tot = (int64_t)N_max * N_max;
    int64_t gx = (tot + SB - 1) / SB;
    gx = gx > 1024 ? 1024 : gx;
    schur_build<<<dim3((unsigned)gx, (unsigned)n_units), SB, 0, st>>>(units_dev, unit_fail);
    DOPINF_TRY(launch_status());
  }
  // forward: partial Cholesky over the S columns, panel by panel
  for (int p0 = 0; p0 < s_max; p0 += NB) {
    schur_potrf<<<n_units, 32, 0, st>>>(units_dev, p0, unit_fail);
    int gx = 1, tiles = 1;
    for (int u = 0; u < n_units; ++u) {
      const SchurUnit& U = units_host[u];
      if (p0 >= U.s) continue;
      const int q0 = p0 + (U.s - p0 < NB ? U.s - p0 : NB);
      const int rows = U.N - q0, T = (rows + TT - 1) / TT;
      gx = (rows + SB - 1) / SB > gx ? (rows + SB - 1) / SB : gx;
      tiles = T * (T + 1) / 2 > tiles ? T * (T + 1) / 2 : tiles;
    }
    schur_trsm<<<dim3((unsigned)gx, (unsigned)n_units), SB, 0, st>>>(units_dev, p0, unit_fail);
    schur_update<<<dim3((unsigned)tiles, (unsigned)n_units), SB, 0, st>>>(units_dev, p0, unit_fail);
    DOPINF_TRY(launch_status());
  }
  // backward: L_S^T [Z | Y] = [W^T | V], panels from the last
  for (int p0 = ((s_max - 1) / NB) * NB; p0 >= 0; p0 -= NB) {
    schur_back_diag<<<n_units, 128, 0, st>>>(units_dev, p0, unit_fail);
    if (p0 > 0) {
      const int blocks = ((p0 + TT - 1) / TT) * ((nc_max + TT - 1) / TT);
      schur_back_update<<<dim3((unsigned)blocks, (unsigned)n_units), SB, 0, st>>>(units_dev, p0, unit_fail);
    }
    DOPINF_TRY(launch_status());
  }
  schur_candidate<<<n_cand, SB, 0, st>>>(cands_dev, unit_fail, cand_status);
  return launch_status();
}

}  // namespace dopinf
