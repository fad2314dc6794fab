// Internal helpers of the dOpInf CUDA library (sm_103a).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "../../include/dopinf.h"

#define DOPINF_API extern "C" __attribute__((visibility("default")))

namespace dopinf {

constexpr int kMaxVars = 64;
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// Carves aligned sub-buffers out of a caller workspace.  With base == nullptr it only
// counts bytes, so the *_workspace() queries and the entry points share one layout.
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    size_t off = used;
    used = align_up(used + count * sizeof(T));
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Text of the last CUDA error the library met (per host thread), for dopinf_last_error().
void set_last_error(const char* where, cudaError_t e);

inline int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DOPINF_OK;
  set_last_error("CUDA call", e);
  return DOPINF_E_CUDA;
}

// Launch-error check after a kernel launch (does not synchronise).
inline int launch_status() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return DOPINF_OK;
  set_last_error("kernel launch", e);
  return DOPINF_E_CUDA;
}

// *flags |= bits if *err is non-zero (device-side status hand-off, no synchronisation).
void flag_if_set(const unsigned* err, unsigned* flags, unsigned bits, cudaStream_t st);
// Bit of a kernel error word that reports NaN/Inf in the data; its other bits report an
// expired bounded wait.
constexpr unsigned kErrNonfinite = 0x100u;
// Finish a call that left a device error word: flag it (asynchronous: DOPINF_FLAG_TIMEOUT /
// DOPINF_FLAG_NONFINITE into *dev_flags) or read it back (DOPINF_E_TIMEOUT, else
// DOPINF_E_NONFINITE).
int finish_timeout(const unsigned* err, unsigned* dev_flags, cudaStream_t st);
// Test knob of the error paths (dopinf_test_expire_waits): bits of the bounded waits whose
// signal is withheld, so that they expire.
constexpr int kStallGridBarrier = 1, kStallTensorGram = 2;
int test_stall();

inline bool misaligned(const void* p, size_t a = kAlign) {
  return (reinterpret_cast<uintptr_t>(p) % a) != 0;
}

#define DOPINF_TRY(expr)                 \
  do {                                   \
    int _st = (expr);                    \
    if (_st != DOPINF_OK) return _st;    \
  } while (0)

#define DOPINF_CUDA(expr) DOPINF_TRY(::dopinf::cuda_status(expr))

// ---------------------------------------------------------------------------------------
// Generic FP64 "TN" product C = A^T B (A: K x M, B: K x N, both column-major, element type
// double or float promoted exactly), split over K with a fixed-order reduction.  Used by the
// Gram of Step III and the normal equations of Step IV.  Implemented in gram_fp64.cu.
// sym = 1 requires A == B, M == N and computes only the upper tiles, mirroring them.
// ---------------------------------------------------------------------------------------
size_t tn_workspace(int64_t K, int64_t M, int64_t N, int sym);
int tn_product(const void* A, int64_t lda, const void* B, int64_t ldb, int dtype, int64_t K,
               int64_t M, int64_t N, int sym, int accumulate, double* C, int64_t ldc, void* ws,
               size_t ws_bytes, cudaStream_t st);

// Split-precision Gram on the tensor cores (gram_tc.cu); synchronises the stream.
size_t gram_tc_workspace(int64_t n, int64_t k);
int64_t gram_tc_set_chunk_rows(int64_t rows);
// FP64-accurate Gram from exact integer digit products on the tensor cores (gram_ozaki.cu).
size_t gram_ozaki_workspace(int64_t n, int64_t k);
// dev_flags == nullptr: synchronise and return DOPINF_E_TIMEOUT if a bounded wait expired;
// otherwise stay asynchronous and OR DOPINF_FLAG_TIMEOUT into *dev_flags on the device.
int gram_ozaki(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int accumulate, double* D, int64_t ldd,
               unsigned* dev_flags, void* ws, size_t ws_bytes, cudaStream_t st);
int gram_tc(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int accumulate, double* D, int64_t ldd,
            unsigned* dev_flags, void* ws, size_t ws_bytes, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// Batched ROM rollouts (rollout.cu): one thread-block cluster per candidate.
// ---------------------------------------------------------------------------------------
// Block-Schur solve of the regularised normal equations of all candidates (schur.cu).
struct SchurUnit {  // one (r, beta2)
  const double* G;  // d x d normal matrix of this r (ld d)
  const double* B;  // d x r right-hand sides (ld d)
  double* E;        // N x N (ld N) working matrix, N = s + m + r
  double b2;
  int r, d, s, m, N, unit;
};
struct SchurCand {  // one (r, beta1, beta2)
  const double* E;  // its unit's working matrix
  double* O;        // r x d operator output (ld r)
  double* scratch;  // schur_cand_doubles(r) doubles
  double b1;
  int r, s, m, N, unit, cand;
};
// QR route of the same regularised problems (qr_solve.cu): the candidates [cand0, cand0 + n) of
// one r, each from the stacked system [Dhat; diag(sqrt(reg))] in its own slice of `work`
// (stride doubles, at least qr_solve_doubles(K, r)); writes O and the candidate's status.
size_t qr_solve_doubles(int64_t K, int r);
int qr_solve(const double* Dh, const double* Y, int64_t K, int r, const SchurUnit* units, const SchurCand* cands,
             int cand0, int n, double* work, size_t stride, int* cand_status, cudaStream_t st);
size_t schur_unit_doubles(int r);
size_t schur_cand_doubles(int r);
int schur_solve(const SchurUnit* units_dev, const SchurUnit* units_host, int n_units, const SchurCand* cands_dev,
                int n_cand, int* unit_fail, int* cand_status, cudaStream_t st);

// Width of the quadratic OpInf data row [q, (q_i q_j)_{i<=j}, 1] for reduced dimension r.
__host__ __device__ inline int dim_d(int r) { return r + r * (r + 1) / 2 + 1; }

struct RolloutCand {
  const double* O;      // r x d column-major operator [A | H | c], leading dimension ldo
  int64_t ldo;
  int r, d;
  int cand;             // index into the per-candidate outputs
  const double* mu;     // temporal mean of the reference data (r), metrics runs only
  const double* denom;  // max_{t<k,i} |qhat - mu|, metrics runs only
  const double* inv_den;  // 1 / sum_i qhat_{i,t}^2 for t < k, metrics runs only
};

struct RolloutBatch {
  const RolloutCand* cands;  // device table of n_cand candidates, or nullptr to use `one`
  RolloutCand one;
  int n_cand, r_max, d_max;
  int mode;
  double dt;
  int64_t n_steps;
  const double* q0;     // initial state (first r entries)
  // metrics (metrics = 1): training error over the first k states against Qhat (ld ldqh)
  int metrics;
  const double* Qhat;
  int64_t ldqh, k;
  double max_growth;
  double* train_err;
  double* growth;
  int* status;
  int64_t* steps;  // optional: steps each rollout advanced (its RHS evaluations = steps x stages)
  // trajectory output (traj = 1): n_steps x r row-major; rows after the first non-finite
  // state are not written
  int traj;
  double* traj_out;
  int* finite;
  // arithmetic (DOPINF_ROLLOUT_FP64 or DOPINF_ROLLOUT_DW), and redo = 1 for the FP64 pass over
  // the candidates a double-word pass handed back (status 4)
  int arith;
  int redo;
};

// Rollouts (rollout.cu).  Column-owned kernel for r <= 32: whether r is supported, the rows per
// CTA and cluster size a launch for r would use (0 if none fits), the process-wide preferred
// rows per CTA (1, 2, 4, 8; other values only query; returns the previous value), and the launch
// of candidates [cand0, cand0 + n) of one r (chained: programmatic dependent launch behind the
// previous rollout launch on the stream, which it completes after).  Shared-memory kernel for
// 32 < r <= 92: the same, with preferred rows per CTA 3..8.
bool rollout_cols_supported(int r);
int rollout_cols_shape(int r, int* rows, int* cluster);
int rollout_set_rows(int rc);
int launch_rollouts_cols(RolloutBatch bt, int cand0, int n, int r, bool chained, cudaStream_t st);
bool rollout_big_supported(int r);
int rollout_big_shape(int r, int* rows, int* cluster, size_t* smem);
int rollout_set_rows_big(int rc);
int launch_rollouts_big(RolloutBatch bt, int cand0, int n, int r, bool chained, cudaStream_t st);
// Either kernel, chosen by r.
bool rollout_supported(int r);
int rollout_shape(int r);
int launch_rollouts_rank(RolloutBatch bt, int cand0, int n, int r, bool chained, cudaStream_t st);
int rollout_set_arith(int a);
int rollout_arith();

}  // namespace dopinf
