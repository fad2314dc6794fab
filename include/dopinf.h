/*
 * dopinf.h - C ABI of the GB300 (sm_103a) dOpInf hot path.
 *
 * Distributed Operator Inference (Farcas, Gundevia, Munipalli, Willcox, arXiv 2504.14338)
 * on one GPU: Step II (centering and max-abs scaling, Section 3.3), Step III (method of
 * snapshots Gram, eigensolve, retained energy and basis-free projection, Section 3.4,
 * eqs. mos_partitioned, mos_Sigma_W, ret_energy, MoS_POD_basis, dOpInf_projection) and
 * Step IV (quadratic OpInf with a regularisation grid search and ROM rollouts, Section 3.5,
 * eqs. ROM_quad_time_cont, ROM_quad_time_discrete, OpInf_reg,
 * OpInf_data_matrices_discrete).
 *
 * Conventions shared by every entry point
 *  - Pointers are caller-owned DEVICE memory unless the comment says "host".  The library
 *    never frees caller memory and allocates no device memory: scratch comes from the
 *    caller's workspace (ws, ws_bytes), sized by the matching *_workspace() query.  The
 *    workspace must be 256-byte aligned.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream unless the comment says the call synchronises it.
 *  - Matrices are column-major with an explicit leading dimension.  The snapshot matrix
 *    Q is n x k: column t (snapshot t) holds rows 0..n-1 contiguously, rows are stacked
 *    variable by variable (all rows of variable 0, then variable 1, ...).
 *  - Argument errors return DOPINF_E_ARG before anything is launched.  Conditions the
 *    GPU detects (non-finite data, a zero scale) are OR-ed as DOPINF_FLAG_* bits into the
 *    optional device word dev_flags; calls that synchronise also return them as codes.
 *  - Thread safety: calls on different streams with disjoint workspaces are independent.
 */
#ifndef DOPINF_H
#define DOPINF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum dopinf_status {
  DOPINF_OK = 0,
  DOPINF_E_ARG = -1,          /* invalid argument (null pointer, bad size, small workspace) */
  DOPINF_E_CUDA = -2,         /* a CUDA runtime call failed */
  DOPINF_E_NONFINITE = -4,    /* NaN or Inf found in the data */
  DOPINF_E_RANK = -6,         /* lambda_r <= 0, or the energy target is not reached by r_cap */
  DOPINF_E_NO_STABLE = -7,    /* no (r, beta1, beta2) candidate is finite and bounded */
  DOPINF_E_TIMEOUT = -8,      /* a bounded wait inside a tensor-core kernel expired */
  DOPINF_E_UNSUPPORTED = -9   /* valid request this build does not implement */
};

/* bits OR-ed into a device flag word */
#define DOPINF_FLAG_NONFINITE 1u   /* NaN/Inf in the data */
#define DOPINF_FLAG_ZERO_SCALE 2u  /* a variable block is constant after centering; scale := 1 */
#define DOPINF_FLAG_TIMEOUT 4u     /* a bounded wait inside a kernel expired: outputs not valid */
#define DOPINF_FLAG_RANK 8u        /* lambda_r <= 0, or the energy target not reached by r_cap */
#define DOPINF_FLAG_NO_STABLE 16u  /* no (r, beta1, beta2) candidate is finite and bounded */

enum dopinf_dtype { DOPINF_F64 = 0, DOPINF_F32 = 1 };

#define DOPINF_CENTER 1u
#define DOPINF_SCALE 2u
#define DOPINF_SCALE_STD 4u  /* scale by the standard deviation of the centred variable instead */

enum dopinf_gram_mode {
  DOPINF_GRAM_FP64 = 0,      /* FP64 FMA over every row (the plain path) */
  DOPINF_GRAM_BF16X4 = 1,    /* two BF16 slices per value, four tensor-core products (see dopinf_gram) */
  DOPINF_GRAM_OZAKI_FP64 = 2 /* FP64-accurate: exact integer digit products on the tensor cores */
};

enum dopinf_rom_mode {
  DOPINF_DISCRETE = 0,       /* q[t+1] = A q[t] + H (q[t] x q[t])_u + c  (eq. ROM_quad_time_discrete) */
  DOPINF_CONTINUOUS_RK4 = 1  /* q' = A q + H (q x q)_u + c, central-difference derivatives, RK4 rollout */
};

/* Arithmetic of the rollouts inside dopinf_learn / dopinf_learn_async (dopinf_rollout always
 * uses FP64): binary64, or double-word binary32 pairs (about 48 significant bits, on the FP32
 * pipe) with compensated dot products.  Double-word candidates whose operator or initial state
 * exceed 2^60 in magnitude, whose state stops being finite, or whose growth comes within 2^-20
 * (relative) of max_growth are rolled out again in FP64, so statuses and step counts follow the
 * FP64 arithmetic; train_err and growth agree with it to rounding of order 1e-12 relative for
 * stable rollouts. */
enum dopinf_rollout_arith {
  DOPINF_ROLLOUT_FP64 = 1,
  DOPINF_ROLLOUT_DW = 2
};

/* Human-readable name of a status code (static storage). */
const char* dopinf_status_string(int status);
/* Text of the last CUDA error behind a DOPINF_E_CUDA in this host thread ("" if none);
 * valid until the next failing call of the same thread. */
const char* dopinf_last_error(void);

/* Test of the error paths (no counterpart in the paper): which = DOPINF_TEST_GRID_BARRIER
 * withholds the release of the cooperative tridiagonalisation's grid barrier (dopinf_reduce),
 * DOPINF_TEST_TENSOR_GRAM keeps the MMA issuer of the tensor-core Grams (BF16X4, and the first
 * digit pass of OZAKI_FP64) from releasing its pipeline stages.  The bounded waits that depend
 * on them then expire at their limit (about 2 s each); the kernels wind down (their copies and
 * MMAs in flight are waited for, tensor memory is released), the calls report
 * DOPINF_E_TIMEOUT or DOPINF_FLAG_TIMEOUT, and the context stays usable.  which = 0 restores
 * normal operation; which < 0 only queries.  Returns the previous value.  Process-wide; for
 * tests only. */
#define DOPINF_TEST_GRID_BARRIER 1
#define DOPINF_TEST_TENSOR_GRAM 2
int dopinf_test_expire_waits(int which);

/* ------------------------------------------------------------------------------------
 * Step II (Section 3.3): centre each row by its temporal mean, then divide each variable
 * block by the largest |centred value| of the block.
 *
 * Q            in/out, n x k, element type dtype, leading dimension ldq >= n (elements).
 * n_vars       number of variable blocks (1..64).
 * var_row_offsets host, n_vars + 1 nondecreasing row offsets, [0] = 0, [n_vars] = n.
 * flags        DOPINF_CENTER | DOPINF_SCALE, or DOPINF_CENTER | DOPINF_SCALE_STD: the other
 *              scaling Section 3.3 names, var_scale[j] = sqrt(sum c^2 / (rows_j k)) over the
 *              variable's centred values c (FP64 sums: per row in time order, rows in a fixed
 *              order; rounded to FP32 for FP32 data), then the same division as below.
 * row_mean     out, n doubles: mean_i = (sum_t Q[i,t], summed in t order in FP64) / k.
 * var_scale    out, n_vars doubles: max_{i in var, t} |Q[i,t] - mean_i|, rounded as the
 *              centred values are (FP64 data: FP64; FP32 data: fp32(fp64(x) - mean));
 *              a zero scale is replaced by 1 and DOPINF_FLAG_ZERO_SCALE is set.
 * Results:     FP64: Q = (Q - mean) / scale, each operation rounded to nearest.
 *              FP32: Q = fp32(fp64(Q) - mean) / fp32(scale), the division in FP32.
 *              Bit-identical to the definition (no reassociation, no contraction).
 * dev_flags    optional device unsigned int; DOPINF_FLAG_* bits are OR-ed in.
 * Workspace:   dopinf_transform_workspace(n, n_vars) bytes (may be NULL when dev_flags is given
 *              and DOPINF_SCALE_STD is not).
 * ------------------------------------------------------------------------------------ */
size_t dopinf_transform_workspace(int64_t n, int n_vars);
int dopinf_transform(void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int n_vars,
                     const int64_t* var_row_offsets, unsigned flags, double* row_mean,
                     double* var_scale, unsigned* dev_flags, void* ws, size_t ws_bytes,
                     void* stream);

/* ------------------------------------------------------------------------------------
 * Step III Gram matrix (eq. mos_partitioned): D = Q^T Q, k x k FP64, column-major,
 * leading dimension ldd >= k, both triangles written (D is exactly symmetric).
 * accumulate = 1 adds Q^T Q to D (row blocks of one snapshot matrix, the paper's
 * partitioned sum).  Results are run-to-run bit-reproducible in both modes.
 *
 * DOPINF_GRAM_FP64: Q is FP64 or FP32 (promoted exactly); FP64 products and sums over row
 *   chunks; the chunk partials are added in a fixed order.  Asynchronous.
 * DOPINF_GRAM_BF16X4: each value is split as x = h + l + e, h = bf16(x), l = bf16(x - h),
 *   and D ~= H^T H + H^T L + L^T H + L^T L on the tcgen05 tensor cores: FP32 accumulation
 *   over 128-row chunks with H^T H in columns of its own, a compensated FP32 (TwoSum) running
 *   sum per work unit, FP64 sum of the units (|e| <= 2^-17 |x|).  Requires k <= 65535.
 *   Synchronises the stream; returns DOPINF_E_TIMEOUT if an internal bounded wait expired,
 *   DOPINF_E_NONFINITE if Q holds a NaN or Inf (D is then not valid).
 * DOPINF_GRAM_OZAKI_FP64: column a is scaled by 2^-s_a (|x| < 2^(s_a - 1) on the column) and
 *   cut into 7 balanced integer digits of 8 bits (|d| <= 128, exact in BF16):
 *   x = 2^s_a sum_i d_i 2^(-8 i) + e, |e| <= 2^(s_a - 57).  The 28 digit products of weight
 *   2..8 are summed on the tensor cores
 *   in row chunks whose partial sums are integers below 2^24 (exact), carried exactly by FP32
 *   TwoSum pairs and combined in FP64: an FP64-accurate D (the method of Ozaki et al. 2012).
 *   Requires k <= 65535.  Synchronises the stream; may return DOPINF_E_TIMEOUT, or
 *   DOPINF_E_NONFINITE if Q holds a NaN or Inf (D is then not valid).
 * Workspace: dopinf_gram_workspace(n, k, dtype, mode) bytes (BF16X4: 4 n k bytes of
 *   slices plus the per-unit FP64 partial tiles; OZAKI_FP64: 14 n k bytes of digits plus
 *   7 partial tiles per unit).
 * ------------------------------------------------------------------------------------ */
size_t dopinf_gram_workspace(int64_t n, int64_t k, int dtype, int mode);
/* Tuning of DOPINF_GRAM_BF16X4: rows summed by one FP32 tensor-memory accumulator before it
 * is added to the compensated (TwoSum) running sum (rounded up to a multiple of 64; default
 * 128).  The tensor core's FP32 accumulation rounds toward zero by about half an ulp per MMA,
 * so longer chunks trade accuracy (a relative bias growing linearly with the chunk: about
 * -1.5e-9 per row of chunk on the diagonal) for fewer drains.
 * rows <= 0 only queries.  Returns the previous value.  Process-wide; not thread-safe against
 * concurrent dopinf_gram calls. */
int64_t dopinf_tune_gram_chunk(int64_t rows);
int dopinf_gram(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int mode,
                int accumulate, double* D, int64_t ldd, void* ws, size_t ws_bytes,
                void* stream);
/* The same product without any synchronisation (every mode; capturable into a CUDA graph):
 * a bounded wait that expired inside a tensor-core kernel ORs DOPINF_FLAG_TIMEOUT, and NaN or
 * Inf met by a tensor-core mode ORs DOPINF_FLAG_NONFINITE, into the device word *dev_flags
 * (required) instead of returning DOPINF_E_TIMEOUT / DOPINF_E_NONFINITE. */
int dopinf_gram_async(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int mode,
                      int accumulate, double* D, int64_t ldd, unsigned* dev_flags, void* ws,
                      size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------
 * Out-of-core Gram (Section 3.4, eq. mos_partitioned): D = Q^T Q (or D += Q^T Q) for a
 * snapshot matrix Q that stays in HOST memory (n x k, dtype, column-major, ld ldq >= n),
 * e.g. one larger than the device.  Row blocks of chunk_rows rows are copied into two device
 * buffers of the workspace on a copy stream of the library's own and accumulated into D (in
 * device memory) on `stream` with the Gram of `mode`, the upload of block c + 1 overlapping the
 * Gram of block c.  Q_host should be page-locked (cudaHostAlloc / cudaHostRegister) for the
 * copies to overlap.  Synchronises the stream; returns DOPINF_E_TIMEOUT / DOPINF_E_NONFINITE
 * as dopinf_gram does.  The copy stream is one per device: calls on one device from several
 * host threads at once are not supported.  Results: the partitioned sum in block order (the
 * same value class as dopinf_gram; bits may differ from a single call, whose row partition
 * differs).
 * Workspace: dopinf_gram_host_workspace(chunk_rows, k, dtype, mode) bytes.
 * ------------------------------------------------------------------------------------ */
size_t dopinf_gram_host_workspace(int64_t chunk_rows, int64_t k, int dtype, int mode);
int dopinf_gram_host(const void* Q_host, int dtype, int64_t n, int64_t k, int64_t ldq, int mode, int accumulate,
                     double* D, int64_t ldd, int64_t chunk_rows, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------
 * Allocation-free FP64 Gram.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory (code running inside a memory pool or an
 * allocator callback, plugins barred from the device allocator, code that runs while
 * another component is building a CUDA graph).  It computes exactly what
 * dopinf_gram(..., DOPINF_GRAM_FP64, ...) computes, same arguments minus the workspace,
 * with its scratch (the split-K partial tiles) in a fixed 32 MiB array of device memory
 * that every GPU loading this library holds until the process exits
 * (dopinf_gram_noalloc_scratch_bytes() returns the size).
 *  - Limit: k <= 2816 (the 64 x 64 upper tiles of D must fit the array); larger k returns
 *    DOPINF_E_UNSUPPORTED before anything is launched.  n >= 1.
 *  - The array is reserved when the driver loads this library's code on a device, which
 *    (under lazy module loading, the CUDA default) happens at the first call of this entry
 *    point or of any other library call that runs the FP64 Gram kernels on that device.
 *    That first use therefore does allocate device memory: make it outside any code that
 *    must not allocate (for example, once at start-up).
 *  - The first call on each device (the device must be current), and the first call after
 *    that device's context was replaced (cudaDeviceReset), resolve the array's device
 *    address; make that call before any stream capture, and not from several host threads
 *    at once.  Later calls only compare the context id.
 *  - Every call on a device shares the one array and leaves its last contents there; calls
 *    that overlap on the GPU (different streams, no ordering between them) race on it and
 *    give wrong results.  Calls on one stream are safe.  Asynchronous; D follows the same
 *    layout and symmetry rules as dopinf_gram.
 * ------------------------------------------------------------------------------------ */
size_t dopinf_gram_noalloc_scratch_bytes(void);
int dopinf_gram_fp64_noalloc(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, int accumulate,
                             double* D, int64_t ldd, void* stream);

/* ------------------------------------------------------------------------------------
 * Step III eigensolve and projection (eqs. mos_Sigma_W, ret_energy, MoS_POD_basis,
 * dOpInf_projection).  Symmetric eigendecomposition of D (k x k FP64, ldd), leading
 * r_cap eigenpairs in descending order; sign of each eigenvector: its largest-magnitude
 * entry is positive.  The energy denominator is trace(D).
 *
 * r_fixed > 0: r = r_fixed; otherwise r = the smallest r with
 *   sum_{i<=r} lambda_i / trace(D) > energy_target (strict), which must be <= r_cap.
 * r_cap        number of eigenpairs computed and of rows of Qhat (1 <= r_cap <= k).
 * eigvals      out, r_cap doubles, descending.
 * Tr           out, k x r_cap (ld k): T = U Lambda^{-1/2} (columns for lambda_i > 0).
 * Qhat         out, r_cap x k (ld r_cap): Qhat = T^T D; column t is the reduced snapshot t.
 *              The Qhat of any r <= r_cap is its leading r rows.
 * r_out, trace_out  host, the chosen r and trace(D).
 * Synchronises the stream (r is returned on the host).  Returns DOPINF_E_RANK if
 * lambda_r <= 0 or the energy target is not reached within r_cap.  Limits: k <= 25600 and
 * r_cap <= 8532 (the eigenvector and its re-orthogonalisation coefficients are kept in
 * shared memory; DOPINF_E_UNSUPPORTED above).
 * Workspace: dopinf_reduce_workspace(k, r_cap) bytes.
 * ------------------------------------------------------------------------------------ */
size_t dopinf_reduce_workspace(int64_t k, int r_cap);
int dopinf_reduce(const double* D, int64_t k, int64_t ldd, double energy_target, int r_fixed,
                  int r_cap, int* r_out, double* trace_out, double* eigvals, double* Tr,
                  double* Qhat, void* ws, size_t ws_bytes, void* stream);
/* The same without synchronisation (capturable into a CUDA graph): r and trace(D) are written
 * to the device words *r_dev and *trace_dev (r <= 0 where dopinf_reduce returns
 * DOPINF_E_RANK: 0 = energy target not reached, -r = lambda_r <= 0), and the failures OR
 * DOPINF_FLAG_RANK / DOPINF_FLAG_TIMEOUT into the device word *dev_flags (all required). */
int dopinf_reduce_async(const double* D, int64_t k, int64_t ldd, double energy_target, int r_fixed,
                        int r_cap, int* r_dev, double* trace_dev, double* eigvals, double* Tr,
                        double* Qhat, unsigned* dev_flags, void* ws, size_t ws_bytes, void* stream);
/* Tuning of dopinf_reduce: 1 (default) reduces D to tridiagonal form in one cooperative
 * launch with a grid barrier per column (where 3 k doubles of shared memory fit, k <= 8533,
 * and the device supports cooperative launches); 0 uses three launches per column.  Both
 * give the same bits.  If the grid barrier waits longer than 2 s, dopinf_reduce returns
 * DOPINF_E_TIMEOUT.  Other values only query.  Returns the previous value.  Process-wide. */
int dopinf_tune_reduce_coop(int on);

/* ------------------------------------------------------------------------------------
 * Step IV: quadratic OpInf with the (r, beta1, beta2) grid search (eqs. OpInf_reg,
 * OpInf_data_matrices_discrete; the training error and growth criterion of Step IV).
 *
 * Qhat       r_max x k reduced data (ld ldqh >= r_max), column t = snapshot t.
 * r_list     host, n_r reduced dimensions (1 <= r <= r_max, r <= 92 (DOPINF_E_UNSUPPORTED
 *            above); k-1 (discrete) or k-2 (continuous) rows of data are used).
 * beta1, beta2  host, n_b1 and n_b2 regularisation values.
 * Candidates are numbered r-major, then beta1, then beta2:
 *   c = (ir * n_b1 + i1) * n_b2 + i2.
 * For each candidate: data matrix Dhat = [q, (q_i q_j)_{i<=j}, 1] over the training rows,
 * G = Dhat^T Dhat, B = Dhat^T Y, Cholesky solve of (G + diag(beta1 1_r, beta2 1_s,
 * beta1)) O^T = B (by block elimination of the quadratic unknowns, which do not depend on
 * beta1: the Cholesky factorisation of the symmetrically permuted matrix); rollout of n_steps states (initial state included) from Qhat[:, 0];
 * train_err = max_{t<k} ||q~_t - qhat_t|| / ||qhat_t||; growth = max_{t,i} |q~ - mu| /
 * max_{t<k,i} |qhat - mu| (mu = temporal mean of Qhat).  Valid iff the factorisation
 * succeeded, the rollout is finite and growth < max_growth.  A rollout stops early once
 * the candidate is certainly invalid (growth already >= max_growth or non-finite).
 *
 * mode, dt   DOPINF_DISCRETE, or DOPINF_CONTINUOUS_RK4 with snapshot spacing dt.
 * train_err, growth  out (device), n_cand doubles (+Inf for invalid candidates).
 * cand_status out (device), n_cand ints: 0 valid, 1 Cholesky breakdown, 2 non-finite,
 *            3 growth >= max_growth.
 * cand_steps optional out (device, NULL = not wanted), n_cand int64: the time steps each
 *            rollout advanced before it ended (n_steps - 1 for a valid candidate); the
 *            right-hand-side evaluations are that times 4 (RK4) or 1 (discrete).
 * best_out   host: best candidate index, -1 if none is valid.
 * O_best     out (device), r_max x (d_max) doubles, ld r_max: operators [A | H | c] of
 *            the best candidate (its r x d leading block), d = r + r(r+1)/2 + 1.
 * stage_ms   optional out (host, NULL = not wanted), 3 doubles: device time (CUDA events on
 *            the stream) of the data matrices and normal equations, of the regularised
 *            solves, and of the rollouts.
 * Synchronises the stream.  Returns DOPINF_E_NO_STABLE if no candidate is valid.
 * n_b1, n_b2 <= 64 (DOPINF_E_UNSUPPORTED above).
 * Workspace: dopinf_learn_workspace(...) bytes.
 * ------------------------------------------------------------------------------------ */
/* Tuning of the rollouts of r <= 32 (dopinf_learn, dopinf_learn_async, dopinf_rollout): rows
 * of O per CTA, 1, 2, 4 or 8 (default 4; raised where the cluster of ceil(r / rows) CTAs would
 * exceed 16 or cannot be resident); other values only query.  Returns the previous value.
 * Process-wide.  The results do not depend on it. */
int dopinf_tune_rollout_rows(int rows);
/* The same for the rollouts of 32 < r <= 92 (operator rows in shared memory): rows of O per
 * CTA, 3 to 8 (default 4; raised where the cluster would exceed 16 CTAs or cannot be
 * resident); other values only query.  Returns the previous value.  Process-wide.  The
 * results do not depend on it. */
int dopinf_tune_rollout_rows_large(int rows);
/* Solver of the regularised problems of dopinf_learn / dopinf_learn_async:
 * DOPINF_SOLVE_CHOLESKY (default): the normal equations G + diag(reg), by block elimination of
 *   the quadratic unknowns shared across beta1 (see dopinf_learn);
 * DOPINF_SOLVE_QR: without the normal equations, the least-squares solution of the stacked
 *   system [Dhat; diag(sqrt(reg))] O^T = [Y; 0] by Householder reflections (one CTA per
 *   candidate) and back substitution: the conditioning of the stacked matrix, the square root
 *   of the normal equations', at several times the cost; operators up to d = 1024 (r <= 44;
 *   DOPINF_E_UNSUPPORTED above).  A zero diagonal of R marks the candidate as status 1.
 * The workspace query reflects the solver set when it is called.  Other values only query.
 * Returns the previous value.  Process-wide. */
#define DOPINF_SOLVE_CHOLESKY 0
#define DOPINF_SOLVE_QR 1
int dopinf_tune_learn_solver(int solver);
/* Rollout arithmetic of dopinf_learn: DOPINF_ROLLOUT_FP64 (default, the paper's) or DOPINF_ROLLOUT_DW; other
 * values only query.  Returns the previous value.  Process-wide. */
int dopinf_tune_rollout_arith(int arith);
size_t dopinf_learn_workspace(int r_max, int64_t k, const int* r_list, int n_r, int n_b1,
                              int n_b2);
int dopinf_learn(const double* Qhat, int r_max, int64_t k, int64_t ldqh, const int* r_list,
                 int n_r, const double* beta1, int n_b1, const double* beta2, int n_b2,
                 int mode, double dt, int64_t n_steps, double max_growth, double* train_err,
                 double* growth, int* cand_status, int64_t* cand_steps, int* best_out,
                 double* O_best, double* stage_ms, void* ws, size_t ws_bytes, void* stream);

/* Every candidate's operators: after dopinf_learn or dopinf_learn_async has run with this grid
 * (k, r_list, n_b1, n_b2) and workspace, and until the workspace is reused, candidate cand's
 * O = [A | H | c] (r x d doubles, column-major, ld r, r = its reduced dimension) lies at this
 * byte offset from the start of the workspace.  Its contents are meaningful where the
 * candidate's Cholesky factorisation succeeded (cand_status != 1).  Host-only query;
 * (size_t)-1 for bad arguments. */
size_t dopinf_learn_operator_offset(int64_t k, const int* r_list, int n_r, int n_b1, int n_b2, int cand);

/* The same without synchronisation and without host copies (capturable into a CUDA graph;
 * the candidate tables are built on the device): best_dev (device int, required) receives the
 * best index (-1 if none is valid, which also ORs DOPINF_FLAG_NO_STABLE into the device word
 * *dev_flags, required), O_best receives its operators.  n_b1, n_b2 <= 64. */
int dopinf_learn_async(const double* Qhat, int r_max, int64_t k, int64_t ldqh, const int* r_list,
                       int n_r, const double* beta1, int n_b1, const double* beta2, int n_b2,
                       int mode, double dt, int64_t n_steps, double max_growth, double* train_err,
                       double* growth, int* cand_status, int64_t* cand_steps, int* best_dev,
                       double* O_best, unsigned* dev_flags, void* ws, size_t ws_bytes,
                       void* stream);

/* ------------------------------------------------------------------------------------
 * Rollout of one quadratic ROM (eq. ROM_quad_time_discrete, or RK4 on
 * eq. ROM_quad_time_cont): O is r x d (ld ldo >= r), d = r + r(r+1)/2 + 1, columns
 * [A | H | c] with H's columns ordered (i, j), i <= j, i-major.  q0 has r entries.
 * Qtilde out, n_steps x r row-major (row t = state t, row 0 = q0).  finite out (device
 * int): 1 if every state is finite.  No workspace.
 * ------------------------------------------------------------------------------------ */
int dopinf_rollout(const double* O, int r, int64_t ldo, const double* q0, int64_t n_steps,
                   int mode, double dt, double* Qtilde, int* finite, void* stream);

/* ------------------------------------------------------------------------------------
 * Step V (Section 3.6): the reduced solution in the original coordinates at chosen rows.
 * V = Q[rows, :] T_r (rows of the POD basis, eq. MoS_POD_basis, from the transformed
 * snapshots Q of Step II), then X[j, t] = scale(row_j) * (V[j, :] Qtilde[:, t]) + mean(row_j),
 * the inverse of Step II's transform.  FP64 throughout.
 *
 * Q            n x k transformed snapshots (dtype, ld ldq >= n), as dopinf_transform left them.
 * Tr           k x r (ld ldt >= k), from dopinf_reduce (its first r columns).
 * Qtilde       r x n_t (ld ldqt >= r): column t = reduced state t, e.g. a dopinf_rollout
 *              trajectory (n_t x r row-major is this layout with ldqt = r).
 * rows         device, n_rows row indices in [0, n) (an index outside gives a NaN row of X), or
 *              NULL for rows 0 .. n_rows - 1 (n_rows <= n).
 * row_mean     optional (NULL: centring not undone), n doubles from dopinf_transform.
 * var_scale    optional (NULL: scaling not undone), n_vars doubles from dopinf_transform, with
 *              var_row_offsets (host, n_vars + 1, as for dopinf_transform; also used by row_mean
 *              when given, else rows of one variable).
 * X            out, n_rows x n_t column-major (ld ldx >= n_rows).
 * Asynchronous.  Workspace: dopinf_lift_workspace(n_rows, r) bytes (the rows of V).
 * ------------------------------------------------------------------------------------ */
size_t dopinf_lift_workspace(int64_t n_rows, int r);
int dopinf_lift(const void* Q, int dtype, int64_t n, int64_t k, int64_t ldq, const double* Tr, int64_t ldt, int r,
                const double* Qtilde, int64_t ldqt, int64_t n_t, const int64_t* rows, int64_t n_rows,
                const double* row_mean, const double* var_scale, int n_vars, const int64_t* var_row_offsets,
                double* X, int64_t ldx, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------
 * Learned proposal of (beta1, beta2, r).  The paper picks (beta1, beta2) by the grid search
 * of Section 3.5 and r by the retained energy of eq. ret_energy; this network proposes the
 * grid indices from statistics of the reduced data, and the grid search stays its fallback.
 * Network: 64 -> 256 -> 256 -> 256 -> H (GELU, exact erf form), H = head_sizes[0] +
 * head_sizes[1] + head_sizes[2] (beta1 index, beta2 index, r index).  Parameters: FP32,
 * flat [W1 (256 x 64 row-major), b1, W2 (256 x 256), b2, W3, b3, W4 (H x 256), b4]; weights are
 * rounded to BF16 (nearest even) where used; FP32 activations and accumulation.
 * ------------------------------------------------------------------------------------ */
/* The 64 features of one reduced system, in FP32 (device, 64 floats):
 *   f[0:32]  log10(max(lambda_i / lambda_1, 1e-30)), i = 2..33 (-30 if absent);
 *   f[32:36] log10(max(1 - sum_{i<=r} lambda_i / trace, 1e-30)), r = 5, 10, 20, 30;
 *   f[36:52] log10(rms_t(q_j[t+1] - q_j[t]) / rms_t(q_j[t])), modes j = 0..15 (0 if absent);
 *   f[52:63] mean(q_j^4) / mean(q_j^2)^2 - 1.5, modes j = 0..10 (0 if absent);
 *   f[63]    log10(k).
 * eigvals: device, n_eig descending eigenvalues; trace > 0 (host); Qhat: r_max x k, ld ldqh. */
int dopinf_proposal_features(const double* eigvals, int n_eig, double trace, const double* Qhat, int r_max,
                             int64_t k, int64_t ldqh, float* features, void* stream);
size_t dopinf_mlp_param_count(int n_out);
size_t dopinf_mlp_workspace(int batch, int n_out);
/* logits (device, batch x n_out row-major) of X (device, batch x 64 row-major). */
int dopinf_mlp_forward(const float* params, int n_out, const float* X, int batch, float* logits, void* ws,
                       size_t ws_bytes, void* stream);
/* One training step: forward, mean over the batch of the summed per-head softmax
 * cross-entropies (loss, device float, optional), backward, and (lr > 0) an Adam update
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with step >= 1) of params with moments
 * adam_m, adam_v (device, param_count floats each).  labels: device, batch x 3 ints.
 * grad_out (optional, device, param_count floats) receives the gradient.  head_sizes: host. */
int dopinf_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr, const int* head_sizes,
                          const float* X, const int* labels, int batch, float* loss, float* grad_out, void* ws,
                          size_t ws_bytes, void* stream);

/* Input standardisation of the network (the training set's statistics) and the ranking of the
 * grid candidates by the network's output.
 * dopinf_mlp_feature_stats: mu, sd (device, 64 doubles each) = per-feature mean and sample
 *   standard deviation (ddof = 1, floored at 1e-6) of X (device, batch x 64 FP32, row-major).
 * dopinf_mlp_standardize: Xs = fp32((X - mu) / sd) per feature (the arithmetic in FP64).
 * dopinf_mlp_rank: for each row of logits (device, batch x (h1 + h2 + h3), the three heads of
 *   dopinf_mlp_forward), the `top` candidates (i1, i2, i3) with the highest joint
 *   log-probability log softmax_1(i1) + log softmax_2(i2) + log softmax_3(i3) (FP64), the lowest
 *   flat index (i1 h2 + i2) h3 + i3 first on ties: ranked (device, batch x top x 3 ints; -1 past
 *   the h1 h2 h3 candidates), score (optional, device, batch x top doubles).  h1 h2 h3 <= 4096,
 *   top <= 64 (DOPINF_E_UNSUPPORTED above).  head_sizes: host, 3 ints.  All asynchronous. */
int dopinf_mlp_feature_stats(const float* X, int batch, double* mu, double* sd, void* stream);
int dopinf_mlp_standardize(const float* X, int batch, const double* mu, const double* sd, float* Xs, void* stream);
int dopinf_mlp_rank(const float* logits, int batch, const int* head_sizes, int top, int* ranked, double* score,
                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DOPINF_H */
