// Learned proposal of (beta1, beta2, r): features of a reduced system and a small MLP
// (64 -> 256 -> 256 -> 256 -> H, GELU, three softmax heads) with its forward pass, backward
// pass and Adam update, all on the GPU.  The paper chooses (beta1, beta2) by grid search
// (Section 3.5) and r by retained energy (Section 3.4); the network proposes both from
// statistics of the reduced data, and the grid search remains the fallback.
//
// Weights are FP32 master copies rounded to BF16 (round-to-nearest-even) where they are
// used; activations and accumulation are FP32.  The layers are small (B x 256 x 256), so a
// tiled SIMT GEMM serves every product: C = op(A) op(B) with optional bias and GELU epilogue.
#include "common.cuh"
#include <cuda_bf16.h>
#include <math.h>

namespace dopinf {
namespace {

constexpr int MLP_IN = 64, MLP_HID = 256;
constexpr int GT = 64, GK = 16;  // GEMM tile and K step

struct GemmArgs {
  const float* A;
  const float* B;
  float* C;        // output (Z when gelu)
  float* Cact;     // GELU(Z) when gelu
  const float* bias;
  int M, N, K;
  int lda, ldb, ldc;
  int transA, transB;  // A(m, k) = transA ? A[k * lda + m] : A[m * lda + k]; B(k, n) likewise
  int bf16B;           // round B to BF16 on load (weights)
  int gelu;
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
  __shared__ float As[GK][GT + 1];
  __shared__ float Bs[GK][GT + 1];
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e % GK, mm = e / GK;
      const int m = m0 + mm, k = k0 + kk;
      float va = 0.f;
      if (m < g.M && k < g.K) va = g.transA ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
      As[kk][mm] = va;
      const int n = n0 + mm;
      float vb = 0.f;
      if (n < g.N && k < g.K) vb = g.transB ? g.B[(size_t)n * g.ldb + k] : g.B[(size_t)k * g.ldb + n];
      Bs[kk][mm] = g.bf16B ? bf16r(vb) : vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= g.M || n >= g.N) continue;
      float z = acc[i][j] + (g.bias ? g.bias[n] : 0.f);
      g.C[(size_t)m * g.ldc + n] = z;
      if (g.gelu) g.Cact[(size_t)m * g.ldc + n] = gelu_f(z);
    }
}

int gemm(const GemmArgs& g, cudaStream_t st) {
  dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT);
  gemm_kernel<<<grid, 256, 0, st>>>(g);
  return launch_status();
}

// dZ = dA * gelu'(Z), elementwise
__global__ void gelu_backward(const float* __restrict__ dA, const float* __restrict__ Z, float* __restrict__ dZ, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dZ[i] = dA[i] * gelu_grad_f(Z[i]);
}

// db[o] = sum_b dZ[b, o] (fixed order)
__global__ void bias_grad(const float* __restrict__ dZ, int B, int O, float* __restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(size_t)b * O + o];
  db[o] = s;
}

// Softmax cross-entropy of three heads: per-sample gradient (softmax - onehot) / B, and the
// mean loss (one block, fixed-order reduction).  One thread per sample, strided.
__global__ void __launch_bounds__(256) heads_ce(const float* __restrict__ logits, const int* __restrict__ labels, int B,
                                                int H, int h0, int h1, int h2, float* __restrict__ dlogits,
                                                float* __restrict__ loss) {
  __shared__ float sh[256];
  const int hs[3] = {h0, h1, h2};
  float part = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int off = 0;
    for (int h = 0; h < 3; ++h) {
      const float* z = logits + (size_t)b * H + off;
      float mx = -INFINITY;
      for (int j = 0; j < hs[h]; ++j) mx = fmaxf(mx, z[j]);
      float se = 0.f;
      for (int j = 0; j < hs[h]; ++j) se += expf(z[j] - mx);
      const float lse = mx + logf(se);
      const int y = labels[b * 3 + h];
      part += lse - z[y];
      for (int j = 0; j < hs[h]; ++j)
        dlogits[(size_t)b * H + off + j] = (expf(z[j] - lse) - (j == y ? 1.f : 0.f)) / (float)B;
      off += hs[h];
    }
  }
  sh[threadIdx.x] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)blockDim.x; ++i) s += sh[i];
    *loss = s / (float)B;
  }
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Features of one reduced system (definitions in the proposal oracle's header): one block.
__global__ void __launch_bounds__(256) features_kernel(const double* __restrict__ lam, int n_eig, double trace,
                                                       const double* __restrict__ Qhat, int r_max, int64_t k,
                                                       int64_t ldqh, float* __restrict__ f) {
  __shared__ double sa[256], sb[256], sc[256];
  const int tid = threadIdx.x;
  if (tid < 32) {
    const int j = tid + 1;
    f[tid] = j < n_eig ? (float)log10(fmax(lam[j] / lam[0], 1e-30)) : -30.0f;
  }
  if (tid == 32) {
    const int rs[4] = {5, 10, 20, 30};
    for (int c = 0; c < 4; ++c) {
      double cum = 0.0;
      for (int i = 0; i < rs[c] && i < n_eig; ++i) cum += lam[i];
      f[32 + c] = (float)log10(fmax(1.0 - cum / trace, 1e-30));
    }
    f[63] = (float)log10((double)k);
  }
  for (int j = 0; j < 16; ++j) {
    double dd = 0.0, q2 = 0.0, q4 = 0.0;
    if (j < r_max) {
      for (int64_t t = tid; t < k; t += blockDim.x) {
        const double q = Qhat[j + t * ldqh];
        q2 += q * q;
        q4 += q * q * q * q;
        if (t + 1 < k) {
          const double d = Qhat[j + (t + 1) * ldqh] - q;
          dd += d * d;
        }
      }
    }
    sa[tid] = dd;
    sb[tid] = q2;
    sc[tid] = q4;
    __syncthreads();
    if (tid == 0 && j < r_max) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int i = 0; i < (int)blockDim.x; ++i) {
        a += sa[i];
        b += sb[i];
        c += sc[i];
      }
      const double ms = b / (double)k;
      f[36 + j] = (float)log10(sqrt(a / (double)(k - 1)) / sqrt(ms));
      if (j < 11) f[52 + j] = (float)(c / (double)k / (ms * ms) - 1.5);
    } else if (tid == 0) {
      f[36 + j] = 0.0f;
      if (j < 11) f[52 + j] = 0.0f;
    }
    __syncthreads();
  }
}

struct MlpLayout {
  size_t off_w[4], off_b[4], count;
  int in[4], out[4];
};

MlpLayout mlp_layout(int n_out) {
  MlpLayout L;
  const int ins[4] = {MLP_IN, MLP_HID, MLP_HID, MLP_HID};
  const int outs[4] = {MLP_HID, MLP_HID, MLP_HID, n_out};
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    L.in[l] = ins[l];
    L.out[l] = outs[l];
    L.off_w[l] = off;
    off += (size_t)outs[l] * ins[l];
    L.off_b[l] = off;
    off += outs[l];
  }
  L.count = off;
  return L;
}

struct MlpWs {
  float *z[4], *a[4], *dA, *dZ, *grad, *loss;
  size_t used;
};

MlpWs carve_mlp(void* base, int B, int n_out) {
  Carver c(base);
  MlpWs w;
  const int outs[4] = {MLP_HID, MLP_HID, MLP_HID, n_out};
  for (int l = 0; l < 4; ++l) {
    w.z[l] = c.take<float>((size_t)B * outs[l]);
    w.a[l] = c.take<float>((size_t)B * outs[l]);
  }
  const int wmax = MLP_HID > n_out ? MLP_HID : n_out;
  w.dA = c.take<float>((size_t)B * wmax);
  w.dZ = c.take<float>((size_t)B * wmax);
  w.grad = c.take<float>(mlp_layout(n_out).count);
  w.loss = c.take<float>(1);
  w.used = c.used;
  return w;
}

int mlp_forward_impl(const float* params, int n_out, const float* X, int B, const MlpWs& w, cudaStream_t st) {
  const MlpLayout L = mlp_layout(n_out);
  const float* a = X;
  for (int l = 0; l < 4; ++l) {
    GemmArgs g = {};
    g.A = a;
    g.lda = L.in[l];
    g.B = params + L.off_w[l];
    g.ldb = L.in[l];
    g.transB = 1;
    g.bf16B = 1;
    g.bias = params + L.off_b[l];
    g.C = w.z[l];
    g.Cact = w.a[l];
    g.ldc = L.out[l];
    g.M = B;
    g.N = L.out[l];
    g.K = L.in[l];
    g.gelu = l < 3;
    DOPINF_TRY(gemm(g, st));
    a = l < 3 ? w.a[l] : w.z[l];
  }
  return DOPINF_OK;
}

// Per-feature mean and sample standard deviation (ddof = 1, floored at 1e-6) of a training
// set X (batch x 64, row-major), FP64: one CTA per feature, each thread a strided sequence of
// rows, then a fixed tree.
__global__ void __launch_bounds__(256) feature_stats_kernel(const float* __restrict__ X, int batch,
                                                            double* __restrict__ mu, double* __restrict__ sd) {
  __shared__ double sh[256];
  const int f = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) s += (double)X[(size_t)b * 64 + f];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  const double m = sh[0] / (double)batch;
  __syncthreads();
  double q = 0.0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const double c = (double)X[(size_t)b * 64 + f] - m;
    q += c * c;
  }
  sh[threadIdx.x] = q;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mu[f] = m;
    const double v = batch > 1 ? sqrt(sh[0] / (double)(batch - 1)) : 0.0;
    sd[f] = v > 1e-6 ? v : 1e-6;
  }
}

// Xs = fp32((x - mu) / sd), the subtraction and division in FP64.
__global__ void standardise_kernel(const float* __restrict__ X, int n, const double* __restrict__ mu,
                                   const double* __restrict__ sd, float* __restrict__ Xs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int f = e % 64;
  Xs[e] = (float)(((double)X[e] - mu[f]) / sd[f]);
}

constexpr int kRankMax = 4096;  // candidates of the joint ranking (h1 h2 h3)

// One CTA per row of logits: per-head log-softmax in FP64, the joint log-probability of every
// (i1, i2, i3), and `top` rounds of a block argmax (highest score, lowest flat index on ties).
__global__ void __launch_bounds__(256) rank_kernel(const float* __restrict__ logits, int n_out, int h1, int h2, int h3,
                                                   int top, int* __restrict__ ranked, double* __restrict__ score) {
  __shared__ double lse[3];
  __shared__ double joint[kRankMax];
  __shared__ double bv[256];
  __shared__ int bi[256];
  const float* z = logits + (size_t)blockIdx.x * n_out;
  const int hs[3] = {h1, h2, h3}, ho[3] = {0, h1, h1 + h2};
  if (threadIdx.x < 3) {
    const int h = threadIdx.x;
    double m = -INFINITY;
    for (int i = 0; i < hs[h]; ++i) m = fmax(m, (double)z[ho[h] + i]);
    double s = 0.0;
    for (int i = 0; i < hs[h]; ++i) s += exp((double)z[ho[h] + i] - m);
    lse[h] = m + log(s);
  }
  __syncthreads();
  const int n = h1 * h2 * h3;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const int i1 = c / (h2 * h3), i2 = (c / h3) % h2, i3 = c % h3;
    joint[c] = ((double)z[i1] - lse[0]) + ((double)z[h1 + i2] - lse[1]) + ((double)z[h1 + h2 + i3] - lse[2]);
  }
  __syncthreads();
  for (int t = 0; t < top; ++t) {
    double v = -INFINITY;
    int idx = 0x7fffffff;
    for (int c = threadIdx.x; c < n; c += blockDim.x)
      if (joint[c] > v || (joint[c] == v && c < idx)) {
        v = joint[c];
        idx = c;
      }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) {
        const double v2 = bv[threadIdx.x + h];
        const int i2 = bi[threadIdx.x + h];
        if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
          bv[threadIdx.x] = v2;
          bi[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int c = bi[0];
      int* o = ranked + ((size_t)blockIdx.x * top + t) * 3;
      const bool ok = c < n;
      o[0] = ok ? c / (h2 * h3) : -1;
      o[1] = ok ? (c / h3) % h2 : -1;
      o[2] = ok ? c % h3 : -1;
      if (score) score[(size_t)blockIdx.x * top + t] = ok ? bv[0] : -INFINITY;
      if (ok) joint[c] = NAN;  // excluded from the next rounds: NaN wins no comparison
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace dopinf

using namespace dopinf;

DOPINF_API int dopinf_mlp_feature_stats(const float* X, int batch, double* mu, double* sd, void* stream) {
  if (!X || batch < 1 || !mu || !sd) return DOPINF_E_ARG;
  feature_stats_kernel<<<64, 256, 0, as_stream(stream)>>>(X, batch, mu, sd);
  return launch_status();
}

DOPINF_API int dopinf_mlp_standardize(const float* X, int batch, const double* mu, const double* sd, float* Xs,
                                      void* stream) {
  if (!X || batch < 1 || !mu || !sd || !Xs || batch > (1 << 24)) return DOPINF_E_ARG;
  const int n = batch * 64;
  standardise_kernel<<<(n + 255) / 256, 256, 0, as_stream(stream)>>>(X, n, mu, sd, Xs);
  return launch_status();
}

DOPINF_API int dopinf_mlp_rank(const float* logits, int batch, const int* head_sizes, int top, int* ranked,
                               double* score, void* stream) {
  if (!logits || batch < 1 || !head_sizes || top < 1 || !ranked) return DOPINF_E_ARG;
  for (int h = 0; h < 3; ++h)
    if (head_sizes[h] < 1) return DOPINF_E_ARG;
  const int h1 = head_sizes[0], h2 = head_sizes[1], h3 = head_sizes[2];
  if ((int64_t)h1 * h2 * h3 > kRankMax || top > 64 || batch > 65535) return DOPINF_E_UNSUPPORTED;
  rank_kernel<<<batch, 256, 0, as_stream(stream)>>>(logits, h1 + h2 + h3, h1, h2, h3, top, ranked, score);
  return launch_status();
}

DOPINF_API size_t dopinf_mlp_param_count(int n_out) { return n_out > 0 ? mlp_layout(n_out).count : 0; }

DOPINF_API size_t dopinf_mlp_workspace(int batch, int n_out) {
  if (batch < 1 || n_out < 1) return 0;
  return carve_mlp(nullptr, batch, n_out).used;
}

DOPINF_API int dopinf_proposal_features(const double* eigvals, int n_eig, double trace, const double* Qhat, int r_max,
                                        int64_t k, int64_t ldqh, float* features, void* stream) {
  if (!eigvals || n_eig < 1 || !Qhat || r_max < 1 || k < 2 || ldqh < r_max || !features || !(trace > 0.0))
    return DOPINF_E_ARG;
  features_kernel<<<1, 256, 0, as_stream(stream)>>>(eigvals, n_eig, trace, Qhat, r_max, k, ldqh, features);
  return launch_status();
}

DOPINF_API int dopinf_mlp_forward(const float* params, int n_out, const float* X, int batch, float* logits, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!params || n_out < 1 || !X || batch < 1 || !logits) return DOPINF_E_ARG;
  if (!ws || ws_bytes < dopinf_mlp_workspace(batch, n_out) || misaligned(ws)) return DOPINF_E_ARG;
  cudaStream_t st = as_stream(stream);
  MlpWs w = carve_mlp(ws, batch, n_out);
  DOPINF_TRY(mlp_forward_impl(params, n_out, X, batch, w, st));
  return cuda_status(cudaMemcpyAsync(logits, w.z[3], sizeof(float) * batch * n_out, cudaMemcpyDeviceToDevice, st));
}

DOPINF_API int dopinf_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr,
                                     const int* head_sizes, const float* X, const int* labels, int batch, float* loss,
                                     float* grad_out, void* ws, size_t ws_bytes, void* stream) {
  if (!params || !adam_m || !adam_v || step < 1 || !(lr >= 0.f) || !head_sizes || !X || !labels || batch < 1 ||
      batch > 65535)
    return DOPINF_E_ARG;
  for (int h = 0; h < 3; ++h)
    if (head_sizes[h] < 1) return DOPINF_E_ARG;
  const int n_out = head_sizes[0] + head_sizes[1] + head_sizes[2];
  if (!ws || ws_bytes < dopinf_mlp_workspace(batch, n_out) || misaligned(ws)) return DOPINF_E_ARG;
  cudaStream_t st = as_stream(stream);
  MlpWs w = carve_mlp(ws, batch, n_out);
  const MlpLayout L = mlp_layout(n_out);
  DOPINF_TRY(mlp_forward_impl(params, n_out, X, batch, w, st));
  heads_ce<<<1, 256, 0, st>>>(w.z[3], labels, batch, n_out, head_sizes[0], head_sizes[1], head_sizes[2], w.dZ,
                              loss ? loss : w.loss);
  DOPINF_TRY(launch_status());
  for (int l = 3; l >= 0; --l) {
    const int O = L.out[l], I = L.in[l];
    if (l < 3) {
      const int n = batch * O;
      gelu_backward<<<(n + 255) / 256, 256, 0, st>>>(w.dA, w.z[l], w.dZ, n);
      DOPINF_TRY(launch_status());
    }
    const float* in = l > 0 ? w.a[l - 1] : X;
    GemmArgs gw = {};  // dW = dZ^T in  (O x I)
    gw.A = w.dZ;
    gw.lda = O;
    gw.transA = 1;
    gw.B = in;
    gw.ldb = I;
    gw.C = w.grad + L.off_w[l];
    gw.ldc = I;
    gw.M = O;
    gw.N = I;
    gw.K = batch;
    DOPINF_TRY(gemm(gw, st));
    bias_grad<<<(O + 255) / 256, 256, 0, st>>>(w.dZ, batch, O, w.grad + L.off_b[l]);
    DOPINF_TRY(launch_status());
    if (l > 0) {
      GemmArgs gx = {};  // dA_prev = dZ W  (B x I), weights rounded as in the forward pass
      gx.A = w.dZ;
      gx.lda = O;
      gx.B = params + L.off_w[l];
      gx.ldb = I;
      gx.bf16B = 1;
      gx.C = w.dA;
      gx.ldc = I;
      gx.M = batch;
      gx.N = I;
      gx.K = O;
      DOPINF_TRY(gemm(gx, st));
    }
  }
  if (grad_out)
    DOPINF_CUDA(cudaMemcpyAsync(grad_out, w.grad, sizeof(float) * L.count, cudaMemcpyDeviceToDevice, st));
  if (lr > 0.f) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(unsigned)((L.count + 255) / 256), 256, 0, st>>>(params, adam_m, adam_v, w.grad, (int64_t)L.count, lr,
                                                                   b1, b2, 1e-8f, c1, c2);
    DOPINF_TRY(launch_status());
  }
  return DOPINF_OK;
}
