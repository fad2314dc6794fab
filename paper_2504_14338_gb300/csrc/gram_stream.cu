// Gram matrix of a snapshot matrix that stays in host memory (larger than the device, or
// simply not uploaded whole): the row blocks of the paper's partitioned Gram (Section 3.4,
// eq. mos_partitioned, D = sum_i Q_i^T Q_i) are copied one after another into two device
// buffers taken from the caller's workspace, on a copy stream of the library's own, while the
// Gram of the previous block accumulates into D on the caller's stream.  Block c's upload
// waits for the Gram that last read its buffer (block c - 2); block c's Gram waits for its
// upload.  Any Gram mode; the tensor-core modes report through a device flag word that is
// read once at the end.
#include "common.cuh"

#include <mutex>

namespace dopinf {
namespace {

struct StreamWs {
  void* buf[2];
  unsigned* flags;
  void* gram_ws;
  size_t gram_bytes, used;
};

StreamWs carve_stream(void* base, int64_t chunk_rows, int64_t k, int dtype, int mode) {
  const size_t es = dtype == DOPINF_F64 ? 8 : 4;
  Carver c(base);
  StreamWs w;
  w.buf[0] = c.take<char>((size_t)chunk_rows * k * es);
  w.buf[1] = c.take<char>((size_t)chunk_rows * k * es);
  w.flags = c.take<unsigned>(1);
  w.gram_bytes = dopinf_gram_workspace(chunk_rows, k, dtype, mode);
  w.gram_ws = c.take<char>(w.gram_bytes);
  w.used = c.used;
  return w;
}

// One copy stream and four events per device, made on first use.
struct CopyRes {
  cudaStream_t copy = nullptr;
  cudaEvent_t uploaded[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
};
constexpr int kMaxDev = 128;
CopyRes g_res[kMaxDev];
std::mutex g_res_mu;

int copy_resources(CopyRes** out) {
  int dev = 0;
  DOPINF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return DOPINF_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_res_mu);
  CopyRes& r = g_res[dev];
  if (!r.copy) {
    DOPINF_CUDA(cudaStreamCreateWithFlags(&r.copy, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      DOPINF_CUDA(cudaEventCreateWithFlags(&r.uploaded[b], cudaEventDisableTiming));
      DOPINF_CUDA(cudaEventCreateWithFlags(&r.done[b], cudaEventDisableTiming));
    }
  }
  *out = &r;
  return DOPINF_OK;
}

}  // namespace
}  // namespace dopinf

using namespace dopinf;

DOPINF_API size_t dopinf_gram_host_workspace(int64_t chunk_rows, int64_t k, int dtype, int mode) {
  if (chunk_rows < 1 || k < 1 || (dtype != DOPINF_F64 && dtype != DOPINF_F32)) return 0;
  if (dopinf_gram_workspace(chunk_rows, k, dtype, mode) == 0) return 0;
  return carve_stream(nullptr, chunk_rows, k, dtype, mode).used;
}

DOPINF_API int dopinf_gram_host(const void* Q_host, int dtype, int64_t n, int64_t k, int64_t ldq, int mode,
                                int accumulate, double* D, int64_t ldd, int64_t chunk_rows, void* ws,
                                size_t ws_bytes, void* stream) {
  if (!Q_host || !D || n < 1 || k < 1 || ldq < n || ldd < k || chunk_rows < 1) return DOPINF_E_ARG;
  if (dtype != DOPINF_F64 && dtype != DOPINF_F32) return DOPINF_E_ARG;
  if (mode != DOPINF_GRAM_FP64 && mode != DOPINF_GRAM_BF16X4 && mode != DOPINF_GRAM_OZAKI_FP64)
    return DOPINF_E_UNSUPPORTED;
  if (chunk_rows > n) chunk_rows = n;
  const size_t need = dopinf_gram_host_workspace(chunk_rows, k, dtype, mode);
  if (!ws || need == 0 || ws_bytes < need || misaligned(ws)) return DOPINF_E_ARG;
  const StreamWs w = carve_stream(ws, chunk_rows, k, dtype, mode);
  CopyRes* res = nullptr;
  DOPINF_TRY(copy_resources(&res));
  cudaStream_t st = as_stream(stream);
  const size_t es = dtype == DOPINF_F64 ? 8 : 4;
  DOPINF_CUDA(cudaMemsetAsync(w.flags, 0, sizeof(unsigned), st));
  // the copy stream starts after everything the caller queued before this call (D, flags)
  DOPINF_CUDA(cudaEventRecord(res->done[0], st));
  DOPINF_CUDA(cudaEventRecord(res->done[1], st));
  const int64_t n_chunks = (n + chunk_rows - 1) / chunk_rows;
  for (int64_t c = 0; c < n_chunks; ++c) {
    const int b = (int)(c & 1);
    const int64_t a = c * chunk_rows;
    const int64_t rows = n - a < chunk_rows ? n - a : chunk_rows;
    DOPINF_CUDA(cudaStreamWaitEvent(res->copy, res->done[b], 0));
    DOPINF_CUDA(cudaMemcpy2DAsync(w.buf[b], (size_t)rows * es, static_cast<const char*>(Q_host) + (size_t)a * es,
                                  (size_t)ldq * es, (size_t)rows * es, (size_t)k, cudaMemcpyHostToDevice,
                                  res->copy));
    DOPINF_CUDA(cudaEventRecord(res->uploaded[b], res->copy));
    DOPINF_CUDA(cudaStreamWaitEvent(st, res->uploaded[b], 0));
    DOPINF_TRY(dopinf_gram_async(w.buf[b], dtype, rows, k, rows, mode, (c > 0 || accumulate) ? 1 : 0, D, ldd, w.flags,
                                 w.gram_ws, w.gram_bytes, stream));
    DOPINF_CUDA(cudaEventRecord(res->done[b], st));
  }
  unsigned f = 0;
  DOPINF_CUDA(cudaMemcpyAsync(&f, w.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  DOPINF_CUDA(cudaStreamSynchronize(st));
  if (f & DOPINF_FLAG_TIMEOUT) return DOPINF_E_TIMEOUT;
  if (f & DOPINF_FLAG_NONFINITE) return DOPINF_E_NONFINITE;
  return DOPINF_OK;
}
