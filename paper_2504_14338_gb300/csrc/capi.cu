// Status strings of the C ABI and the last CUDA error met.
#include "common.cuh"
#include <stdio.h>

namespace dopinf {
namespace {
thread_local char g_last_error[256] = "";
}
void set_last_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
}

namespace {
__global__ void flag_if_set_kernel(const unsigned* err, unsigned* flags, unsigned bits) {
  if (*err) atomicOr(flags, bits);
}
__global__ void flag_status_kernel(const unsigned* err, unsigned* flags) {
  const unsigned e = *err;
  if (e & ~kErrNonfinite) atomicOr(flags, DOPINF_FLAG_TIMEOUT);
  if (e & kErrNonfinite) atomicOr(flags, DOPINF_FLAG_NONFINITE);
}
int g_test_stall = 0;
}  // namespace

int test_stall() { return g_test_stall; }

void flag_if_set(const unsigned* err, unsigned* flags, unsigned bits, cudaStream_t st) {
  flag_if_set_kernel<<<1, 1, 0, st>>>(err, flags, bits);
}

int finish_timeout(const unsigned* err, unsigned* dev_flags, cudaStream_t st) {
  if (dev_flags) {
    flag_status_kernel<<<1, 1, 0, st>>>(err, dev_flags);
    return launch_status();
  }
  unsigned e = 0;
  DOPINF_CUDA(cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  DOPINF_CUDA(cudaStreamSynchronize(st));
  if (e & ~kErrNonfinite) {
    set_last_error("a bounded wait inside a tensor-core kernel", cudaErrorTimeout);
    return DOPINF_E_TIMEOUT;
  }
  return (e & kErrNonfinite) ? DOPINF_E_NONFINITE : DOPINF_OK;
}
}  // namespace dopinf

DOPINF_API const char* dopinf_last_error(void) { return dopinf::g_last_error; }

DOPINF_API int dopinf_test_expire_waits(int which) {
  const int prev = dopinf::g_test_stall;
  if (which >= 0) dopinf::g_test_stall = which & (dopinf::kStallGridBarrier | dopinf::kStallTensorGram);
  return prev;
}

DOPINF_API const char* dopinf_status_string(int status) {
  switch (status) {
    case DOPINF_OK: return "ok";
    case DOPINF_E_ARG: return "invalid argument";
    case DOPINF_E_CUDA: return "CUDA runtime error";
    case DOPINF_E_NONFINITE: return "non-finite value in the data";
    case DOPINF_E_RANK: return "reduced dimension exceeds the numerical rank or energy target not reached";
    case DOPINF_E_NO_STABLE: return "no finite, bounded regularisation candidate";
    case DOPINF_E_TIMEOUT: return "a bounded wait inside a GPU kernel expired";
    case DOPINF_E_UNSUPPORTED: return "request not supported by this build";
    default: return "unknown status";
  }
}

DOPINF_API int64_t dopinf_tune_gram_chunk(int64_t rows) { return dopinf::gram_tc_set_chunk_rows(rows); }
