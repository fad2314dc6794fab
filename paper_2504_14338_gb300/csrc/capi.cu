// Status strings of the C ABI.
#include "common.cuh"

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
