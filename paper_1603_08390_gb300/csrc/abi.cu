// Error reporting and version of the C ABI (see include/genie.h).
#include <cstdio>
#include <string>

#include "internal.h"

namespace {
thread_local std::string g_last_error;
}

namespace genie {

genie_status fail(genie_status status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

genie_status fail_cuda(cudaError_t err, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
  g_last_error = msg;
  if (err == cudaErrorMemoryAllocation) return GENIE_ERR_OUT_OF_MEMORY;
  return GENIE_ERR_CUDA;
}

}  // namespace genie

extern "C" const char* genie_last_error(void) { return g_last_error.c_str(); }

extern "C" int genie_version(void) { return 100; }
