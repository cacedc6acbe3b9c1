// Thread-local error text for the C-ABI (status codes cross the boundary, text stays here).
#include <string>

#include "common.cuh"

namespace ipeps {

static thread_local std::string g_msg;

void set_thread_error(const std::string& msg) { g_msg = msg; }
const char* thread_error_message() { return g_msg.c_str(); }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what,
           file, line);
  g_msg = buf;
  return 5;  // IPEPS_ECUDA
}

}  // namespace ipeps
