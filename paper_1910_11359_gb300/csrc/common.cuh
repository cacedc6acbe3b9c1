// Shared device/host helpers for the iPEPS CTMRG / simple-update library (sm_103a).
// Complex numbers are double2 (x = real, y = imaginary), row-major storage throughout.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

namespace ipeps {

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ cplx cmulc(cplx a, cplx b) {
  return cmk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfmac(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

// Device-side error word: kernels that detect a problem (bad size, non-finite value, iteration
// cap) OR a code in here instead of trapping; the host reads it after synchronising.
enum DevErr : unsigned {
  DEV_OK = 0u,
  DEV_NONFINITE = 1u,
  DEV_JACOBI_CAP = 2u,
  DEV_BAD_SIZE = 4u,
  DEV_TIMEOUT = 8u,
};

}  // namespace ipeps

#define IPEPS_CUDA_TRY(expr)                                                             \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess) {                                                             \
      return ::ipeps::cuda_fail(_e, #expr, __FILE__, __LINE__);                          \
    }                                                                                    \
  } while (0)

namespace ipeps {
// Records a CUDA failure in a thread-local message buffer; returns the library's ECUDA code.
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
const char* thread_error_message();
void set_thread_error(const std::string& msg);
}  // namespace ipeps
