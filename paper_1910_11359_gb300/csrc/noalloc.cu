// Allocation-free variant of the batched Jacobi SVD entry point (ipeps_kernel_svd).
//
// Some callers cannot call cudaMalloc: code that runs while an application's own allocator owns the
// device memory pool, plug-ins handed only pre-allocated buffers, or hosts that forbid device
// allocation after start-up.  ipeps_kernel_svd allocates a small device buffer per call for its
// operand pointer tables and its error word; this variant keeps those in a fixed array in device
// global memory instead (g_noalloc_scratch below, kNoallocScratchBytes bytes, held by every GPU that
// loads the library until the process exits).  The caller still provides A, U, S, V.
//
// Host code must not use the array's name as a device address (on the host it is only a stand-in
// symbol).  The device address is obtained once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on that device; make that first call before any stream
// capture begins.  Every call shares the one array and leaves its contents behind; the error word is
// cleared at the start of each call.  Calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race on the array: serialise them.
#include <mutex>

#include "../../include/ipeps.h"
#include "../../include/ipeps_kernels.h"
#include "linalg.cuh"

namespace ipeps {
namespace {

constexpr int kNoallocMaxBatch = 1024;
constexpr size_t kTableOffset = 256;                       // pointer tables after the error word
constexpr size_t kNoallocScratchBytes = kTableOffset + 4 * kNoallocMaxBatch * sizeof(void*);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (set up on first use).
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
  if (dev < 0 || dev >= kMaxDevices) {
    set_thread_error("device index out of range for the allocation-free entry point");
    return IPEPS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    unsigned char* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return 0;
}

// Writes the operand pointer tables of `batch` contiguous problems into the scratch array and
// clears the error word.
__global__ void noalloc_tables_kernel(unsigned char* scratch, const cplx* A, cplx* U, double* S,
                                      cplx* V, int m, int n, int batch) {
  void** tab = reinterpret_cast<void**>(scratch + kTableOffset);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    tab[b] = (void*)(A + (size_t)b * m * n);
    tab[batch + b] = U ? (void*)(U + (size_t)b * m * n) : nullptr;
    tab[2 * batch + b] = (void*)(S + (size_t)b * n);
    tab[3 * batch + b] = V ? (void*)(V + (size_t)b * n * n) : nullptr;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<unsigned*>(scratch) = 0u;
}

}  // namespace
}  // namespace ipeps

using namespace ipeps;

extern "C" int ipeps_kernel_svd_noalloc(int m, int n, int batch, const double* A, double* U, double* S,
                                        double* V, double tol, int max_sweeps, int* sweeps_out,
                                        void* stream) {
  if (m < n || n < 1 || batch < 1 || !A || !S) {
    set_thread_error("bad svd arguments");
    return IPEPS_EINVAL;
  }
  if (batch > kNoallocMaxBatch) {
    set_thread_error("ipeps_kernel_svd_noalloc: batch exceeds the fixed scratch capacity of 1024 problems");
    return IPEPS_EINVAL;
  }
  if (!jacobi_svd_fits(m, n)) {
    set_thread_error("ipeps_kernel_svd_noalloc: the m x n block does not fit in the shared memory of "
                     "one cluster (ipeps_kernel_svd serves such blocks with an allocated column buffer)");
    return IPEPS_EUNSUPPORTED;
  }
  unsigned char* scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  noalloc_tables_kernel<<<(batch + 255) / 256, 256, 0, st>>>(scratch, (const cplx*)A, (cplx*)U, S,
                                                             (cplx*)V, m, n, batch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "noalloc tables", __FILE__, __LINE__);
  void** tab = reinterpret_cast<void**>(scratch + kTableOffset);
  unsigned* derr = reinterpret_cast<unsigned*>(scratch);
  SvdDesc d;
  d.m = m; d.n = n; d.batch = batch;
  d.A = (const cplx* const*)tab; d.lda = n;
  d.U = U ? (cplx* const*)(tab + batch) : nullptr; d.ldu = n;
  d.S = (double* const*)(tab + 2 * batch);
  d.V = V ? (cplx* const*)(tab + 3 * batch) : nullptr; d.ldv = n;
  d.tol = tol; d.max_sweeps = max_sweeps; d.err = derr; d.sweeps_out = sweeps_out; d.skip = nullptr;
  if (int rc = jacobi_svd(d, st)) return rc;
  unsigned herr = 0;
  e = cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "noalloc svd sync", __FILE__, __LINE__);
  if (herr & DEV_NONFINITE) { set_thread_error("non-finite input"); return IPEPS_ENAN; }
  if (herr & DEV_JACOBI_CAP) { set_thread_error("sweep limit reached"); return IPEPS_ENOCONV; }
  return 0;
}
