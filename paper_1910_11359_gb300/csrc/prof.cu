// Launch accounting and optional per-class CUDA-event timing (see prof.cuh).
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/ipeps_kernels.h"
#include "common.cuh"
#include "prof.cuh"

namespace ipeps {

namespace {
const char* kNames[K_NCLASS] = {"zgemm_f64", "permute", "jacobi_svd", "su_absorb", "su_theta",
                                "su_truncate", "su_rebuild", "gate", "phys_tensors", "double_layer",
                                "env_init", "proj_prep", "normalize_store", "spectra_delta",
                                "ket_layer", "rho1", "rho2", "observables", "init_state", "bond_op",
                                "tc_gemm_bf16", "tc_split_prep", "orth_cqr", "ed_elementwise"};
std::atomic<unsigned long long> g_launches{0};
std::mutex g_mu;
std::atomic<bool> g_on{false};
struct Rec { int cls; cudaEvent_t a, b; double flops; };
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;
double g_flops[K_NCLASS];
unsigned long long g_count[K_NCLASS];
double g_ms[K_NCLASS];
unsigned long long g_devflops_host[K_NCLASS];
double g_tc_executed = 0.0;

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

__device__ unsigned long long g_dev_flops;
__device__ unsigned long long g_dev_ctr[CTR_N];

namespace {
// device addresses of the counters, looked up once per device
constexpr int kMaxDev = 64;
std::mutex g_sym_mu;
unsigned long long* g_flops_addr[kMaxDev] = {nullptr};
unsigned long long* g_ctr_addr[kMaxDev] = {nullptr};

unsigned long long* symbol_addr(unsigned long long** cache, const void* sym) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
  std::lock_guard<std::mutex> lk(g_sym_mu);
  if (!cache[dev]) {
    unsigned long long* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, sym) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cache[dev] = p;
  }
  return cache[dev];
}
}  // namespace

unsigned long long* prof_device_flops() { return symbol_addr(g_flops_addr, (const void*)&g_dev_flops); }

unsigned long long* prof_device_counters() { return symbol_addr(g_ctr_addr, (const void*)&g_dev_ctr); }

const char* kernel_class_name(int k) { return (k >= 0 && k < K_NCLASS) ? kNames[k] : "?"; }

void prof_add_tc_executed(double flops) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_tc_executed += flops;
}

cudaEvent_t prof_begin(int cls, cudaStream_t st) {
  (void)cls;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on.load(std::memory_order_relaxed)) return nullptr;
  cudaEvent_t e;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    e = take_event();
  }
  cudaEventRecord(e, st);
  return e;
}

void prof_end(int cls, cudaStream_t st, double flops, cudaEvent_t start) {
  if (!start) return;
  cudaEvent_t e;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    e = take_event();
  }
  cudaEventRecord(e, st);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({cls, start, e, flops});
}

bool prof_enabled() { return g_on.load(std::memory_order_relaxed); }

}  // namespace ipeps

using namespace ipeps;

extern "C" {

unsigned long long ipeps_launch_count(void) { return g_launches.load(); }

int ipeps_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaDeviceSynchronize();
  for (auto& r : g_recs) { g_free.push_back(r.a); g_free.push_back(r.b); }
  g_recs.clear();
  for (int k = 0; k < K_NCLASS; ++k) { g_flops[k] = 0; g_count[k] = 0; g_ms[k] = 0; }
  g_tc_executed = 0.0;
  unsigned long long zero[CTR_N] = {0};
  cudaMemcpyToSymbol(g_dev_flops, zero, sizeof(unsigned long long));
  cudaMemcpyToSymbol(g_dev_ctr, zero, sizeof(zero));
  g_on.store(on != 0);
  return 0;
}

int ipeps_profile_classes(void) { return K_NCLASS; }

int ipeps_profile_counters(unsigned long long* out, int n) {
  if (!out || n < 1) return 1;
  unsigned long long v[CTR_N] = {0};
  if (cudaDeviceSynchronize() != cudaSuccess) return 5;
  cudaMemcpyFromSymbol(v, g_dev_ctr, sizeof(v));
  for (int i = 0; i < n; ++i) out[i] = i < CTR_N ? v[i] : 0;
  return 0;
}

int ipeps_profile_tc_executed(double* flops_out) {
  if (!flops_out) return 1;
  std::lock_guard<std::mutex> lk(g_mu);
  *flops_out = g_tc_executed;
  return 0;
}

const char* ipeps_profile_name(int k) { return kernel_class_name(k); }

int ipeps_profile_read(double* ms, double* flops, unsigned long long* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (cudaDeviceSynchronize() != cudaSuccess) return 5;
  for (auto& r : g_recs) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    g_ms[r.cls] += t;
    g_flops[r.cls] += r.flops;
    g_count[r.cls] += 1;
    g_free.push_back(r.a);
    g_free.push_back(r.b);
  }
  g_recs.clear();
  unsigned long long devf = 0;
  cudaMemcpyFromSymbol(&devf, g_dev_flops, sizeof(devf));
  for (int k = 0; k < K_NCLASS; ++k) {
    if (ms) ms[k] = g_ms[k];
    if (flops) flops[k] = g_flops[k] + (k == K_JACOBI ? (double)devf : 0.0);
    if (launches) launches[k] = g_count[k];
  }
  return 0;
}

}  // extern "C"

// ----------------------------------------------------------------------------- FP64 peak probe
// Eight independent FMA chains per thread over 152 x 8 CTAs; the measured rate is the denominator
// of the roofline for kernels bound by FP64 arithmetic (this part has no FP64 tensor path).
namespace ipeps {
__global__ void dfma_probe_kernel(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
}  // namespace ipeps

extern "C" int ipeps_kernel_fp64_peak(double* tflops_out) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256, iters = 200;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_probe_kernel<<<blocks, threads>>>(out, 10, 0.999999, 1e-7);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    dfma_probe_kernel<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return 5;
  const double flops = 2.0 * blocks * threads * (double)iters * 16 * 8;
  *tflops_out = flops / (best * 1e-3) / 1e12;
  return 0;
}
