// Launch accounting: every kernel launch of the library goes through IPEPS_LAUNCH, which counts it
// and, while profiling is switched on, brackets it with CUDA events on its own stream and adds its
// algorithmic FP64 flop count to the kernel class.
#pragma once
#include <cuda_runtime.h>

namespace ipeps {

enum KernelClass : int {
  K_ZGEMM = 0, K_PERMUTE, K_JACOBI, K_SU_ABSORB, K_SU_THETA, K_SU_TRUNCATE, K_SU_REBUILD, K_GATE,
  K_PHYS, K_DLAYER, K_ENV_INIT, K_PROJ_PREP, K_NORM_STORE, K_SPECTRA, K_OPEN_LAYER, K_RHO1, K_RHO2,
  K_OBS, K_INIT_STATE, K_BONDOP, K_TC_GEMM, K_TC_PREP, K_NCLASS
};

const char* kernel_class_name(int k);
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double flops);
// device-side flop counter used by kernels whose work is data dependent (Jacobi sweeps)
unsigned long long* prof_device_flops();

}  // namespace ipeps

#define IPEPS_LAUNCH(cls, flops, st, ...)             \
  do {                                               \
    ::ipeps::prof_begin((cls), (st));                \
    __VA_ARGS__;                                     \
    ::ipeps::prof_end((cls), (st), (double)(flops)); \
  } while (0)
