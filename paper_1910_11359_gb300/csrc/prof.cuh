// Launch accounting: every kernel launch of the library goes through IPEPS_LAUNCH, which counts it
// and, while profiling is switched on, brackets it with CUDA events on its own stream and adds its
// algorithmic FP64 flop count to the kernel class.
#pragma once
#include <cuda_runtime.h>

namespace ipeps {

enum KernelClass : int {
  K_ZGEMM = 0, K_PERMUTE, K_JACOBI, K_SU_ABSORB, K_SU_THETA, K_SU_TRUNCATE, K_SU_REBUILD, K_GATE,
  K_PHYS, K_DLAYER, K_ENV_INIT, K_PROJ_PREP, K_NORM_STORE, K_SPECTRA, K_KET_LAYER, K_RHO1, K_RHO2,
  K_OBS, K_INIT_STATE, K_BONDOP, K_TC_GEMM, K_TC_PREP, K_ORTH, K_ED, K_NCLASS
};

const char* kernel_class_name(int k);
// prof_begin counts the launch and, while timing is on, records and returns its start event
// (nullptr otherwise); prof_end records the matching end event.  The start event travels with the
// launch site, so launches of one class from several host threads pair their own events.
cudaEvent_t prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double flops, cudaEvent_t start);
// device-side flop counter used by kernels whose work is data dependent (Jacobi sweeps)
unsigned long long* prof_device_flops();
// device-side work counters (reset by ipeps_profile_enable): indices below
enum DevCounter : int {
  CTR_JACOBI_PROBLEMS = 0,   // Jacobi SVD problems factorised (skipped ones not counted)
  CTR_JACOBI_ROUNDS,         // rotation rounds run, summed over problems
  CTR_JACOBI_SWEEPS,         // sweeps run, summed over problems
  CTR_SUB_ROUNDS,            // subspace-iteration rounds evaluated, summed over projector problems
  CTR_SUB_ACCEPTED,          // projector problems whose subspace iteration met its acceptance test
  CTR_SUB_UNCONVERGED,       // projector problems handed on at the round cap without meeting it
  CTR_ORTH_FALLBACK,         // subspace blocks orthonormalised by the tall Jacobi SVD instead of
                             // Cholesky QR (the factorisation broke down)
  CTR_N
};
unsigned long long* prof_device_counters();
// executed tensor-pipe flops of the tcgen05 GEMM launches (tallied while timing is on)
void prof_add_tc_executed(double flops);

// whether launches are being timed (convergence graphs are used only when they are not)
bool prof_enabled();

}  // namespace ipeps

#define IPEPS_LAUNCH(cls, flops, st, ...)                                  \
  do {                                                                    \
    cudaEvent_t ipeps_launch_start_ = ::ipeps::prof_begin((cls), (st));  \
    __VA_ARGS__;                                                          \
    ::ipeps::prof_end((cls), (st), (double)(flops), ipeps_launch_start_); \
  } while (0)
