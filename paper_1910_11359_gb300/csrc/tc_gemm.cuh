// Split-precision (3-term BF16) complex GEMM on tcgen05 tensor cores (see tc_gemm.cu).
#pragma once
#include "linalg.cuh"

namespace ipeps {
namespace tc {
// workspace needed by zgemm_split_bf16 for one batched product of these sizes
size_t split_workspace_bytes(int M, int N, int K, int batch);
// C = alpha op(A) op(B) + beta C, complex, each operand split into two BF16 terms, FP32 accumulation
int zgemm_split_bf16(const GemmDesc& g, void* work, size_t work_bytes, unsigned* err, cudaStream_t st);
// plain BF16 x BF16 -> FP32 GEMM: C32[b] (Mp x Np) = A3[b] (Mp x Kp) * B3t[b]^T, K-major operands,
// 128 x bn output tiles (bn = 128 or 256); Mp a multiple of 128, Np of bn and Kp of 64.
// algo_flops: the algorithmic flops this launch serves (recorded by the launch accounting; <= 0
// records the executed 2 Mp Np Kp batch instead)
int gemm_bf16_raw(const void* A3, const void* B3t, float* C32, int Mp, int Np, int Kp, int batch,
                  int bn, double algo_flops, unsigned* err, cudaStream_t st, const int* skip = nullptr,
                  int skip_mod = 0);
}  // namespace tc
}  // namespace ipeps
