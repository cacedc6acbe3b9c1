// Split-precision (3-term) complex GEMM on the tcgen05 tensor cores (see tc_gemm.cu).
#pragma once
#include "linalg.cuh"

namespace ipeps {
namespace tc {
// operand split of the 3-term products: two BF16 terms per value (kind::f16) or two TF32 terms
// (kind::tf32)
enum SplitOp : int { SPLIT_BF16 = 0, SPLIT_TF32 = 1 };
// workspace needed by zgemm_split for one batched product of these sizes
size_t split_workspace_bytes(int M, int N, int K, int batch, int op);
// C = alpha op(A) op(B) + beta C, complex, each operand split into two terms of the operand type,
// the three leading products accumulated in FP32
int zgemm_split(const GemmDesc& g, int op, void* work, size_t work_bytes, unsigned* err, cudaStream_t st);
// plain BF16 x BF16 -> FP32 GEMM: C32[b] (Mp x Np) = A3[b] (Mp x Kp) * B3t[b]^T, K-major operands,
// 128 x bn output tiles (bn = 128 or 256); Mp a multiple of 128, Np of bn and Kp of 64.
// algo_flops: the algorithmic flops this launch serves (recorded by the launch accounting; <= 0
// records the executed 2 Mp Np Kp batch instead)
int gemm_bf16_raw(const void* A3, const void* B3t, float* C32, int Mp, int Np, int Kp, int batch,
                  int bn, double algo_flops, unsigned* err, cudaStream_t st, const int* skip = nullptr,
                  int skip_mod = 0);
// tile width the autotuner chose for BF16 products of this shape (0: not tuned yet)
int tuned_tile_width(int M, int N, int K);
}  // namespace tc
}  // namespace ipeps
