// FP64 dense building blocks: batched complex GEMM, tensor permutation, cluster one-sided Jacobi SVD.
#pragma once
#include "common.cuh"

namespace ipeps {

enum Op : int { OP_N = 0, OP_T = 1, OP_C = 2 };

// One batched complex GEMM description: for b in [0, batch):
//   C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b]       (row-major, leading dimensions lda..ldc)
// op(A) is M x K: OP_N reads A[m*lda + k]; OP_T reads A[k*lda + m]; OP_C reads conj(A[k*lda + m]).
// op(B) is K x N: OP_N reads B[k*ldb + n]; OP_T reads B[n*ldb + k]; OP_C reads conj(B[n*ldb + k]).
// Pointers are either strided (base + b * stride) or taken from device pointer arrays (ptrs != 0).
struct GemmDesc {
  int M, N, K, batch;
  int opA, opB;
  long long lda, ldb, ldc;
  long long sA, sB, sC;           // batch strides in elements (used when the pointer arrays are null)
  const cplx* A; const cplx* B; cplx* C;
  const cplx* const* Aptr; const cplx* const* Bptr; cplx* const* Cptr;
  cplx alpha, beta;
  const int* skip;                // optional: problem b is left untouched when skip[b] != 0, or
  int skip_mod;                   // skip[b % skip_mod] != 0 when skip_mod > 0 (per-instance flags)
};

__host__ __device__ __forceinline__ bool skipped(const int* skip, int skip_mod, int b) {
  return skip && skip[skip_mod > 0 ? b % skip_mod : b];
}

int zgemm_f64(const GemmDesc& g, cudaStream_t st);

// out = permute(in): out axis j is in axis perm[j]; rank <= 8; batched with element strides;
// problems with skipped(skip, skip_mod, b) are left untouched.
int permute_c128(const cplx* in, cplx* out, int rank, const int* dims, const int* perm, int batch,
                 long long s_in, long long s_out, cudaStream_t st, const int* skip = nullptr,
                 int skip_mod = 0);

// One-sided (Hestenes) Jacobi SVD of a batch of m x n complex matrices (m >= n), A = U S V^+.
// Each problem is handled by one thread-block cluster (8 CTAs, or 16 for m >= 1024 where the part
// accepts that size) whose CTAs own disjoint row slices of [A; W], in shared memory or, when they
// do not fit, in SvdDesc::gwork; pair dot products are reduced across the cluster through
// distributed shared memory.  Singular values are sorted in descending order.  U (m x n, row-major, may be null),
// V (n x n row-major with V[i*ldv + j] = V_ij, may be null).
struct SvdDesc {
  int m, n, batch;
  const cplx* const* A; long long lda;
  cplx* const* U; long long ldu;
  double* const* S;
  cplx* const* V; long long ldv;
  double tol;          // rotate a pair when |a_p^+ a_q| > tol * ||a_p|| ||a_q||
  int max_sweeps;
  unsigned* err;       // device error word (DevErr bits)
  int* sweeps_out;     // optional: sweeps used per problem (1 = the input columns were orthogonal)
  const int* skip;     // optional: problems with skipped(skip, skip_mod, b) are left untouched
  int skip_mod = 0;
  // optional global-memory column storage for blocks whose rows do not fit in shared memory
  // (jacobi_svd_global_bytes(m, n, batch) bytes; the columns then live in L2 instead of SMEM)
  cplx* gwork = nullptr;
  size_t gwork_bytes = 0;
};

int jacobi_svd(const SvdDesc& d, cudaStream_t st);
size_t jacobi_svd_smem_bytes(int m, int n);
// the columns of [A; W] fit in the shared memory of the 8-CTA cluster
bool jacobi_svd_fits(int m, int n);
// the block can be factorised at all (with gwork when it does not fit in shared memory)
bool jacobi_svd_supported(int m, int n);
size_t jacobi_svd_global_bytes(int m, int n, int batch);

}  // namespace ipeps
