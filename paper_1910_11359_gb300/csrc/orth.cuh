// Column-scaled Cholesky QR of batched tall-skinny complex blocks and split-K A^+ B products
// (see orth.cu).
#pragma once
#include "linalg.cuh"

namespace ipeps {

struct OrthDesc {
  int N, k, batch;
  const cplx* X; long long sX;   // inputs N x k, row-major, batch stride sX (not modified)
  cplx* Q; long long sQ;         // outputs: orthonormal columns spanning X's (zero where X's are ~0)
  void* work; size_t work_bytes; // orth_work_bytes(N, k, batch)
  const int* skip;               // optional [batch]: problems left untouched
  int* fail;                     // [batch]: set to 1 (never cleared here) when the factorisation
                                 // broke down or the last pass still saw a Gram matrix off the
                                 // identity by more than dev_fail
  int passes;                    // Cholesky QR passes (>= 1)
  bool shifted;                  // the first pass adds the diagonal shift (for blocks that may be
                                 // far from orthonormal after column scaling; then passes >= 3)
  double dev_fail;
};

size_t orth_work_bytes(int N, int k, int batch);
size_t orth_smem_bytes(int k);
bool orth_supported(int k);
int orth_cqr(const OrthDesc& d, cudaStream_t st);
// C[q] (k x k, batch stride sC) = A[q]^+ B[q] for N x k blocks A, B (batch strides sA, sB), summed
// over row blocks in a fixed order; partial needs batch * ceil(N / 64) * k * k elements
int atb_product(const cplx* A, long long sA, const cplx* B, long long sB, int N, int k, int batch,
                cplx* partial, cplx* C, long long sC, const int* skip, cudaStream_t st);

}  // namespace ipeps
