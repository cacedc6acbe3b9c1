// Device model helpers (see model.cu).
#pragma once
#include "common.cuh"

namespace ipeps {
int build_gates(const double* J, const double* V, const double* h, const double* deltas, int ndelta,
                int batch, int d, int dA, cplx* out, cudaStream_t st);
int build_bond_ops(const double* J, const double* V, int batch, int d, int dA, cplx* out,
                   cudaStream_t st);
int init_state(cplx* GA, cplx* GB, double* lam, int d, int dA, int D, int batch, cudaStream_t st);
int physical_tensors(const cplx* GA, const cplx* GB, const double* lam, cplx* A, cplx* B, int d, int D,
                     int batch, cudaStream_t st);
int double_layers(const cplx* A, cplx* out, int d, int D, int batch, int nrot, cudaStream_t st);
}  // namespace ipeps
