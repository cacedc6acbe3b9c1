// Simple-update device work buffers and driver (see su.cu).
#pragma once
#include "linalg.cuh"

namespace ipeps {

struct SuWork {
  cplx *Amat, *Bmat;            // [B][D^3][dD] absorbed tensors
  cplx *UA, *UB;                // [B][D^3][dD]
  double *SA, *SB;              // [B][dD]
  cplx *VA, *VB;                // [B][dD][dD]
  cplx* theta;                  // [B][nt][nt], nt = d * dD
  cplx *X, *Y;                  // [B][nt][nt]
  double* Stheta;               // [B][nt]
  int* kept;                    // [B]
  cplx* tgwork;                 // Jacobi column storage for theta when it exceeds shared memory
  size_t tgwork_bytes;
  // device pointer arrays for the batched SVDs
  const cplx* const* qA; cplx* const* qU; double* const* qS; cplx* const* qV;   // 2B
  const cplx* const* tA; cplx* const* tU; double* const* tS; cplx* const* tV;   // B
};

int su_bond_update(SuWork& w, cplx* GA, cplx* GB, double* lam, double* eps, const cplx* gate,
                   int legA, int d, int D, int batch, unsigned* err, cudaStream_t st);

}  // namespace ipeps
