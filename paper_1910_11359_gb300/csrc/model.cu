// Dilated site model on the device: bond Hamiltonian, Trotter gate, initial state, physical tensors,
// double layers (paper Sec. "Set up for iPEPS": Eq. Hanc in hard-core boson form, Initialization,
// Fig. 1).  Local basis s = n * d_A + a, d = 2 d_A; two-site index sA * d + sB.
#include "model.cuh"
#include "prof.cuh"

namespace ipeps {

// --------------------------------------------------------------------------- local operators
__device__ __forceinline__ int occ_of(int s, int dA) { return s / dA; }
__device__ __forceinline__ double level_of(int s, int dA) {
  int a = s % dA;
  return dA > 1 ? 1.0 - 2.0 * a / (dA - 1) : 0.0;
}
// <s|b|s'>: 1 when s' has the boson and s is the same auxiliary level without it
__device__ __forceinline__ double b_elem(int s, int sp, int dA) {
  return (occ_of(sp, dA) == 1 && occ_of(s, dA) == 0 && (s % dA) == (sp % dA)) ? 1.0 : 0.0;
}

// h_b[(sA sB), (sA' sB')] = -J (b+_A b_B + b_A b+_B) + V n_A n_B + (h / 4) (tau_A n_A + tau_B n_B)
__device__ double bond_h_elem(int row, int col, int d, int dA, double J, double V, double h) {
  int sA = row / d, sB = row % d, tA = col / d, tB = col % d;
  double v = 0.0;
  // b+_A b_B: <sA|b+|tA> = <tA|b|sA>
  v += -J * (b_elem(tA, sA, dA) * b_elem(sB, tB, dA) + b_elem(sA, tA, dA) * b_elem(tB, sB, dA));
  if (sA == tA && sB == tB) {
    v += V * occ_of(sA, dA) * occ_of(sB, dA);
    v += 0.25 * h * (level_of(sA, dA) * occ_of(sA, dA) + level_of(sB, dA) * occ_of(sB, dA));
  }
  return v;
}

// The bond Hamiltonian conserves every auxiliary level, so h_b is block diagonal: for each pair of
// levels (aA, aB) it acts on the four occupation states (nA, nB) only, and
// exp(-i h_b delta) = direct sum over (aA, aB) of exp(-i h_(aA,aB) delta) (4 x 4 each).
// One CTA per (instance, delta), one thread per block: U_block = exp(X), X = -i h_block delta, by
// scaling and squaring of the Taylor series (Moler & Van Loan, "Nineteen dubious ways to compute
// the exponential of a matrix", method 3): X / 2^s with ||X||_1 / 2^s <= 1/2, the series summed
// to order 24 by Horner's rule, then squared s times.  Output [delta][instance][d^2][d^2], two-site
// index sA * d + sB with s = n * d_A + a.
__global__ void gate_kernel(const double* J, const double* V, const double* h, const double* deltas,
                            int ndelta, int d, int dA, cplx* out) {
  const int b = blockIdx.x / ndelta, g = blockIdx.x % ndelta;
  const int d2 = d * d;
  cplx* U = out + ((size_t)g * gridDim.x / ndelta + b) * d2 * d2;
  for (int idx = threadIdx.x; idx < d2 * d2; idx += blockDim.x) U[idx] = cmk(0.0, 0.0);
  __syncthreads();
  const int blk = threadIdx.x;
  if (blk >= dA * dA) return;
  const int aA = blk / dA, aB = blk % dA;
  const double delta = deltas[g];
  int idx[4];                                    // two-site index of local state (nA, nB) = (m/2, m%2)
  for (int m = 0; m < 4; ++m) idx[m] = ((m >> 1) * dA + aA) * d + ((m & 1) * dA + aB);
  cplx X[16], E[16], T[16];
  double nrm = 0.0;
  for (int c = 0; c < 4; ++c) {
    double col = 0.0;
    for (int r = 0; r < 4; ++r) {
      const double hv = bond_h_elem(idx[r], idx[c], d, dA, J[b], V[b], h[b]);
      X[r * 4 + c] = cmk(0.0, -hv * delta);
      col += fabs(hv * delta);
    }
    nrm = fmax(nrm, col);
  }
  int sh = 0;
  double scale = 1.0;
  while (nrm > 0.5) { nrm *= 0.5; scale *= 0.5; ++sh; }
  for (int e = 0; e < 16; ++e) {
    X[e] = cscale(X[e], scale);
    E[e] = cmk((e / 4) == (e % 4) ? 1.0 : 0.0, 0.0);
  }
  // Horner: E <- I + X E / q for q = 24 .. 1
  for (int q = 24; q >= 1; --q) {
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        cplx acc = cmk(0.0, 0.0);
        for (int t = 0; t < 4; ++t) cfma(acc, X[r * 4 + t], E[t * 4 + c]);
        T[r * 4 + c] = cadd(cmk(r == c ? 1.0 : 0.0, 0.0), cscale(acc, 1.0 / q));
      }
    for (int e = 0; e < 16; ++e) E[e] = T[e];
  }
  for (int q = 0; q < sh; ++q) {
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        cplx acc = cmk(0.0, 0.0);
        for (int t = 0; t < 4; ++t) cfma(acc, E[r * 4 + t], E[t * 4 + c]);
        T[r * 4 + c] = acc;
      }
    for (int e = 0; e < 16; ++e) E[e] = T[e];
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) U[(size_t)idx[r] * d2 + idx[c]] = E[r * 4 + c];
}

int build_gates(const double* J, const double* V, const double* h, const double* deltas, int ndelta,
                int batch, int d, int dA, cplx* out, cudaStream_t st) {
  if (dA < 1 || dA * dA > 1024 || d != 2 * dA)
    return cuda_fail(cudaErrorInvalidValue, "gate size", __FILE__, __LINE__);
  const int threads = dA * dA < 32 ? 32 : ((dA * dA + 31) / 32) * 32;
  IPEPS_LAUNCH(K_GATE, 0, st, gate_kernel<<<batch * ndelta, threads, 0, st>>>(J, V, h, deltas, ndelta, d, dA, out));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

// Bond operator without the field term, used by the energy readout: -J (b+ b + b b+) + V n n.
__global__ void bond_op_kernel(const double* J, const double* V, int d, int dA, cplx* out) {
  const int b = blockIdx.x, d2 = d * d;
  for (int idx = threadIdx.x; idx < d2 * d2; idx += blockDim.x)
    out[(size_t)b * d2 * d2 + idx] = cmk(bond_h_elem(idx / d2, idx % d2, d, dA, J[b], V[b], 0.0), 0.0);
}

int build_bond_ops(const double* J, const double* V, int batch, int d, int dA, cplx* out,
                   cudaStream_t st) {
  IPEPS_LAUNCH(K_BONDOP, 0, st, bond_op_kernel<<<batch, 256, 0, st>>>(J, V, d, dA, out));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

// --------------------------------------------------------------------------- initial state
// CDW (x) |+>: A holds the boson on every auxiliary level, B none; bond index 0 only; lam = (1,0,..)
__global__ void init_state_kernel(cplx* GA, cplx* GB, double* lam, int d, int dA, int D, int batch) {
  const int D4 = D * D * D * D;
  const long long ng = (long long)batch * d * D4;
  const double amp = 1.0 / sqrt((double)dA);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ng;
       i += (long long)gridDim.x * blockDim.x) {
    long long r = i % ((long long)d * D4);
    int s = (int)(r / D4), v = (int)(r % D4);
    GA[i] = cmk((v == 0 && s / dA == 1) ? amp : 0.0, 0.0);
    GB[i] = cmk((v == 0 && s / dA == 0) ? amp : 0.0, 0.0);
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)batch * 4 * D;
       i += (long long)gridDim.x * blockDim.x)
    lam[i] = (i % D == 0) ? 1.0 : 0.0;
}

int init_state(cplx* GA, cplx* GB, double* lam, int d, int dA, int D, int batch, cudaStream_t st) {
  IPEPS_LAUNCH(K_INIT_STATE, 0, st, init_state_kernel<<<64, 256, 0, st>>>(GA, GB, lam, d, dA, D, batch));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

// --------------------------------------------------------------------------- physical tensors
// A = Gamma_A sqrt(lam) on every leg; B's leg g carries lam[(g + 2) % 4] (it joins A's opposite leg).
__global__ void phys_kernel(const cplx* GA, const cplx* GB, const double* lam, cplx* A, cplx* B, int d,
                            int D, int batch) {
  const int D4 = D * D * D * D;
  const long long n = (long long)batch * d * D4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / ((long long)d * D4));
    const int v = (int)(i % D4);
    const int u = v / (D * D * D), l = (v / (D * D)) % D, dd = (v / D) % D, r = v % D;
    const double* L = lam + (size_t)b * 4 * D;
    double wa = sqrt(L[0 * D + u] * L[1 * D + l] * L[2 * D + dd] * L[3 * D + r]);
    double wb = sqrt(L[2 * D + u] * L[3 * D + l] * L[0 * D + dd] * L[1 * D + r]);
    A[i] = cscale(GA[i], wa);
    B[i] = cscale(GB[i], wb);
  }
}

int physical_tensors(const cplx* GA, const cplx* GB, const double* lam, cplx* A, cplx* B, int d, int D,
                     int batch, cudaStream_t st) {
  IPEPS_LAUNCH(K_PHYS, 0, st, phys_kernel<<<152 * 4, 256, 0, st>>>(GA, GB, lam, A, B, d, D, batch));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

// --------------------------------------------------------------------------- double layers
// a[(u u'), (l l'), (d d'), (r r')] = sum_s A[s,u,l,d,r] conj(A[s,u',l',d',r']) written in the four
// rotations rot^k(a)[i0,i1,i2,i3] = a[i_k, i_{k+1}, i_{k+2}, i_{k+3}] (indices mod 4); rot is the
// 90-degree counter-clockwise relabelling (new up = old right).  Output [k][batch][D2^4].
__global__ void double_layer_kernel(const cplx* A, cplx* out, int d, int D, int batch, int nrot) {
  const int D2 = D * D;
  const long long D8 = (long long)D2 * D2 * D2 * D2;
  const int D4 = D2 * D2;
  const long long n = (long long)batch * D8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / D8);
    long long o = i % D8;
    int idx[4];
    idx[3] = (int)(o % D2); o /= D2;
    idx[2] = (int)(o % D2); o /= D2;
    idx[1] = (int)(o % D2); o /= D2;
    idx[0] = (int)o;
    int ket = 0, bra = 0;
    for (int k = 0; k < 4; ++k) { ket = ket * D + idx[k] / D; bra = bra * D + idx[k] % D; }
    const cplx* Ab = A + (size_t)b * d * D4;
    cplx acc = cmk(0.0, 0.0);
    for (int s = 0; s < d; ++s) cfmac(acc, Ab[(size_t)s * D4 + bra], Ab[(size_t)s * D4 + ket]);
    // acc = sum_s A[s,ket] conj(A[s,bra]); scatter into every rotation
    for (int k = 0; k < nrot; ++k) {
      // rot^k(a)[p] = a[q] with q_j = p_{(j + k) mod 4}; here q = idx, so p_{(j + k) mod 4} = idx[j]
      int p[4];
      for (int j = 0; j < 4; ++j) p[(j + k) % 4] = idx[j];
      long long off = (((long long)p[0] * D2 + p[1]) * D2 + p[2]) * D2 + p[3];
      out[((size_t)k * batch + b) * D8 + off] = acc;
    }
  }
}

int double_layers(const cplx* A, cplx* out, int d, int D, int batch, int nrot, cudaStream_t st) {
  const double D8 = (double)D * D * D * D * D * D * D * D;
  IPEPS_LAUNCH(K_DLAYER, 8.0 * d * D8 * batch, st,
               double_layer_kernel<<<152 * 8, 256, 0, st>>>(A, out, d, D, batch, nrot));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace ipeps
