// Simple-update bond step on the device (Jiang, Weng & Xiang, PRL 101, 090603 (2008); the paper's
// quench, Sec. "Set up for iPEPS" and Appendix).  Reduced-tensor form: each site tensor with the
// weights of its three other legs absorbed is factorised A~ = U_A (S_A V_A^+) by a Jacobi SVD (this
// plays the role of the QR step), the gate acts on the small theta = R_A lam R_B, a second Jacobi
// SVD truncates theta back to D, and U_A / U_B map the kept vectors back to full site tensors.  The
// nonzero singular values equal those of the unreduced two-site tensor.
#include "su.cuh"
#include "prof.cuh"

namespace ipeps {

// other legs of a leg g in increasing order
__device__ __forceinline__ void other_legs(int g, int* o) {
  int k = 0;
  for (int j = 0; j < 4; ++j)
    if (j != g) o[k++] = j;
}

// Amat[b][(o1 o2 o3)][(s k)] = Gamma[b][s][legs] * prod lamLeg[o] ; lamLeg for A is lam[g'],
// for B it is lam[(g' + 2) % 4].  One output element per thread.
__global__ void su_absorb_kernel(const cplx* GA, const cplx* GB, const double* lam, int legA, int d,
                                 int D, int batch, cplx* Amat, cplx* Bmat) {
  const int D3 = D * D * D, D4 = D3 * D, n = d * D;
  const long long per = (long long)D3 * n;
  const long long total = 2LL * batch * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int side = (int)(i / (batch * per));     // 0 = A, 1 = B
    const long long r0 = i % (batch * per);
    const int b = (int)(r0 / per);
    const int row = (int)((r0 % per) / n), col = (int)(r0 % n);
    const int s = col / D, k = col % D;
    const int g = side == 0 ? legA : (legA + 2) % 4;
    int o[3];
    other_legs(g, o);
    int idx[4];
    idx[o[0]] = row / (D * D);
    idx[o[1]] = (row / D) % D;
    idx[o[2]] = row % D;
    idx[g] = k;
    const double* L = lam + (size_t)b * 4 * D;
    double w = 1.0;
    for (int j = 0; j < 3; ++j) {
      int leg = o[j];
      int lamleg = side == 0 ? leg : (leg + 2) % 4;
      w *= L[lamleg * D + idx[leg]];
    }
    const int v = ((idx[0] * D + idx[1]) * D + idx[2]) * D + idx[3];
    const cplx* G = (side == 0 ? GA : GB) + (size_t)b * d * D4;
    cplx val = cscale(G[(size_t)s * D4 + v], w);
    (side == 0 ? Amat : Bmat)[(size_t)b * per + (size_t)row * n + col] = val;
  }
}

// theta[b][(a sA') , (c sB')] = sum_{sA,sB} U[(sA' sB'),(sA sB)] sum_k R_A[a][(sA k)] lam_g[k] R_B[c][(sB k)]
// with R = diag(S) V^+, i.e. R[a][(s k)] = S[a] conj(V[(s k)][a]).
__global__ void su_theta_kernel(const double* SA, const cplx* VA, const double* SB, const cplx* VB,
                                const double* lam, const cplx* U, int legA, int d, int D, int batch,
                                cplx* theta) {
  const int n = d * D, nt = n * d;
  const long long per = (long long)nt * nt;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)batch * per;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per);
    const int row = (int)((i % per) / nt), col = (int)(i % nt);
    const int a = row / d, sAp = row % d, c = col / d, sBp = col % d;
    const double* lg = lam + (size_t)b * 4 * D + legA * D;
    const cplx* Ub = U + (size_t)b * d * d * d * d;
    const cplx* VAb = VA + (size_t)b * n * n;
    const cplx* VBb = VB + (size_t)b * n * n;
    // factor singular values at roundoff level relative to the largest are exact zeros
    double sa = SA[(size_t)b * n + a], sc = SB[(size_t)b * n + c];
    if (!(sa > 1e-14 * SA[(size_t)b * n])) sa = 0.0;
    if (!(sc > 1e-14 * SB[(size_t)b * n])) sc = 0.0;
    cplx acc = cmk(0.0, 0.0);
    for (int sA = 0; sA < d; ++sA)
      for (int sB = 0; sB < d; ++sB) {
        cplx x = cmk(0.0, 0.0);
        for (int k = 0; k < D; ++k) {
          // R_A[a][(sA k)] = sa conj(VA[(sA k)][a]);  R_B likewise
          cplx ra = cconj(VAb[(size_t)(sA * D + k) * n + a]);
          cplx rb = cconj(VBb[(size_t)(sB * D + k) * n + c]);
          cfma(x, cscale(ra, lg[k]), rb);
        }
        cfma(acc, Ub[(size_t)(sAp * d + sBp) * d * d + sA * d + sB], x);
      }
    theta[i] = cscale(acc, sa * sc);
  }
}

// Truncation (multiplets at the cut are kept whole), discarded weight, new bond weights.
__global__ void su_truncate_kernel(const double* S, int nt, int D, int legA, double* lam, double* eps,
                                   int* kept, double degen_rtol, double tiny_rel) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  const double* s = S + (size_t)b * nt;
  int K = D < nt ? D : nt;
  while (K > 1 && K < nt && s[K] > tiny_rel * s[0] && s[K - 1] / s[K] - 1.0 < degen_rtol) --K;
  double tot = 0.0, disc = 0.0, keep = 0.0;
  for (int j = 0; j < nt; ++j) tot += s[j] * s[j];
  for (int j = K; j < nt; ++j) disc += s[j] * s[j];
  for (int j = 0; j < K; ++j) keep += s[j] * s[j];
  eps[b] += tot > 0.0 ? disc / tot : 0.0;
  const double nk = sqrt(keep);
  double* l = lam + (size_t)b * 4 * D + legA * D;
  for (int j = 0; j < D; ++j) l[j] = (j < K && nk > 0.0) ? s[j] / nk : 0.0;
  kept[b] = K;
}

// New site tensors: Gamma'[s][legs] with the bond leg = kept index k < K,
// A: (1/lam others) sum_a U_A[(others)][a] X[(a s)][k];  B: conj(Y[(c s)][k]) instead of X.
// The weights lam of the other legs are unchanged by this bond step.
__global__ void su_rebuild_kernel(const cplx* UA, const cplx* UB, const cplx* X, const cplx* Y,
                                  const double* lam, const int* kept, int legA, int d, int D, int batch,
                                  cplx* GA, cplx* GB, double pinv_rel) {
  const int D3 = D * D * D, D4 = D3 * D, n = d * D, nt = n * d;
  const long long per = (long long)d * D4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2LL * batch * per;
       i += (long long)gridDim.x * blockDim.x) {
    const int side = (int)(i / (batch * per));
    const long long r0 = i % (batch * per);
    const int b = (int)(r0 / per);
    const int s = (int)((r0 % per) / D4), v = (int)(r0 % D4);
    int idx[4] = {v / (D * D * D), (v / (D * D)) % D, (v / D) % D, v % D};
    const int g = side == 0 ? legA : (legA + 2) % 4;
    const int k = idx[g];
    cplx out = cmk(0.0, 0.0);
    if (k < kept[b]) {
      int o[3];
      other_legs(g, o);
      const int row = (idx[o[0]] * D + idx[o[1]]) * D + idx[o[2]];
      const double* L = lam + (size_t)b * 4 * D;
      double w = 1.0;
      for (int j = 0; j < 3; ++j) {
        const int lamleg = side == 0 ? o[j] : (o[j] + 2) % 4;
        const double* lv = L + lamleg * D;
        double mx = 0.0;
        for (int q = 0; q < D; ++q) mx = fmax(mx, lv[q]);
        const double x = lv[idx[o[j]]];
        w *= (x > pinv_rel * mx) ? 1.0 / x : 0.0;
      }
      if (w != 0.0) {
        const cplx* Uq = (side == 0 ? UA : UB) + (size_t)b * D3 * n;
        const cplx* Z = (side == 0 ? X : Y) + (size_t)b * nt * nt;
        cplx acc = cmk(0.0, 0.0);
        for (int a = 0; a < n; ++a) {
          cplx z = Z[(size_t)(a * d + s) * nt + k];
          if (side == 1) z = cconj(z);
          cfma(acc, Uq[(size_t)row * n + a], z);
        }
        out = cscale(acc, w);
      }
    }
    (side == 0 ? GA : GB)[(size_t)b * per + (size_t)s * D4 + v] = out;
  }
}

int su_bond_update(SuWork& w, cplx* GA, cplx* GB, double* lam, double* eps, const cplx* gate,
                   int legA, int d, int D, int batch, unsigned* err, cudaStream_t st) {
  const int D3 = D * D * D, n = d * D, nt = n * d;
  if (D3 < n) return cuda_fail(cudaErrorInvalidValue, "simple update needs D^3 >= d D", __FILE__, __LINE__);
  const int blocks = 152 * 4, threads = 256;
  IPEPS_LAUNCH(K_SU_ABSORB, 0, st,
               su_absorb_kernel<<<blocks, threads, 0, st>>>(GA, GB, lam, legA, d, D, batch, w.Amat, w.Bmat));
  IPEPS_CUDA_TRY(cudaGetLastError());
  // factorise both absorbed tensors in one batch of 2B problems
  SvdDesc q;
  q.m = D3; q.n = n; q.batch = 2 * batch;
  q.A = w.qA; q.lda = n; q.U = w.qU; q.ldu = n; q.S = w.qS; q.V = w.qV; q.ldv = n;
  q.tol = 4e-16 * D3; q.max_sweeps = 60; q.err = err; q.sweeps_out = nullptr; q.skip = nullptr;
  if (int rc = jacobi_svd(q, st)) return rc;
  IPEPS_LAUNCH(K_SU_THETA, 8.0 * batch * (double)nt * nt * d * d * (D + 1), st,
               su_theta_kernel<<<blocks, threads, 0, st>>>(w.SA, w.VA, w.SB, w.VB, lam, gate, legA, d, D, batch, w.theta));
  IPEPS_CUDA_TRY(cudaGetLastError());
  SvdDesc t;
  t.m = nt; t.n = nt; t.batch = batch;
  t.A = w.tA; t.lda = nt; t.U = w.tU; t.ldu = nt; t.S = w.tS; t.V = w.tV; t.ldv = nt;
  t.tol = 4e-16 * nt; t.max_sweeps = 60; t.err = err; t.sweeps_out = nullptr; t.skip = nullptr;
  t.gwork = w.tgwork; t.gwork_bytes = w.tgwork_bytes;
  if (int rc = jacobi_svd(t, st)) return rc;
  IPEPS_LAUNCH(K_SU_TRUNCATE, 0, st,
               su_truncate_kernel<<<batch, 32, 0, st>>>(w.Stheta, nt, D, legA, lam, eps, w.kept, 1e-10, 1e-14));
  IPEPS_CUDA_TRY(cudaGetLastError());
  IPEPS_LAUNCH(K_SU_REBUILD, 16.0 * batch * d * (double)D3 * D * n, st,
               su_rebuild_kernel<<<blocks, threads, 0, st>>>(w.UA, w.UB, w.X, w.Y, lam, w.kept, legA, d, D, batch,
                                                            GA, GB, 1e-14));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace ipeps
