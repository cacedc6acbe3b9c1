// Readout from the converged environment (paper Sec. "Set up for iPEPS", Readout: local expectation
// values of |Psi(t)> are exact disorder averages with the auxiliaries traced out; Sec. "Results for
// interacting case": imbalance I = n_A - n_B).
//
// Every reduced density matrix is assembled from "left halves": in rotated frame f, at logical
// position q, with the open (ket x bra) site tensor,
//   Lh[e3r, c1r, s, s', kR] = C1 T1 T4 C4 T3 (around q) x A[s, uU, uL, uD, uR] conj(A)[s', bU, bL, bD, bR]
// where e3r / c1r are the right ends of T3 / T1, each double leg k = (u, b) pairs a ket and a bra
// index, and kR = (uR, bR) is the open right leg.  The ket and bra layers are contracted one after
// the other (cost 8 chi^2 d D^7 + 8 chi^2 d^2 D^5 per left half) rather than as the open double
// layer (8 chi^2 d^2 D^8, and d^2 D^8 numbers to hold).
//   rho1(q)          = Lh_f0(q) . (C2 T2 C3)(q)                          (A at (0,0), B at (1,0))
//   rho_h(p -> p+x)  = Lh_f0(p) . Lh_f2(p+x)                              (the right half is a left
//   rho_v(p -> p+y)  = Lh_f1(rot p) . Lh_f3(rot^3 (p+y))                   half rotated by 180 deg)
// The eight left halves needed (frames 0..3 x logical positions (0,0) [site A], (1,0) [site B])
// are computed as one batch.
#include <algorithm>
#include <vector>

#include "ctx.cuh"
#include "measure.cuh"
#include "prof.cuh"
#include "reduce.cuh"

namespace ipeps {

// single layer, rotated and reshaped for the ket and bra contractions:
// Ak[(a0 a1 a2), (s a3)] = rot^f(A)[s, a0, a1, a2, a3] (legs u, l, d, r of the rotated frame) and
// Akc = conj(Ak); leg j of the unrotated tensor carries the rotated frame's index a_{(j + f) mod 4}
__global__ void ket_layer_kernel(const cplx* A, int d, int D, int B, cplx* Ak, cplx* Akc, int f) {
  const int D3 = D * D * D, D4 = D3 * D, cols = d * D;
  const long long per = (long long)D3 * cols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)B * per;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / per);
    const int r = (int)((idx % per) / cols), cc = (int)(idx % cols);
    int p[4];
    p[0] = r / (D * D); p[1] = (r / D) % D; p[2] = r % D;
    const int s = cc / D;
    p[3] = cc % D;
    int q = 0;
    for (int j = 0; j < 4; ++j) q = q * D + p[(j + f) & 3];
    const cplx v = A[(size_t)b * d * D4 + (size_t)s * D4 + q];
    Ak[idx] = v;
    Akc[idx] = cconj(v);
  }
}

// rho1[q][s][s'] = sum_{a,b,k} Lh[a, b, s, s', k] RC[b, k, a];  one CTA per (site, b)
__global__ void rho1_kernel(const cplx* Lh, const cplx* RC, int chi, int D2, int d, cplx* rho) {
  const int q = blockIdx.x;
  const long long per = (long long)chi * chi * d * d * D2;
  const cplx* L = Lh + (size_t)q * per;
  const cplx* R = RC + (size_t)q * chi * D2 * chi;
  for (int ss = 0; ss < d * d; ++ss) {
    cplx acc = cmk(0.0, 0.0);
    for (long long t = threadIdx.x; t < (long long)chi * chi * D2; t += blockDim.x) {
      const int a = (int)(t / (chi * D2)), bb = (int)((t / D2) % chi), k = (int)(t % D2);
      cfma(acc, L[(((size_t)a * chi + bb) * d * d + ss) * D2 + k], R[((size_t)bb * D2 + k) * chi + a]);
    }
    const cplx sum = block_sum<256>(acc);
    if (threadIdx.x == 0) rho[(size_t)q * d * d + ss] = sum;
  }
}

// rho2[s, s', v, v'] = sum_{a,b,k} Lh1[a, b, s, s', k] Lh2[b, a, v, v', k]; one CTA per output entry
__global__ void rho2_kernel(const cplx* const* L1, const cplx* const* L2, int chi, int D2, int d,
                            cplx* rho) {
  const int d2 = d * d;
  const int job = blockIdx.x / (d2 * d2), e = blockIdx.x % (d2 * d2);
  const int ss = e / d2, vv = e % d2;
  const cplx* X = L1[job];
  const cplx* Yp = L2[job];
  cplx acc = cmk(0.0, 0.0);
  for (long long t = threadIdx.x; t < (long long)chi * chi * D2; t += blockDim.x) {
    const int a = (int)(t / (chi * D2)), bb = (int)((t / D2) % chi), k = (int)(t % D2);
    cfma(acc, X[(((size_t)a * chi + bb) * d2 + ss) * D2 + k], Yp[(((size_t)bb * chi + a) * d2 + vv) * D2 + k]);
  }
  const cplx sum = block_sum<256>(acc);
  if (threadIdx.x == 0) {
    // rho index [s][s'][v][v'] from ss = s * d + s', vv = v * d + v'
    const int s = ss / d, sp = ss % d, v = vv / d, vp = vv % d;
    rho[(size_t)job * d2 * d2 + ((s * d + sp) * d + v) * d + vp] = sum;
  }
}

// z / w for complex w != 0
__device__ __forceinline__ cplx cdiv(cplx z, cplx w) {
  const double n = w.x * w.x + w.y * w.y;
  return cmk((z.x * w.x + z.y * w.y) / n, (z.y * w.x - z.x * w.y) / n);
}

// Renyi entropies S_1, S_1/2, S_2 of the physical one-site RDM of A: the auxiliary level traced out
// of rho_A (s = n * d_A + a) and the result divided by its (complex) trace; its two eigenvalues in
// closed form (2 x 2 Hermitian).
__device__ void renyi_phys(const cplx* r, int d, int dA, double* S1, double* Sh, double* S2) {
  cplx a = cmk(0.0, 0.0), c = cmk(0.0, 0.0), off = cmk(0.0, 0.0);
  for (int x = 0; x < dA; ++x) {
    a = cadd(a, r[(size_t)x * d + x]);                            // n = 0
    c = cadd(c, r[(size_t)(dA + x) * d + dA + x]);                // n = 1
    off = cadd(off, r[(size_t)x * d + dA + x]);                   // <n=0| rho |n=1>
  }
  const cplx tr = cadd(a, c);
  const double an = cdiv(a, tr).x, cn = cdiv(c, tr).x;
  const cplx o = cdiv(off, tr);
  const double mid = 0.5 * (an + cn), rad = sqrt(0.25 * (an - cn) * (an - cn) + o.x * o.x + o.y * o.y);
  double p[2] = {fmax(mid + rad, 0.0), fmax(mid - rad, 0.0)};
  double s1 = 0.0, sq = 0.0, p2 = 0.0;
  for (int i = 0; i < 2; ++i) {
    if (p[i] > 0.0) s1 -= p[i] * log(p[i]);
    sq += sqrt(p[i]);
    p2 += p[i] * p[i];
  }
  *S1 = s1;
  *Sh = 2.0 * log(sq);
  *S2 = -log(p2);
}

// Observables per instance from rho1 (A, B) and the four bond RDMs:
// out[b] = {nA, nB, I, tauzA, tauzB, energy, purityA, |tr rho_A|, S1_A, S1/2_A, S2_A}.
// Every RDM is divided by its own complex trace: the environment fixes the network's value only up
// to a complex factor, which a ratio of real parts would not remove from the quadratic quantities
// (purity, Renyi entropies).
__global__ void observables_kernel(const cplx* rho1, const cplx* rho2, const cplx* bondop,
                                   const double* h, int B, int d, int dA, double* out) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  const int d2 = d * d;
  double n[2], tz[2], tn[2];
  cplx tr[2];
  for (int site = 0; site < 2; ++site) {
    const cplx* r = rho1 + (size_t)(site * B + b) * d2;
    cplx trc = cmk(0.0, 0.0), nn = cmk(0.0, 0.0), tt = cmk(0.0, 0.0), tnn = cmk(0.0, 0.0);
    for (int s = 0; s < d; ++s) {
      const cplx p = r[s * d + s];
      const int occ = s / dA;
      const double lev = dA > 1 ? 1.0 - 2.0 * (s % dA) / (dA - 1) : 0.0;
      trc = cadd(trc, p);
      nn = cadd(nn, cscale(p, occ));
      tt = cadd(tt, cscale(p, lev));
      tnn = cadd(tnn, cscale(p, lev * occ));
    }
    tr[site] = trc;
    n[site] = cdiv(nn, trc).x; tz[site] = cdiv(tt, trc).x; tn[site] = cdiv(tnn, trc).x;
  }
  double eb = 0.0;
  const cplx* H = bondop + (size_t)b * d2 * d2;
  for (int k = 0; k < 4; ++k) {
    const cplx* r = rho2 + (size_t)(k * B + b) * d2 * d2;
    cplx num = cmk(0.0, 0.0), den = cmk(0.0, 0.0);
    for (int s = 0; s < d; ++s)
      for (int t = 0; t < d; ++t)
        for (int v = 0; v < d; ++v)
          for (int w = 0; w < d; ++w)
            cfma(num, H[(size_t)(t * d + w) * d2 + s * d + v], r[((s * d + t) * d + v) * d + w]);
    for (int s = 0; s < d; ++s)
      for (int v = 0; v < d; ++v) den = cadd(den, r[((s * d + s) * d + v) * d + v]);
    eb += cdiv(num, den).x;
  }
  const cplx* rA = rho1 + (size_t)b * d2;
  cplx pur = cmk(0.0, 0.0);
  for (int s = 0; s < d; ++s)
    for (int t = 0; t < d; ++t) pur = cadd(pur, cmul(rA[s * d + t], rA[t * d + s]));
  pur = cdiv(pur, cmul(tr[0], tr[0]));
  double* o = out + (size_t)b * kObsPerInstance;
  o[0] = n[0]; o[1] = n[1]; o[2] = n[0] - n[1]; o[3] = tz[0]; o[4] = tz[1];
  o[5] = 0.5 * (eb + h[b] * (tn[0] + tn[1]));
  o[6] = pur.x; o[7] = sqrt(tr[0].x * tr[0].x + tr[0].y * tr[0].y);
  renyi_phys(rA, d, dA, &o[8], &o[9], &o[10]);
}

static GemmDesc gdm(int M, int N, int K, int batch) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.alpha = cmk(1.0, 0.0); g.beta = cmk(0.0, 0.0);
  return g;
}

size_t measure_bytes(int B, int d, int D, int chi) {
  Arena a;
  MeasureWork w;
  measure_carve(a, w, B, d, D, chi);
  return a.used;
}

// jobs per pass: as many of the 8 B left-half jobs as fit their intermediates in kMeasurePassBytes
// (at least one)
int measure_group(int B, int d, int D, int chi) {
  const long long D2 = (long long)D * D, T = (long long)chi * D2 * chi, chi2 = (long long)chi * chi;
  const size_t per_job = sizeof(cplx) * (size_t)(2 * T + T * D2 + 2 * T * D2 * D2 + chi2 * d * D2 * D2 +
                                                 chi2 * d * d * D2);
  const long long fit = (long long)(kMeasurePassBytes / per_job);
  return (int)std::max(1LL, std::min(fit, 8LL * B));
}

void measure_carve(Arena& a, MeasureWork& w, int B, int d, int D, int chi) {
  const long long D2 = (long long)D * D;
  const long long T = chi * D2 * chi;
  const long long G = w.group = measure_group(B, d, D, chi), chi2 = (long long)chi * chi;
  w.tl = a.take<cplx>((size_t)G * T);
  w.W1 = a.take<cplx>((size_t)G * T * D2);
  w.bl = a.take<cplx>((size_t)G * T);
  w.W2 = a.take<cplx>((size_t)G * T * D2 * D2);
  w.W2p = a.take<cplx>((size_t)G * T * D2 * D2);
  w.X = a.take<cplx>((size_t)G * chi2 * d * D2 * D2);
  w.Y = a.take<cplx>((size_t)G * chi2 * d * d * D2);
  w.ak = a.take<cplx>((size_t)8 * B * d * D2 * D2);
  w.akc = a.take<cplx>((size_t)8 * B * d * D2 * D2);
  w.Lh = a.take<cplx>((size_t)8 * B * chi * chi * d * d * D2);
  w.RCt = a.take<cplx>((size_t)2 * B * T);
  w.RC = a.take<cplx>((size_t)2 * B * T);
  w.rho1 = a.take<cplx>((size_t)2 * B * d * d);
  w.rho2 = a.take<cplx>((size_t)4 * B * d * d * d * d);
  w.obs = a.take<double>((size_t)kObsPerInstance * B);
}

void measure_build(Ctx& c, MeasureWork& w, PtrPool& pool, MeasureOff& o) {
  const int B = c.B, chi = c.chi;
  const long long D2 = c.D2, T = chi * D2 * chi, chi2 = (long long)chi * chi;
  auto Cp = [&](int i, int pos, int b) -> const void* { return c.Cenv[i & 3][pos] + (size_t)b * chi2; };
  auto Tp = [&](int i, int pos, int b) -> const void* { return c.Tenv[i & 3][pos] + (size_t)b * T; };
  std::vector<const void*> tlA, tlB, w1A, blA, blB, aoB;
  for (int f = 0; f < 4; ++f)
    for (int l = 0; l < 2; ++l)
      for (int b = 0; b < B; ++b) {
        const int lpos = l;                                   // logical (0,0) or (1,0)
        const int pp = (f & 1) ? pos_of(lpos >> 1, lpos & 1) : lpos;
        const int job = (f * 2 + l) * B + b;
        tlA.push_back(Cp(0 + f, pp, b));
        tlB.push_back(Tp(0 + f, pp, b));
        w1A.push_back(Tp(3 + f, pp, b));
        blA.push_back(Tp(2 + f, pp, b));
        blB.push_back(Cp(3 + f, pp, b));
        aoB.push_back(w.ak + (size_t)job * c.d * D2 * D2);
      }
  o.tlA = pool.add(tlA); o.tlB = pool.add(tlB); o.w1A = pool.add(w1A);
  o.blA = pool.add(blA); o.blB = pool.add(blB); o.aoB = pool.add(aoB);
  std::vector<const void*> rcA, rcB, rcC;
  for (int l = 0; l < 2; ++l)
    for (int b = 0; b < B; ++b) {
      rcA.push_back(Cp(1, l, b));
      rcB.push_back(Tp(1, l, b));
      rcC.push_back(Cp(2, l, b));
    }
  o.rcA = pool.add(rcA); o.rcB = pool.add(rcB); o.rcC = pool.add(rcC);
  // bond RDM operands: k = 0 rho_h(A->B), 1 rho_h(B->A), 2 rho_v(A->B), 3 rho_v(B->A)
  const long long Lper = (long long)chi * chi * c.d * c.d * D2;
  auto L = [&](int f, int l, int b) -> const void* { return w.Lh + (size_t)((f * 2 + l) * B + b) * Lper; };
  std::vector<const void*> r1, r2;
  for (int k = 0; k < 4; ++k)
    for (int b = 0; b < B; ++b) {
      if (k == 0) { r1.push_back(L(0, 0, b)); r2.push_back(L(2, 1, b)); }
      if (k == 1) { r1.push_back(L(0, 1, b)); r2.push_back(L(2, 0, b)); }
      if (k == 2) { r1.push_back(L(1, 0, b)); r2.push_back(L(3, 1, b)); }
      if (k == 3) { r1.push_back(L(1, 1, b)); r2.push_back(L(3, 0, b)); }
    }
  o.r1 = pool.add(r1); o.r2 = pool.add(r2);
}

void measure_resolve(const PtrPool& P, const MeasureOff& o, MeasurePlan& m) {
  m.tlA = P.dev<const cplx* const*>(o.tlA); m.tlB = P.dev<const cplx* const*>(o.tlB);
  m.w1A = P.dev<const cplx* const*>(o.w1A); m.blA = P.dev<const cplx* const*>(o.blA);
  m.blB = P.dev<const cplx* const*>(o.blB); m.aoB = P.dev<const cplx* const*>(o.aoB);
  m.rcA = P.dev<const cplx* const*>(o.rcA); m.rcB = P.dev<const cplx* const*>(o.rcB);
  m.rcC = P.dev<const cplx* const*>(o.rcC);
  m.r1 = P.dev<const cplx* const*>(o.r1); m.r2 = P.dev<const cplx* const*>(o.r2);
}

int measure_run(Ctx& c, MeasureWork& w, const MeasurePlan& m, double* host_out) {
  const int B = c.B, chi = c.chi, D2 = c.D2, d = c.d;
  const long long T = (long long)chi * D2 * chi;
  cudaStream_t st = c.st;
  int rc;
  const int D = c.D, D3 = D * D * D, dD = d * D;
  const long long akper = (long long)D3 * dD, chi2 = (long long)chi * chi;
  for (int f = 0; f < 4; ++f)
    for (int l = 0; l < 2; ++l) {
      const cplx* A = l == 0 ? c.Aph : c.Bph;
      const size_t off = (size_t)(f * 2 + l) * B * akper;
      const int blocks = (int)std::min<long long>((B * akper + 255) / 256, 152 * 4);
      IPEPS_LAUNCH(K_KET_LAYER, 0, st,
                   ket_layer_kernel<<<blocks, 256, 0, st>>>(A, d, D, B, w.ak + off, w.akc + off, f));
      IPEPS_CUDA_TRY(cudaGetLastError());
    }
  // left halves, in passes of w.group jobs (job = (f * 2 + l) * B + b)
  const long long Lper = (long long)chi * chi * d * d * D2;
  for (int j0 = 0; j0 < 8 * B; j0 += w.group) {
    const int G = std::min(w.group, 8 * B - j0);
    GemmDesc g = gdm(chi, D2 * chi, chi, G);             // tl = C1 T1
    g.Aptr = m.tlA + j0; g.lda = chi; g.Bptr = m.tlB + j0; g.ldb = D2 * chi; g.C = w.tl; g.sC = T;
    g.ldc = D2 * chi;
    if ((rc = zgemm_f64(g, st))) return rc;
    g = gdm(chi * D2, D2 * chi, chi, G);                 // W1 = T4 tl -> [c4d][kL][kU][c1r]
    g.Aptr = m.w1A + j0; g.lda = chi; g.B = w.tl; g.sB = T; g.ldb = D2 * chi; g.C = w.W1; g.sC = T * D2;
    g.ldc = D2 * chi;
    if ((rc = zgemm_f64(g, st))) return rc;
    g = gdm(chi * D2, chi, chi, G);                      // bl = T3 C4 -> [e3r][kD][c4d]
    g.Aptr = m.blA + j0; g.lda = chi; g.Bptr = m.blB + j0; g.ldb = chi; g.C = w.bl; g.sC = T; g.ldc = chi;
    if ((rc = zgemm_f64(g, st))) return rc;
    g = gdm(chi * D2, D2 * D2 * chi, chi, G);            // W2 = bl W1 -> [e3r][kD][kL][kU][c1r]
    g.A = w.bl; g.sA = T; g.lda = chi; g.B = w.W1; g.sB = T * D2; g.ldb = (long long)D2 * D2 * chi;
    g.C = w.W2; g.sC = T * D2 * D2; g.ldc = (long long)D2 * D2 * chi;
    if ((rc = zgemm_f64(g, st))) return rc;
    {
      // W2 [e3r][uD bD][uL bL][uU bU][c1r] -> W2p [e3r][c1r][bU bL bD][uU uL uD]
      const int dims[8] = {chi, D, D, D, D, D, D, chi}, perm[8] = {0, 7, 6, 4, 2, 5, 3, 1};
      if ((rc = permute_c128(w.W2, w.W2p, 8, dims, perm, G, T * D2 * D2, T * D2 * D2, st))) return rc;
    }
    // ket layer: X[(e3r c1r bU bL bD), (s uR)] = W2p . Ak
    g = gdm(chi * chi * D3, dD, D3, G);
    g.A = w.W2p; g.sA = T * D2 * D2; g.lda = D3;
    g.Bptr = m.aoB + j0; g.ldb = dD;
    g.C = w.X; g.sC = chi2 * D3 * dD; g.ldc = dD;
    if ((rc = zgemm_f64(g, st))) return rc;
    // bra layer, per job and (e3r c1r): Y[(s uR), (s' bR)] = X^T conj(Ak)
    for (int jj = 0; jj < G; ++jj) {
      g = gdm(dD, dD, D3, chi * chi);
      g.opA = OP_T; g.A = w.X + (size_t)jj * chi2 * D3 * dD; g.sA = (long long)D3 * dD; g.lda = dD;
      g.B = w.akc + (size_t)(j0 + jj) * akper; g.sB = 0; g.ldb = dD;
      g.C = w.Y + (size_t)jj * chi2 * dD * dD; g.sC = (long long)dD * dD; g.ldc = dD;
      if ((rc = zgemm_f64(g, st))) return rc;
    }
    {
      // Y [p][s][uR][s'][bR] -> Lh [p][s][s'][uR bR]
      const int dims[5] = {chi * chi, d, D, d, D}, perm[5] = {0, 1, 3, 2, 4};
      if ((rc = permute_c128(w.Y, w.Lh + (size_t)j0 * Lper, 5, dims, perm, G, chi2 * dD * dD, Lper, st)))
        return rc;
    }
  }
  GemmDesc g;
  // right column C2 T2 C3 at (0,0) and (1,0)
  g = gdm(chi, D2 * chi, chi, 2 * B);
  g.Aptr = m.rcA; g.lda = chi; g.Bptr = m.rcB; g.ldb = D2 * chi; g.C = w.RCt; g.sC = T; g.ldc = D2 * chi;
  if ((rc = zgemm_f64(g, st))) return rc;
  g = gdm(chi * D2, chi, chi, 2 * B);
  g.A = w.RCt; g.sA = T; g.lda = chi; g.Bptr = m.rcC; g.ldb = chi; g.C = w.RC; g.sC = T; g.ldc = chi;
  if ((rc = zgemm_f64(g, st))) return rc;
  IPEPS_LAUNCH(K_RHO1, 8.0 * 2 * B * d * d * (double)chi * chi * D2, st,
               rho1_kernel<<<2 * B, 256, 0, st>>>(w.Lh, w.RC, chi, D2, d, w.rho1));
  IPEPS_CUDA_TRY(cudaGetLastError());
  IPEPS_LAUNCH(K_RHO2, 8.0 * 4 * B * d * d * d * d * (double)chi * chi * D2, st,
               rho2_kernel<<<4 * B * d * d * d * d, 256, 0, st>>>(m.r1, m.r2, chi, D2, d, w.rho2));
  IPEPS_CUDA_TRY(cudaGetLastError());
  IPEPS_LAUNCH(K_OBS, 0, st, observables_kernel<<<B, 32, 0, st>>>(w.rho1, w.rho2, c.bondop, c.dh, B, d, c.dA, w.obs));
  IPEPS_CUDA_TRY(cudaGetLastError());
  IPEPS_CUDA_TRY(cudaMemcpyAsync(host_out, w.obs, sizeof(double) * kObsPerInstance * B, cudaMemcpyDeviceToHost, st));
  IPEPS_CUDA_TRY(cudaStreamSynchronize(st));
  return 0;
}

}  // namespace ipeps
