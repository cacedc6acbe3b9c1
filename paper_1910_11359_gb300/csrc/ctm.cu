// Directional CTMRG with full 2x2-block projectors on the device (paper Sec. "Set up for iPEPS",
// Readout, and Appendix: CTMRG of Orus & Vidal 2009 / Orus 2012, chi >= D^2, converged environment;
// projectors of Corboz, Rice & Troyer, PRL 113, 046402 (2014)).
//
// Conventions (shared with the rest of the library):
//   double layer a[U, L, D, R], each index ket * D + bra (dimension D2 = D^2), rotations
//   rot^k(a)[i0..i3] = a[i_k .. i_{k+3}] (90-degree counter-clockwise relabellings);
//   corners C1[c_T4, c_T1], C2[c_T1, c_T2], C3[c_T2, c_T3], C4[c_T3, c_T4];
//   edges T1[left, k, right], T2[up, k, down], T3[right, k, left], T4[down, k, up]
//   (clockwise walk: the last index of each tensor joins the first index of the next).
// A counter-clockwise rotation of the lattice maps (x, y) -> (y, -x), C_i -> C_{i-1}, T_i -> T_{i-1}
// with no index permutation, so every directional move is the left move in a rotated frame f:
// logical tensor X_i at logical position q is physical X_{(i + f) mod 4} at position rot^{-f}(q), and
// the logical site tensor there is rot^f of the physical one.  On the 2 x 2 cell rot^{-f} swaps x
// and y for odd f.
//
// Left move at logical column x, for both cuts y (between rows y and y+1) at once:
//   enlarged corners Q_i (i = 0..3: the block's top-left, top-right, bottom-right, bottom-left):
//     Q_i[(e_ccw, k_row), (e_cw, k_col)] = T_ccw[e_ccw, kA, c] C[c, c'] T_cw[c', kB, e_cw]
//                                          rot^i(a)[kB, kA, k_row, k_col]
//   R~ = Q_0 Q_1, R = Q_2 Q_3, M = R R~ = U S V^+ (contracted over the cut), truncated to chi:
//     P = R~ V S^{-1/2} (lower side of the cut), P~ = S^{-1/2} U^+ R (upper side)
//   C1'(x+1, y) = P~[y-1] (C1 T1),  T4'(x+1, y) = P~[y] (T4 a) P[y-1],  C4'(x+1, y) = (T3 C4) P[y],
//   each divided by its largest modulus.
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "model.cuh"
#include "orth.cuh"
#include "prof.cuh"
#include "reduce.cuh"
#include "tc_gemm.cuh"

namespace ipeps {

constexpr int kOrthMinRows = 400;   // subspace blocks of at least this many rows use Cholesky QR

static inline int rot_pos(int pos, int f) {   // physical position of logical position `pos` in frame f
  return (f & 1) ? pos_of(pos >> 1, pos & 1) : pos;
}

void ctm_carve(Ctx& c) {
  Arena& a = c.arena;
  const int B = c.B;
  const long long N2 = c.N2(), Nc = (long long)c.N * c.chi, chi2 = (long long)c.chi * c.chi;
  const long long T = (long long)c.chi * c.D2 * c.chi;
  c.Aph = a.take<cplx>((size_t)B * c.d * c.D2 * c.D2);
  c.Bph = a.take<cplx>((size_t)B * c.d * c.D2 * c.D2);
  c.arot = a.take<cplx>((size_t)2 * 4 * B * c.D8());
  for (int i = 0; i < 4; ++i)
    for (int p = 0; p < NPOS; ++p) {
      c.Cenv[i][p] = a.take<cplx>((size_t)B * chi2);
      c.Tenv[i][p] = a.take<cplx>((size_t)B * T);
    }
  CtmWork& w = c.w;
  w.X1 = a.take<cplx>((size_t)8 * B * Nc);
  w.X2 = a.take<cplx>((size_t)8 * B * N2);
  w.X2p = a.take<cplx>((size_t)8 * B * N2);
  w.Y = a.take<cplx>((size_t)8 * B * N2);
  w.Q = a.take<cplx>((size_t)8 * B * N2);
  w.H = a.take<cplx>((size_t)4 * B * N2);
  w.M = a.take<cplx>((size_t)2 * B * N2);
  w.U = a.take<cplx>((size_t)2 * B * N2);
  w.V = a.take<cplx>((size_t)2 * B * N2);
  w.S = a.take<double>((size_t)2 * B * c.N);
  w.Us = a.take<cplx>((size_t)2 * B * Nc);
  w.Vs = a.take<cplx>((size_t)2 * B * Nc);
  w.P = a.take<cplx>((size_t)2 * B * Nc);
  w.Pt = a.take<cplx>((size_t)2 * B * Nc);
  w.Z1 = a.take<cplx>((size_t)2 * B * N2);
  w.Z1p = a.take<cplx>((size_t)2 * B * N2);
  w.Z2 = a.take<cplx>((size_t)2 * B * N2);
  w.Z2p = a.take<cplx>((size_t)2 * B * N2);
  w.T4n = a.take<cplx>((size_t)2 * B * T);
  w.W1 = a.take<cplx>((size_t)2 * B * T);
  w.W1p = a.take<cplx>((size_t)2 * B * T);
  w.C1n = a.take<cplx>((size_t)2 * B * chi2);
  w.C4n = a.take<cplx>((size_t)2 * B * chi2);
  w.kept = a.take<int>((size_t)2 * B);
  w.cs = a.take<double>((size_t)16 * B * c.chi);
  w.prev = a.take<double>((size_t)16 * B * c.chi);
  w.delta = a.take<double>(B);
  w.frozen = a.take<int>(B);
  w.sweeps = a.take<int>(B);
  w.have_prev = a.take<int>(1);
  w.best = a.take<double>(B);
  w.since = a.take<int>(B);
  const long long Nk = (long long)c.N * c.k, kk = (long long)c.k * c.k;
  w.Vfin = a.take<cplx>((size_t)8 * 2 * B * Nk);
  w.Vw = a.take<cplx>((size_t)2 * B * Nk);
  w.Ysub = a.take<cplx>((size_t)2 * B * Nk);
  w.Uy = a.take<cplx>((size_t)2 * B * Nk);
  w.W = a.take<cplx>((size_t)2 * B * kk);
  w.Zsub = a.take<cplx>((size_t)2 * B * Nk);
  w.Vz = a.take<cplx>((size_t)2 * B * Nk);
  w.Sy = a.take<double>((size_t)2 * B * c.k);
  w.Sz = a.take<double>((size_t)2 * B * c.k);
  w.sub_done = a.take<int>((size_t)2 * B);
  w.sub_rounds = a.take<int>((size_t)2 * B);
  w.sub_res = a.take<double>((size_t)2 * B);
  // Cholesky QR pays off for tall blocks: its k x k factorisations are a fixed chain of ~2k
  // dependent steps, while the tall Jacobi's cost per round grows with N (measured: D = 3,
  // N = 162, tall Jacobi faster; D >= 4, N >= 512, Cholesky QR 1.4-1.6x faster per sweep)
  c.orth = c.subspace && c.N >= kOrthMinRows && orth_supported(c.k) && jacobi_svd_fits(c.k, c.k);
  w.orth_work = nullptr; w.orth_bytes = 0;
  w.Uq = w.Bk = w.Xk = w.part = nullptr;
  w.ofail = a.take<int>((size_t)2 * B);
  w.skip_new = a.take<int>((size_t)2 * B);
  w.skip_old = a.take<int>((size_t)2 * B);
  if (c.orth) {
    w.orth_bytes = orth_work_bytes(c.N, c.k, 2 * B);
    w.orth_work = a.take<unsigned char>(w.orth_bytes);
    w.Uq = a.take<cplx>((size_t)2 * B * Nk);
    w.Bk = a.take<cplx>((size_t)2 * B * kk);
    w.Xk = a.take<cplx>((size_t)2 * B * kk);
    w.part = a.take<cplx>((size_t)2 * B * ((c.N + 63) / 64) * kk);
  }
  w.jgwork = nullptr;
  w.jgwork_bytes = 0;
  if (c.subspace && !jacobi_svd_fits(c.N, c.k)) {
    w.jgwork_bytes = jacobi_svd_global_bytes(c.N, c.k, 2 * B);
    w.jgwork = a.take<cplx>(w.jgwork_bytes / sizeof(cplx));
  }
  if (c.precision != 0) {
    // largest split product of a left move: corner GEMM 3 / edge GEMM (chi^2 x D2^2 x D2^2, 8B),
    // halves (N^3, 4B), M (N^3, 2B), projectors (N chi N, 2B), edge absorption (chi D2chi N, 2B)
    const int D2 = c.D2, chi = c.chi, N = c.N;
    size_t mx = 0;
    const long long shapes[][4] = {{(long long)chi * chi, D2 * D2, D2 * D2, 8 * B},
                                   {N, N, N, 4 * B}, {N, N, N, 2 * B}, {N, chi, N, 2 * B},
                                   {chi, N, N, 2 * B}, {chi, (long long)D2 * chi, N, 2 * B},
                                   {(long long)chi * D2, (long long)D2 * chi, chi, 8 * B}};
    for (auto& sh : shapes) {
      const size_t b = tc::split_workspace_bytes((int)sh[0], (int)sh[1], (int)sh[2], (int)sh[3],
                                                 c.precision == 2 ? tc::SPLIT_TF32 : tc::SPLIT_BF16);
      mx = b > mx ? b : mx;
    }
    c.tcwork_bytes = mx;
    c.tcwork = a.take<unsigned char>(mx);
  }
}

void ctm_build_plans(Ctx& c) {
  const int B = c.B, chi = c.chi, D2 = c.D2;
  const long long N2 = c.N2(), Nc = (long long)c.N * chi, chi2 = (long long)chi * chi;
  const long long T = (long long)chi * D2 * chi;
  PtrPool& pool = c.pool;
  CtmWork& w = c.w;
  auto Cp = [&](int i, int pos, int b) -> const void* { return c.Cenv[i & 3][pos] + (size_t)b * chi2; };
  auto Tp = [&](int i, int pos, int b) -> const void* { return c.Tenv[i & 3][pos] + (size_t)b * T; };
  for (int f = 0; f < 4; ++f)
    for (int x = 0; x < 2; ++x) {
      MoveOff& o = c.off.mv[f][x];
      std::vector<const void*> g1A, g1B, g1C, g2A, g2B, g2C, g3B;
      for (int y = 0; y < 2; ++y)
        for (int i = 0; i < 4; ++i)
          for (int b = 0; b < B; ++b) {
            const int lx[4] = {x, x + 1, x + 1, x}, ly[4] = {y, y, y + 1, y + 1};
            const int pp = rot_pos(pos_of(lx[i], ly[i]), f);
            const int slot = (y * 4 + i) * B + b;
            g1A.push_back(Cp(i + f, pp, b));
            g1B.push_back(Tp(i + f, pp, b));
            g1C.push_back(w.X1 + (size_t)slot * Nc);
            g2A.push_back(Tp(i + 3 + f, pp, b));
            g2B.push_back(w.X1 + (size_t)slot * Nc);
            g2C.push_back(w.X2 + (size_t)slot * N2);
            g3B.push_back(c.a_rot(site_of(pp), (i + f) & 3) + (size_t)b * c.D8());
          }
      o.g1A = pool.add(g1A); o.g1B = pool.add(g1B); o.g1C = pool.add(g1C);
      o.g2A = pool.add(g2A); o.g2B = pool.add(g2B); o.g2C = pool.add(g2C);
      o.g3B = pool.add(g3B);
      std::vector<const void*> hA, hB, hC;
      for (int half = 0; half < 2; ++half)          // 0: R~ = Q0 Q1, 1: R = Q2 Q3
        for (int y = 0; y < 2; ++y)
          for (int b = 0; b < B; ++b) {
            const int s0 = (y * 4 + 2 * half) * B + b, s1 = (y * 4 + 2 * half + 1) * B + b;
            hA.push_back(w.Q + (size_t)s0 * N2);
            hB.push_back(w.Q + (size_t)s1 * N2);
            hC.push_back(w.H + (size_t)((half * 2 + y) * B + b) * N2);
          }
      o.hA = pool.add(hA); o.hB = pool.add(hB); o.hC = pool.add(hC);
      std::vector<const void*> c1A, c1B, z1A, z1B, z2B, t4A, w1A, w1B, c4B, sC1, sT4, sC4;
      for (int y = 0; y < 2; ++y)
        for (int b = 0; b < B; ++b) {
          const int ym = (y + 1) & 1;   // y - 1 on the two-row cell
          const int pp = rot_pos(pos_of(x, y), f);
          const int npp = rot_pos(pos_of(x + 1, y), f);
          c1A.push_back(w.Pt + (size_t)(ym * B + b) * Nc);
          c1B.push_back(w.X1 + (size_t)((y * 4 + 0) * B + b) * Nc);
          z1A.push_back(Tp(3 + f, pp, b));
          z1B.push_back(w.P + (size_t)(ym * B + b) * Nc);
          z2B.push_back(c.a_rot(site_of(pp), f & 3) + (size_t)b * c.D8());
          t4A.push_back(w.Pt + (size_t)(y * B + b) * Nc);
          w1A.push_back(Tp(2 + f, pp, b));
          w1B.push_back(Cp(3 + f, pp, b));
          c4B.push_back(w.P + (size_t)(y * B + b) * Nc);
          sC1.push_back(Cp(0 + f, npp, b));
          sT4.push_back(Tp(3 + f, npp, b));
          sC4.push_back(Cp(3 + f, npp, b));
        }
      o.c1A = pool.add(c1A); o.c1B = pool.add(c1B); o.z1A = pool.add(z1A); o.z1B = pool.add(z1B);
      o.z2B = pool.add(z2B); o.t4A = pool.add(t4A); o.w1A = pool.add(w1A); o.w1B = pool.add(w1B);
      o.c4B = pool.add(c4B); o.sC1 = pool.add(sC1); o.sT4 = pool.add(sT4); o.sC4 = pool.add(sC4);
    }
  std::vector<const void*> csA, csS, pA, pU, pS, pV, envC, envT;
  for (int i = 0; i < 4; ++i)
    for (int p = 0; p < NPOS; ++p)
      for (int b = 0; b < B; ++b) {
        csA.push_back(Cp(i, p, b));
        csS.push_back(w.cs + (size_t)((i * NPOS + p) * B + b) * chi);
        envC.push_back(Cp(i, p, b));
        envT.push_back(Tp(i, p, b));
      }
  for (int q = 0; q < 2 * B; ++q) {
    pA.push_back(w.M + (size_t)q * N2);
    pU.push_back(w.U + (size_t)q * N2);
    pS.push_back(w.S + (size_t)q * c.N);
    pV.push_back(w.V + (size_t)q * N2);
  }
  c.off.csA = pool.add(csA); c.off.csS = pool.add(csS);
  c.off.pA = pool.add(pA); c.off.pU = pool.add(pU); c.off.pS = pool.add(pS); c.off.pV = pool.add(pV);
  c.off.envC = pool.add(envC); c.off.envT = pool.add(envT);
  const long long Nk = (long long)c.N * c.k, kk = (long long)c.k * c.k;
  std::vector<const void*> yA, yU, yS, yV, zA, zU, zS;
  for (int q = 0; q < 2 * B; ++q) {
    yA.push_back(w.Ysub + (size_t)q * Nk);
    yU.push_back(w.Uy + (size_t)q * Nk);
    yS.push_back(w.Sy + (size_t)q * c.k);
    yV.push_back(w.W + (size_t)q * kk);
    zA.push_back(w.Zsub + (size_t)q * Nk);
    zU.push_back(w.Vz + (size_t)q * Nk);
    zS.push_back(w.Sz + (size_t)q * c.k);
  }
  c.off.yA = pool.add(yA); c.off.yU = pool.add(yU); c.off.yS = pool.add(yS); c.off.yV = pool.add(yV);
  c.off.zA = pool.add(zA); c.off.zU = pool.add(zU); c.off.zS = pool.add(zS);
  std::vector<const void*> bA, bU;
  for (int q = 0; q < 2 * B; ++q) {
    bA.push_back(w.Bk ? w.Bk + (size_t)q * kk : nullptr);
    bU.push_back(w.Xk ? w.Xk + (size_t)q * kk : nullptr);
  }
  c.off.bA = pool.add(bA); c.off.bU = pool.add(bU);
}

void ctm_resolve_plans(Ctx& c) {
  const PtrPool& P = c.pool;
  for (int f = 0; f < 4; ++f)
    for (int x = 0; x < 2; ++x) {
      const MoveOff& o = c.off.mv[f][x];
      MovePlan& m = c.plan[f][x];
      m.g1A = P.dev<const cplx* const*>(o.g1A); m.g1B = P.dev<const cplx* const*>(o.g1B);
      m.g1C = P.dev<cplx* const*>(o.g1C);
      m.g2A = P.dev<const cplx* const*>(o.g2A); m.g2B = P.dev<const cplx* const*>(o.g2B);
      m.g2C = P.dev<cplx* const*>(o.g2C);
      m.g3B = P.dev<const cplx* const*>(o.g3B);
      m.hA = P.dev<const cplx* const*>(o.hA); m.hB = P.dev<const cplx* const*>(o.hB);
      m.hC = P.dev<cplx* const*>(o.hC);
      m.c1A = P.dev<const cplx* const*>(o.c1A); m.c1B = P.dev<const cplx* const*>(o.c1B);
      m.z1A = P.dev<const cplx* const*>(o.z1A); m.z1B = P.dev<const cplx* const*>(o.z1B);
      m.z2B = P.dev<const cplx* const*>(o.z2B); m.t4A = P.dev<const cplx* const*>(o.t4A);
      m.w1A = P.dev<const cplx* const*>(o.w1A); m.w1B = P.dev<const cplx* const*>(o.w1B);
      m.c4B = P.dev<const cplx* const*>(o.c4B);
      m.sC1 = P.dev<cplx* const*>(o.sC1); m.sT4 = P.dev<cplx* const*>(o.sT4);
      m.sC4 = P.dev<cplx* const*>(o.sC4);
    }
  c.w.csA = P.dev<const cplx* const*>(c.off.csA);
  c.w.csS = P.dev<double* const*>(c.off.csS);
  c.w.pA = P.dev<const cplx* const*>(c.off.pA);
  c.w.pU = P.dev<cplx* const*>(c.off.pU);
  c.w.pS = P.dev<double* const*>(c.off.pS);
  c.w.pV = P.dev<cplx* const*>(c.off.pV);
  c.w.envC = P.dev<cplx* const*>(c.off.envC);
  c.w.envT = P.dev<cplx* const*>(c.off.envT);
  c.w.yA = P.dev<const cplx* const*>(c.off.yA); c.w.yU = P.dev<cplx* const*>(c.off.yU);
  c.w.yS = P.dev<double* const*>(c.off.yS); c.w.yV = P.dev<cplx* const*>(c.off.yV);
  c.w.zA = P.dev<const cplx* const*>(c.off.zA); c.w.zU = P.dev<cplx* const*>(c.off.zU);
  c.w.zS = P.dev<double* const*>(c.off.zS);
  c.w.bA = P.dev<const cplx* const*>(c.off.bA); c.w.bU = P.dev<cplx* const*>(c.off.bU);
}

// ----------------------------------------------------------------------------- small kernels
// Initial environment: each neighbour's double layer with its outward ket/bra legs traced, zero-
// padded to chi.  Neighbour offsets: C1 (-1,-1) C2 (1,-1) C3 (1,1) C4 (-1,1) T1 (0,-1) T2 (1,0)
// T3 (0,1) T4 (-1,0).  Grid: (kind 0..7, pos, b).
__global__ void env_init_kernel(const cplx* a0A, const cplx* a0B, int B, int D, int chi,
                                cplx* const* Cout, cplx* const* Tout) {
  const int D2 = D * D;
  const int job = blockIdx.x;
  const int b = job % B, pos = (job / B) % NPOS, kind = job / (B * NPOS);
  const int x = pos & 1, y = pos >> 1;
  const int dxs[8] = {-1, 1, 1, -1, 0, 1, 0, -1};
  const int dys[8] = {-1, -1, 1, 1, -1, 0, 1, 0};
  const int spos = pos_of(x + dxs[kind] + 2, y + dys[kind] + 2);
  const long long D8 = (long long)D2 * D2 * D2 * D2;
  const cplx* a = (site_of(spos) == 0 ? a0A : a0B) + (size_t)b * D8;
  const int D1 = D + 1;
#define A4(u, l, d, r) a[(((long long)(u) * D2 + (l)) * D2 + (d)) * D2 + (r)]
  if (kind < 4) {
    cplx* out = Cout[(kind * NPOS + pos) * B + b];
    for (int idx = threadIdx.x; idx < chi * chi; idx += blockDim.x) {
      const int i = idx / chi, j = idx % chi;
      cplx acc = cmk(0.0, 0.0);
      if (i < D2 && j < D2)
        for (int t1 = 0; t1 < D; ++t1)
          for (int t2 = 0; t2 < D; ++t2) {
            const int p = t1 * D1, q = t2 * D1;
            if (kind == 0) acc = cadd(acc, A4(p, q, i, j));         // C1[D, R], trace U, L
            else if (kind == 1) acc = cadd(acc, A4(p, i, j, q));    // C2[L, D], trace U, R
            else if (kind == 2) acc = cadd(acc, A4(i, j, p, q));    // C3[U, L], trace D, R
            else acc = cadd(acc, A4(j, p, q, i));                   // C4[R, U], trace L, D
          }
      out[idx] = acc;
    }
  } else {
    const int e = kind - 4;
    cplx* out = Tout[(e * NPOS + pos) * B + b];
    for (int idx = threadIdx.x; idx < chi * D2 * chi; idx += blockDim.x) {
      const int i = idx / (D2 * chi), k = (idx / chi) % D2, j = idx % chi;
      cplx acc = cmk(0.0, 0.0);
      if (i < D2 && j < D2)
        for (int t1 = 0; t1 < D; ++t1) {
          const int p = t1 * D1;
          if (e == 0) acc = cadd(acc, A4(p, i, k, j));              // T1[L, D, R], trace U
          else if (e == 1) acc = cadd(acc, A4(i, k, j, p));         // T2[U, L, D], trace R
          else if (e == 2) acc = cadd(acc, A4(k, j, p, i));         // T3[R, U, L], trace D
          else acc = cadd(acc, A4(j, p, i, k));                     // T4[D, R, U], trace L
        }
      out[idx] = acc;
    }
  }
#undef A4
}

// Projector truncation: singular values of M = R R~ below c.cut_rel (default 1e-10) of the largest
// are dropped.  Rounding in the singular vectors of M is amplified by ~ eps s_1 / (s_K gap) in the
// projectors; a larger cutoff (e.g. 1e-6) trades a small truncation bias for a fixed point that does
// not depend on rounding when the cut falls in a cluster of tiny singular values.

// Projector factors from the SVD of M: rank K (multiplets at the cut kept whole, values below
// cut_rel of the largest dropped), Vs = V[:, :K] S^{-1/2}, Us = U[:, :K] S^{-1/2}, zero-padded to chi.
// Two values at the cut form a multiplet when their relative gap is below degen_rtol or their
// absolute gap below degen_abs * s_1: a computed singular value is accurate to about eps * s_1, so
// for small values a purely relative test would decide on rounding noise.
constexpr double kDegenRtol = 1e-10, kDegenAbs = 1e-11, kTinyRel = 1e-14;

__global__ void proj_prep_kernel(const double* S, long long s_stride, int ns, const cplx* U,
                                 const cplx* V, int N, int chi, long long ldu, long long stride_uv,
                                 cplx* Us, cplx* Vs, int* kept, double degen_rtol, double degen_abs,
                                 double tiny_rel, double cut_rel, const int* frozen, int B,
                                 const int* done = nullptr, unsigned long long* ctr = nullptr) {
  // S: ns singular values (descending) per problem; U, V: N x (>= chi) with leading dimension ldu
  const int q = blockIdx.x;
  if (skipped(frozen, B, q)) return;
  const double* s = S + (size_t)q * s_stride;
  __shared__ int sK;
  if (threadIdx.x == 0) {
    int K = chi < ns ? chi : ns;
    while (K > 1 && K < ns && s[K] > tiny_rel * s[0] &&
           (s[K - 1] / s[K] - 1.0 < degen_rtol || s[K - 1] - s[K] < degen_abs * s[0]))
      --K;
    int cnt = 0;
    for (int j = 0; j < K; ++j) cnt += s[j] > cut_rel * s[0];
    K = cnt < K ? cnt : K;
    if (!(s[0] > 0.0)) K = 0;
    else if (K < 1) K = 1;
    sK = K;
    kept[q] = K;
    if (done && ctr && !done[q]) atomicAdd(ctr + CTR_SUB_UNCONVERGED, 1ull);
  }
  __syncthreads();
  const int K = sK;
  const cplx* Uq = U + (size_t)q * stride_uv;
  const cplx* Vq = V + (size_t)q * stride_uv;
  cplx* Uo = Us + (size_t)q * N * chi;
  cplx* Vo = Vs + (size_t)q * N * chi;
  // Phase convention: the largest-magnitude entry of every kept u_j is made real and positive
  // (u_j and v_j are multiplied by the same phase, so M = U S V^+ is unchanged).  It removes the
  // arbitrary phases of the SVD from the new environment, so that consecutive sweeps produce
  // nearly equal environment tensors once CTMRG settles and the warm-started subspace iteration
  // of the next sweep starts close to its answer.
  extern __shared__ double ph[];                 // [chi][2]: conj of the phase of column j
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int j = warp; j < K; j += nwarps) {
    double best = -1.0;
    int bi = 0;
    for (int i = lane; i < N; i += 32) {
      const double v = cabs2(Uq[(size_t)i * ldu + j]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) {
      const cplx u = Uq[(size_t)bi * ldu + j];
      const double a = sqrt(cabs2(u));
      ph[2 * j] = a > 0.0 ? u.x / a : 1.0;
      ph[2 * j + 1] = a > 0.0 ? -u.y / a : 0.0;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * chi; idx += blockDim.x) {
    const int i = idx / chi, j = idx % chi;
    if (j < K) {
      const double f = 1.0 / sqrt(s[j]);
      const cplx e = cmk(ph[2 * j] * f, ph[2 * j + 1] * f);
      Uo[idx] = cmul(Uq[(size_t)i * ldu + j], e);
      Vo[idx] = cmul(Vq[(size_t)i * ldu + j], e);
    } else {
      Uo[idx] = cmk(0.0, 0.0);
      Vo[idx] = cmk(0.0, 0.0);
    }
  }
}

// counter-based uniform draws in [-1, 1): splitmix64 of (seed, stream, index)
__device__ __forceinline__ double rand_unit(unsigned long long seed, unsigned long long stream,
                                            unsigned long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (stream * 0x100000001B3ull + i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Starting block of the subspace iteration: the slot's previous right vectors, or random columns
// on the slot's first use.  Columns of `src` whose singular value (sv, may be null) is not above
// tiny * sv[0] are refilled with random columns so the block keeps full rank.
__global__ void sub_fill_kernel(const cplx* src, const double* sv, int N, int k, int random_all,
                                unsigned long long seed, unsigned long long stream, cplx* dst,
                                const int* skip = nullptr, int B = 1) {
  const int q = blockIdx.x;
  if (skip && skip[q]) return;
  // the draws depend on the cut (q / B) and the element only, never on the instance's place in
  // the batch, so an instance gets the same random columns alone and in any batch
  const unsigned long long cut = (unsigned long long)(q / B);
  const cplx* sq = src ? src + (size_t)q * N * k : nullptr;
  const double* s = sv ? sv + (size_t)q * k : nullptr;
  cplx* dq = dst + (size_t)q * N * k;
  for (int idx = threadIdx.x; idx < N * k; idx += blockDim.x) {
    const int j = idx % k;
    const bool fresh = random_all || (s && !(s[j] > 1e-300 && s[j] > 1e-15 * s[0]));
    if (fresh) {
      const unsigned long long id = (cut * N * k + idx) * 2;
      dq[idx] = cmk(rand_unit(seed, stream, id), rand_unit(seed, stream, id + 1));
    } else {
      dq[idx] = sq[idx];
    }
  }
}

// Divide each new tensor by its largest modulus and store it into its environment slot, except for
// instances whose environment has already converged.  Grid: (tensor kind 0..2, problem q < 2B).
__global__ void normalize_store_kernel(const cplx* C1n, const cplx* T4n, const cplx* C4n, int B,
                                       long long nC, long long nT, cplx* const* sC1, cplx* const* sT4,
                                       cplx* const* sC4, const int* frozen, unsigned* err) {
  const int kind = blockIdx.x / (2 * B), q = blockIdx.x % (2 * B), b = q % B;
  if (frozen[b]) return;
  const long long n = kind == 1 ? nT : nC;
  const cplx* src = (kind == 0 ? C1n : kind == 1 ? T4n : C4n) + (size_t)q * n;
  cplx* dst = (kind == 0 ? sC1 : kind == 1 ? sT4 : sC4)[q];
  double m = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, cabs2(src[i]));
  const double mx = sqrt(block_max<256>(m));
  if (!isfinite(mx) && threadIdx.x == 0) atomicOr(err, (unsigned)DEV_NONFINITE);
  const double f = mx > 0.0 ? 1.0 / mx : 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) dst[i] = cscale(src[i], f);
}

// Convergence number per instance: max over the 16 corners of || s/s_1 - s_prev/s_1,prev ||_2.
// first != 0 only records the spectra of the starting environment.  An instance is frozen (its
// environment no longer updated) once delta < tol, or once delta has stalled at its rounding floor:
// no factor-2 improvement of the best delta for kStallWindow sweeps while that best and the current
// delta are below stall_max and the current delta is within kStallGrowth of the best
// ("sufficiently well converged", Appendix): stall_threshold(precision), 1e-7 on the FP64 path and
// higher on the split paths, whose contractions leave a noise floor.  A delta that grows again after
// coming close to a fixed point means the environment is leaving an unstable fixed point; the
// instance keeps sweeping.  tol <= 0 never freezes.
constexpr int kStallWindow = 10;
constexpr double kStallGrowth = 4.0;

__global__ void spectra_delta_kernel(const double* cs, double* prev, int B, int chi, int first,
                                     double tol, double stall_max, double* delta, int* frozen, int* sweeps,
                                     double* best, int* since) {
  const int b = blockIdx.x;
  __shared__ double dmax[16];
  const int c = threadIdx.x;
  if (frozen[b]) return;
  if (c < 16) {
    const double* s = cs + (size_t)(c * B + b) * chi;
    double* p = prev + (size_t)(c * B + b) * chi;
    const double s0 = s[0];
    double acc = 0.0;
    for (int k = 0; k < chi; ++k) {
      const double v = s0 > 0.0 ? s[k] / s0 : 0.0;
      const double dv = v - p[k];
      acc += dv * dv;
      p[k] = v;
    }
    dmax[c] = sqrt(acc);
  }
  __syncthreads();
  if (c != 0) return;
  if (first) {
    best[b] = INFINITY;
    since[b] = 0;
    return;
  }
  double m = 0.0;
  for (int k = 0; k < 16; ++k) m = fmax(m, dmax[k]);
  if (!(m == m)) m = INFINITY;
  delta[b] = m;
  sweeps[b] += 1;
  if (m < tol) {
    frozen[b] = 1;
    return;
  }
  if (m < 0.5 * best[b]) {
    best[b] = m;
    since[b] = 0;
  } else {
    since[b] += 1;
  }
  if (tol > 0.0 && since[b] >= kStallWindow && best[b] < stall_max && m < stall_max &&
      m <= kStallGrowth * best[b])
    frozen[b] = 1;
}

// ----------------------------------------------------------------------------- drivers
int ctm_prepare_tensors(Ctx& c) {
  if (int rc = physical_tensors(c.GA, c.GB, c.lam, c.Aph, c.Bph, c.d, c.D, c.B, c.st)) return rc;
  if (int rc = double_layers(c.Aph, c.a_rot(0, 0), c.d, c.D, c.B, 4, c.st)) return rc;
  if (int rc = double_layers(c.Bph, c.a_rot(1, 0), c.d, c.D, c.B, 4, c.st)) return rc;
  return 0;
}

int ctm_init_env(Ctx& c) {
  IPEPS_LAUNCH(K_ENV_INIT, 0, c.st,
               env_init_kernel<<<8 * NPOS * c.B, 256, 0, c.st>>>(c.a_rot(0, 0), c.a_rot(1, 0), c.B, c.D, c.chi,
                                                                 c.w.envC, c.w.envT));
  IPEPS_CUDA_TRY(cudaGetLastError());
  c.env_valid = true;
  for (int f = 0; f < 4; ++f)
    for (int x = 0; x < 2; ++x) c.slot_warm[f][x] = false;
  return 0;
}

// Contraction dispatcher: with precision = split BF16x3, products of at least kSplitMinWork complex
// multiply-adds per problem run on the tensor cores; everything else (and the FP64 path) uses the
// FP64 GEMM.  The choice depends on the problem's shape only, never on the batch size, so an
// instance gets the same arithmetic alone and in any batch.
constexpr double kSplitMinWork = 1 << 18;

static int contract(Ctx& c, const GemmDesc& g) {
  if (c.precision != 0 && (double)g.M * g.N * (double)g.K >= kSplitMinWork)
    return tc::zgemm_split(g, c.precision == 2 ? tc::SPLIT_TF32 : tc::SPLIT_BF16, c.tcwork, c.tcwork_bytes,
                           c.derr, c.st);
  return zgemm_f64(g, c.st);
}

static GemmDesc gd(int M, int N, int K, int batch) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.opA = OP_N; g.opB = OP_N;
  g.alpha = cmk(1.0, 0.0); g.beta = cmk(0.0, 0.0);
  return g;
}

// A product of a directional move, one problem per (slot, instance) with the instance index
// b = problem % B: instances whose environment has converged (frozen) are skipped.
static GemmDesc gdm(const Ctx& c, int M, int N, int K, int batch) {
  GemmDesc g = gd(M, N, K, batch);
  g.skip = c.w.frozen;
  g.skip_mod = c.B;
  return g;
}

// subspace problems q < 2B start "done" when their instance has converged
__global__ void sub_init_kernel(int* done, int* rounds, const int* frozen, int B) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 2 * B) {
    done[q] = frozen[q % B] ? 1 : 0;
    rounds[q] = 0;
  }
}

// Columns of Z = M^+ U_y with negligible norm (M has rank below k, or u_j is a zero column) are
// replaced by random columns before Z is orthonormalised, so the block keeps full rank.
__global__ void sub_refill_kernel(cplx* Z, int N, int k, unsigned long long seed,
                                  unsigned long long stream_base, const int* round_ctr, const int* skip,
                                  int B) {
  const int q = blockIdx.x;
  if (skip[q]) return;
  // draws of round r (the test kernel has already counted it: *round_ctr = r + 1)
  const unsigned long long stream = stream_base + (unsigned long long)(*round_ctr - 1);
  const unsigned long long cut = (unsigned long long)(q / B);   // batch-independent draws
  cplx* Zq = Z + (size_t)q * N * k;
  __shared__ double nrm[256];
  __shared__ double mx;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += cabs2(Zq[(size_t)i * k + j]);
    nrm[j] = sqrt(acc);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int j = 0; j < k; ++j) m = fmax(m, nrm[j]);
    mx = m;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * k; idx += blockDim.x) {
    const int j = idx % k;
    if (!(nrm[j] > 1e-300 && nrm[j] > 1e-13 * mx)) {
      const unsigned long long id = (cut * N * k + idx) * 2;
      Zq[idx] = cmk(rand_unit(seed, stream, id), rand_unit(seed, stream, id + 1));
    }
  }
}

// Convergence of the subspace iteration: with Y = M V = U_y S_y W^+ and V_f = V W (so that
// M v_j = s_j u_j holds by construction), the triplets are converged when M^+ u_j = s_j v_j too:
// residual_j = || (M^+ U_y)_j - s_j (V_f)_j || <= rtol * s_1 for the first min(k, chi + 1) columns
// (rtol = 1e-14, near the accuracy of a dense FP64 SVD: the projectors then stay within rounding
// of the exact ones, to which the readouts and corner spectra are compared).
__global__ void sub_residual_kernel(const cplx* Z, const cplx* Vf, const double* S, int N, int k,
                                    int ncheck, double rtol, double stag, int* done, int* rounds,
                                    double* prev, unsigned long long* ctr) {
  const int q = blockIdx.x;
  if (done[q]) return;
  const cplx* Zq = Z + (size_t)q * N * k;
  const cplx* Vq = Vf + (size_t)q * N * k;
  const double* s = S + (size_t)q * k;
  __shared__ double red[256];
  double worst = 0.0;
  for (int j = 0; j < ncheck; ++j) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const cplx r = csub(Zq[(size_t)i * k + j], cscale(Vq[(size_t)i * k + j], s[j]));
      acc += cabs2(r);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) worst = fmax(worst, red[0]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double r = sqrt(worst);
    // accepted at rtol, or once the residual has stopped shrinking (less than 10% per round) below
    // stag s_1: then it sits at the rounding floor of the small directions (slow convergence above
    // that level is not a floor and goes on iterating)
    if (r <= rtol * s[0] || (rounds[q] > 0 && r <= stag * s[0] && r >= 0.9 * prev[q])) {
      done[q] = 1;
      if (ctr) atomicAdd(ctr + CTR_SUB_ACCEPTED, 1ull);
    }
    prev[q] = r;
    rounds[q] += 1;
    if (ctr) atomicAdd(ctr + CTR_SUB_ROUNDS, 1ull);
  }
}

// Per-problem path flags after a Cholesky-QR orthonormalisation: problems whose factorisation
// broke down (fail) go to the tall Jacobi SVD (skip_old == 0), the others stay on the Cholesky-QR
// path (skip_new == 0); converged problems take neither.
__global__ void orth_route_kernel(const int* done, const int* fail, int* skip_new, int* skip_old, int n,
                                  unsigned long long* ctr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const bool dn = done[q] != 0, fl = fail[q] != 0;
  skip_new[q] = dn || fl;
  skip_old[q] = dn || !fl;
  if (!dn && fl && ctr) atomicAdd(ctr + CTR_ORTH_FALLBACK, 1ull);
}

// flag = 1 when every subspace problem has converged (or is skipped)
// End of a subspace round: counts it in *ctr, writes whether every problem has converged to *flag
// and (graph mode) continues the loop while some problem is open and fewer than `rounds` ran.
__global__ void sub_test_kernel(const int* done, int n, int* ctr, int rounds, cudaGraphConditionalHandle h,
                                int graph, int* flag) {
  __shared__ int any_open;
  if (threadIdx.x == 0) any_open = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x)
    if (!done[q]) any_open = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int r = *ctr + 1;
    *ctr = r;
    *flag = any_open ? 0 : 1;
    loop_set(h, graph, any_open && r < rounds);
  }
}

// eager mode: rounds after which the host reads back whether every problem has converged (a
// readback is a stream synchronisation, so they are spaced out geometrically)
static bool sub_checkpoint(int rounds_done) {
  const int marks[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48};
  for (int m : marks)
    if (rounds_done == m) return true;
  return false;
}

// Top-k SVD of M = R R~ (k = subspace_size(chi, N) < N/2) by block subspace iteration.  Each round: Y = M V,
// Y = U_y S_y W^+ (see below), V_f = V W (so that M v_j = s_j u_j holds by construction),
// Z = M^+ U_y; the triplets (U_y, S_y, V_f) are accepted once Z matches V_f S_y (residual test
// above); otherwise Z (negligible columns refilled at random) is orthonormalised into the next V.
// The SVD of the N x k block Y and the orthonormalisation of Z are done in one of two ways:
//  * Cholesky QR (c.orth: blocks of at least kOrthMinRows rows whose k x k factors fit): Y = U B
//    with U from column-scaled Cholesky QR
//    (orth.cu) and B = U^+ Y; the one-sided Jacobi SVD then runs on the k x k matrix
//    B = X S_y W^+ only, and U_y = U X; Z is orthonormalised by Cholesky QR alone.  A problem whose
//    factorisation breaks down (a start block far from orthonormal after column scaling) takes the
//    tall Jacobi SVD of that round instead.
//  * otherwise the one-sided Jacobi SVD of the N x k blocks themselves.
// Converged problems are skipped by every later launch.  The iteration starts from the slot's
// previous right vectors (random on the slot's first use); at most 40 rounds per call (60 on first
// use; converged problems make the later rounds' launches exit at once).  The round loop is a
// conditional WHILE node when a convergence graph is being captured (c.gb): the test kernel ends
// it on the device; eagerly, the host reads the same kernel's flag at the checkpoints.  The second
// half of a round (refill, orthonormalisation of Z into the next V) then also runs after the last
// round; it writes only the next start block, which nothing reads.
static int subspace_svd(Ctx& c, int f, int x, const cplx* R, const cplx* Rt) {
  CtmWork& w = c.w;
  const int B = c.B, N = c.N, k = c.k, chi = c.chi;
  const long long N2 = c.N2(), Nk = (long long)N * k, kk = (long long)k * k;
  cudaStream_t st = c.st;
  int rc;
  cplx* slot = w.Vfin + (size_t)(f * 2 + x) * 2 * B * Nk;
  const bool warm = c.slot_warm[f][x];
  const unsigned long long stream_id = (unsigned long long)(f * 2 + x);
  IPEPS_LAUNCH(K_PROJ_PREP, 0, st, sub_init_kernel<<<(2 * B + 127) / 128, 128, 0, st>>>(w.sub_done, w.sub_rounds,
                                                                                     w.frozen, B));
  IPEPS_LAUNCH(K_PROJ_PREP, 0, st,
               sub_fill_kernel<<<2 * B, 256, 0, st>>>(slot, nullptr, N, k, warm ? 0 : 1, c.seed,
                                                      stream_id, w.Vw, w.sub_done, B));
  const int rounds = warm ? 40 : 60;
  SvdDesc yd;
  yd.m = N; yd.n = k; yd.batch = 2 * B;
  yd.A = w.yA; yd.lda = k; yd.U = w.yU; yd.ldu = k; yd.S = w.yS; yd.V = w.yV; yd.ldv = k;
  yd.tol = 4e-16 * N; yd.max_sweeps = 60; yd.err = c.derr; yd.sweeps_out = nullptr;
  yd.skip = c.orth ? w.skip_old : w.sub_done;
  yd.gwork = w.jgwork; yd.gwork_bytes = w.jgwork_bytes;
  SvdDesc zd = yd;
  zd.A = w.zA; zd.U = w.zU; zd.S = w.zS; zd.V = nullptr;
  SvdDesc bd = yd;                                // k x k Jacobi of B = U^+ Y
  bd.m = k; bd.n = k; bd.A = w.bA; bd.lda = k; bd.U = w.bU; bd.ldu = k;
  bd.tol = 4e-16 * k; bd.skip = w.skip_new; bd.gwork = nullptr; bd.gwork_bytes = 0;
  OrthDesc od;
  od.N = N; od.k = k; od.batch = 2 * B; od.work = w.orth_work; od.work_bytes = w.orth_bytes;
  // warm rounds: blocks close to orthonormal after column scaling; a shifted pass and a plain pass
  // whose input must already be within 1e-2 of orthonormal (else the tall Jacobi takes over);
  // cold rounds (random start): the full three-pass shifted Cholesky QR
  od.skip = w.sub_done; od.fail = w.ofail; od.passes = warm ? 2 : 3; od.shifted = true; od.dev_fail = 1e-2;
  const int ncheck = chi + 1 < k ? chi + 1 : k;
  const double rtol = 1e-14, stag = 1e-12;
  auto route = [&]() -> int {
    IPEPS_LAUNCH(K_ORTH, 0, st,
                 orth_route_kernel<<<(2 * B + 127) / 128, 128, 0, st>>>(w.sub_done, w.ofail, w.skip_new, w.skip_old,
                                                                       2 * B, prof_device_counters()));
    IPEPS_CUDA_TRY(cudaGetLastError());
    return 0;
  };
  const int graph = c.gb ? 1 : 0;
  int* rctr = c.loopctl + 2;
  cudaGraphConditionalHandle hl = 0;
  if (graph) {
    if ((rc = c.gb->loop_begin(rctr, &hl))) return rc;
  } else {
    IPEPS_LAUNCH(K_PROJ_PREP, 0, st, loop_arm_kernel<<<1, 32, 0, st>>>(0, 0, rctr));
  }
  for (int it = 0; it < (graph ? 1 : rounds); ++it) {
    GemmDesc g = gd(N, k, N, 2 * B);            // Y = M V
    g.A = w.M; g.sA = N2; g.lda = N; g.B = w.Vw; g.sB = Nk; g.ldb = k;
    g.C = w.Ysub; g.sC = Nk; g.ldc = k; g.skip = w.sub_done;
    if ((rc = zgemm_f64(g, st))) return rc;
    if (c.orth) {
      IPEPS_CUDA_TRY(cudaMemsetAsync(w.ofail, 0, sizeof(int) * 2 * B, st));
      od.X = w.Ysub; od.sX = Nk; od.Q = w.Uq; od.sQ = Nk;
      if ((rc = orth_cqr(od, st)) || (rc = route())) return rc;
      if ((rc = atb_product(w.Uq, Nk, w.Ysub, Nk, N, k, 2 * B, w.part, w.Bk, kk, w.skip_new, st))) return rc;
      if ((rc = jacobi_svd(bd, st))) return rc;
      g = gd(N, k, k, 2 * B);                   // U_y = U X
      g.A = w.Uq; g.sA = Nk; g.lda = k; g.B = w.Xk; g.sB = kk; g.ldb = k;
      g.C = w.Uy; g.sC = Nk; g.ldc = k; g.skip = w.skip_new;
      if ((rc = zgemm_f64(g, st))) return rc;
    }
    if ((rc = jacobi_svd(yd, st))) return rc;   // all problems, or the fall-back ones
    g = gd(N, k, k, 2 * B);                     // V_f = V W
    g.A = w.Vw; g.sA = Nk; g.lda = k; g.B = w.W; g.sB = kk; g.ldb = k; g.C = slot; g.sC = Nk;
    g.ldc = k; g.skip = w.sub_done;
    if ((rc = zgemm_f64(g, st))) return rc;
    g = gd(N, k, N, 2 * B);                     // Z = M^+ U_y
    g.opA = OP_C; g.A = w.M; g.sA = N2; g.lda = N;
    g.B = w.Uy; g.sB = Nk; g.ldb = k; g.C = w.Zsub; g.sC = Nk; g.ldc = k; g.skip = w.sub_done;
    if ((rc = zgemm_f64(g, st))) return rc;
    IPEPS_LAUNCH(K_PROJ_PREP, 0, st,
                 sub_residual_kernel<<<2 * B, 256, 0, st>>>(w.Zsub, slot, w.Sy, N, k, ncheck, rtol,
                                                            stag, w.sub_done, w.sub_rounds, w.sub_res,
                                                            prof_device_counters()));
    IPEPS_LAUNCH(K_PROJ_PREP, 0, st,
                 sub_test_kernel<<<1, 128, 0, st>>>(w.sub_done, 2 * B, rctr, rounds, hl, graph, c.dflag));
    if (!graph) {
      if (it + 1 == rounds) break;
      if (sub_checkpoint(it + 1)) {
        IPEPS_CUDA_TRY(cudaMemcpyAsync(c.hflag, c.dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
        IPEPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (*c.hflag) break;
      }
    }
    IPEPS_LAUNCH(K_PROJ_PREP, 0, st,
                 sub_refill_kernel<<<2 * B, 256, 0, st>>>(w.Zsub, N, k, c.seed, stream_id * 1000, rctr,
                                                          w.sub_done, B));
    if (c.orth) {
      IPEPS_CUDA_TRY(cudaMemsetAsync(w.ofail, 0, sizeof(int) * 2 * B, st));
      od.X = w.Zsub; od.sX = Nk; od.Q = w.Vw; od.sQ = Nk;
      if ((rc = orth_cqr(od, st)) || (rc = route())) return rc;
    }
    if ((rc = jacobi_svd(zd, st))) return rc;   // all problems, or the fall-back ones
    IPEPS_LAUNCH(K_PROJ_PREP, 0, st,
                 sub_fill_kernel<<<2 * B, 256, 0, st>>>(w.Vz, nullptr, N, k, 0, c.seed, 0, w.Vw,
                                                        c.orth ? w.skip_old : w.sub_done, B));
  }
  if (graph && (rc = c.gb->loop_end())) return rc;
  c.slot_warm[f][x] = true;
  IPEPS_LAUNCH(K_PROJ_PREP, 0, st,
               proj_prep_kernel<<<2 * B, 256, 2 * chi * sizeof(double), st>>>(w.Sy, k, k, w.Uy, slot, N, chi, k, Nk, w.Us,
                                                       w.Vs, w.kept, kDegenRtol, kDegenAbs, kTinyRel, c.cut_rel,
                                                       w.frozen, B, w.sub_done, prof_device_counters()));
  return 0;
}

static int left_move(Ctx& c, int f, int x) {
  const MovePlan& m = c.plan[f][x];
  CtmWork& w = c.w;
  const int B = c.B, chi = c.chi, D2 = c.D2, N = c.N;
  const long long N2 = c.N2(), Nc = (long long)N * chi, chi2 = (long long)chi * chi;
  const long long T = (long long)chi * D2 * chi;
  cudaStream_t st = c.st;
  int rc;
  // enlarged corners (8B problems)
  GemmDesc g = gdm(c, chi, D2 * chi, chi, 8 * B);
  g.Aptr = m.g1A; g.Bptr = m.g1B; g.Cptr = m.g1C; g.lda = chi; g.ldb = D2 * chi; g.ldc = D2 * chi;
  if ((rc = contract(c, g))) return rc;
  g = gdm(c, chi * D2, D2 * chi, chi, 8 * B);
  g.Aptr = m.g2A; g.Bptr = m.g2B; g.Cptr = m.g2C; g.lda = chi; g.ldb = D2 * chi; g.ldc = D2 * chi;
  if ((rc = contract(c, g))) return rc;
  {
    const int dims[4] = {chi, D2, D2, chi}, perm[4] = {0, 3, 2, 1};
    if ((rc = permute_c128(w.X2, w.X2p, 4, dims, perm, 8 * B, N2, N2, st, w.frozen, B))) return rc;
  }
  g = gdm(c, chi * chi, D2 * D2, D2 * D2, 8 * B);
  g.A = w.X2p; g.sA = N2; g.lda = D2 * D2;
  g.Bptr = m.g3B; g.ldb = D2 * D2;
  g.C = w.Y; g.sC = N2; g.ldc = D2 * D2;
  if ((rc = contract(c, g))) return rc;
  {
    const int dims[4] = {chi, chi, D2, D2}, perm[4] = {0, 2, 1, 3};
    if ((rc = permute_c128(w.Y, w.Q, 4, dims, perm, 8 * B, N2, N2, st, w.frozen, B))) return rc;
  }
  // halves and the product over the cut
  g = gdm(c, N, N, N, 4 * B);
  g.Aptr = m.hA; g.Bptr = m.hB; g.Cptr = m.hC; g.lda = N; g.ldb = N; g.ldc = N;
  if ((rc = contract(c, g))) return rc;
  cplx* Rt = w.H;
  cplx* R = w.H + (size_t)2 * B * N2;
  g = gdm(c, N, N, N, 2 * B);
  g.A = R; g.sA = N2; g.lda = N; g.B = Rt; g.sB = N2; g.ldb = N; g.C = w.M; g.sC = N2; g.ldc = N;
  if ((rc = contract(c, g))) return rc;
  if (!c.subspace) {
    // projector SVD: full one-sided Jacobi of M
    SvdDesc sd;
    sd.m = N; sd.n = N; sd.batch = 2 * B;
    sd.A = w.pA; sd.lda = N; sd.U = w.pU; sd.ldu = N; sd.S = w.pS; sd.V = w.pV; sd.ldv = N;
    sd.tol = 4e-16 * N; sd.max_sweeps = 80; sd.err = c.derr; sd.sweeps_out = nullptr;
    sd.skip = w.frozen; sd.skip_mod = B;
    if ((rc = jacobi_svd(sd, st))) return rc;
    IPEPS_LAUNCH(K_PROJ_PREP, 0, st,
                 proj_prep_kernel<<<2 * B, 256, 2 * chi * sizeof(double), st>>>(w.S, N, N, w.U, w.V, N, chi, N, N2, w.Us,
                                                         w.Vs, w.kept, kDegenRtol, kDegenAbs, kTinyRel, c.cut_rel,
                                                         w.frozen, B));
  } else {
    if ((rc = subspace_svd(c, f, x, R, Rt))) return rc;
  }
  // the projectors themselves are always formed in FP64: P = R~ V S^{-1/2} recovers the small
  // singular directions through cancellation, which a split product (error ~1e-5 of |R~| |v|)
  // would swamp for s_j below ~1e-5 s_1
  g = gdm(c, N, chi, N, 2 * B);     // P = R~ Vs
  g.A = Rt; g.sA = N2; g.lda = N; g.B = w.Vs; g.sB = Nc; g.ldb = chi; g.C = w.P; g.sC = Nc; g.ldc = chi;
  if ((rc = zgemm_f64(g, st))) return rc;
  g = gdm(c, chi, N, N, 2 * B);     // P~ = Us^+ R
  g.opA = OP_C; g.A = w.Us; g.sA = Nc; g.lda = chi;
  g.B = R; g.sB = N2; g.ldb = N; g.C = w.Pt; g.sC = Nc; g.ldc = N;
  if ((rc = zgemm_f64(g, st))) return rc;
  // absorption: C1' = P~[y-1] (C1 T1)
  g = gdm(c, chi, chi, N, 2 * B);
  g.Aptr = m.c1A; g.lda = N; g.Bptr = m.c1B; g.ldb = chi; g.C = w.C1n; g.sC = chi2; g.ldc = chi;
  if ((rc = contract(c, g))) return rc;
  // T4' = P~[y] (T4 a) P[y-1]
  g = gdm(c, chi * D2, D2 * chi, chi, 2 * B);
  g.Aptr = m.z1A; g.lda = chi; g.Bptr = m.z1B; g.ldb = D2 * chi; g.C = w.Z1; g.sC = N2; g.ldc = D2 * chi;
  if ((rc = contract(c, g))) return rc;
  {
    const int dims[4] = {chi, D2, D2, chi}, perm[4] = {0, 3, 2, 1};
    if ((rc = permute_c128(w.Z1, w.Z1p, 4, dims, perm, 2 * B, N2, N2, st, w.frozen, B))) return rc;
  }
  g = gdm(c, chi * chi, D2 * D2, D2 * D2, 2 * B);
  g.A = w.Z1p; g.sA = N2; g.lda = D2 * D2; g.Bptr = m.z2B; g.ldb = D2 * D2;
  g.C = w.Z2; g.sC = N2; g.ldc = D2 * D2;
  if ((rc = contract(c, g))) return rc;
  {
    const int dims[4] = {chi, chi, D2, D2}, perm[4] = {0, 2, 3, 1};
    if ((rc = permute_c128(w.Z2, w.Z2p, 4, dims, perm, 2 * B, N2, N2, st, w.frozen, B))) return rc;
  }
  g = gdm(c, chi, D2 * chi, N, 2 * B);
  g.Aptr = m.t4A; g.lda = N; g.B = w.Z2p; g.sB = N2; g.ldb = D2 * chi; g.C = w.T4n; g.sC = T;
  g.ldc = D2 * chi;
  if ((rc = contract(c, g))) return rc;
  // C4' = (T3 C4) P[y]
  g = gdm(c, chi * D2, chi, chi, 2 * B);
  g.Aptr = m.w1A; g.lda = chi; g.Bptr = m.w1B; g.ldb = chi; g.C = w.W1; g.sC = T; g.ldc = chi;
  if ((rc = contract(c, g))) return rc;
  {
    const int dims[3] = {chi, D2, chi}, perm[3] = {0, 2, 1};
    if ((rc = permute_c128(w.W1, w.W1p, 3, dims, perm, 2 * B, T, T, st, w.frozen, B))) return rc;
  }
  g = gdm(c, chi, chi, N, 2 * B);
  g.A = w.W1p; g.sA = T; g.lda = N; g.Bptr = m.c4B; g.ldb = chi; g.C = w.C4n; g.sC = chi2; g.ldc = chi;
  if ((rc = contract(c, g))) return rc;
  IPEPS_LAUNCH(K_NORM_STORE, 0, st,
               normalize_store_kernel<<<3 * 2 * B, 256, 0, st>>>(w.C1n, w.T4n, w.C4n, B, chi2, T, m.sC1, m.sT4,
                                                                m.sC4, w.frozen, c.derr));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

int ctm_sweep(Ctx& c) {
  for (int f = 0; f < 4; ++f)
    for (int x = 0; x < 2; ++x)
      if (int rc = left_move(c, f, x)) return rc;
  return 0;
}

int ctm_spectra(Ctx& c, double tol, int first) {
  SvdDesc sd;
  sd.m = c.chi; sd.n = c.chi; sd.batch = 16 * c.B;
  sd.A = c.w.csA; sd.lda = c.chi; sd.U = nullptr; sd.ldu = 0; sd.S = c.w.csS; sd.V = nullptr; sd.ldv = 0;
  sd.tol = 4e-16 * c.chi; sd.max_sweeps = 80; sd.err = c.derr; sd.sweeps_out = nullptr;
  sd.skip = c.w.frozen; sd.skip_mod = c.B;
  if (int rc = jacobi_svd(sd, c.st)) return rc;
  IPEPS_LAUNCH(K_SPECTRA, 0, c.st,
               spectra_delta_kernel<<<c.B, 32, 0, c.st>>>(c.w.cs, c.w.prev, c.B, c.chi, first, tol,
                                                          stall_threshold(c.precision), c.w.delta,
                                                          c.w.frozen, c.w.sweeps, c.w.best, c.w.since));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace ipeps
