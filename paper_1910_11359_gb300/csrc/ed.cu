// Free-fermion exact diagonalisation workload (include/ipeps_ed.h; paper Sec. "Set up for
// non-interacting fermions", Sec. "Results" non-interacting case, Eq. IPR).
//
// Per call, for R realisations of an open Lx x Ly lattice (N sites):
//   1. A[r] = H[r] + c_r I (complex N x N, c_r = 4|J| - min_i h_i + 1, so A[r] is positive definite
//      by Gershgorin and its singular vectors are H's eigenvectors, E = sigma - c_r);
//   2. one-sided Jacobi SVD of all A[r] in one batched launch (linalg.cu): U[r] (columns by
//      descending sigma), S[r];
//   3. spectrum ascending and the IPR of each eigenvector (one thread per column, rows walked with
//      consecutive threads on consecutive columns), cumulative IPR per realisation, means;
//   4. Neel propagation in blocks of Tb times: W = U exp(-i E t) (elementwise), Phi = W Bo (batched
//      FP64 GEMM, Bo[r][k][j] = U[r][occ_j][k] gathered once), n_i = sum_j |Phi_ij|^2 (one warp per
//      row, shuffle reduction), even / odd means per (time, realisation) (block reduction in a
//      fixed order), means over the realisations.
// Every reduction runs in a fixed order, so results do not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/ipeps_ed.h"
#include "arena.cuh"
#include "common.cuh"
#include "linalg.cuh"
#include "prof.cuh"

namespace ipeps {
namespace {

__global__ void ed_build_kernel(const double* fields, const double* shift, int Lx, int Ly, int R, double J,
                                cplx* A) {
  const int N = Lx * Ly;
  const long long NN = (long long)N * N, total = (long long)R * NN;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / NN);
    const int i = (int)((idx % NN) / N), j = (int)(idx % N);
    double v = 0.0;
    if (i == j) {
      v = fields[(size_t)r * N + i] + shift[r];
    } else {
      const int xi = i % Lx, yi = i / Lx, xj = j % Lx, yj = j / Lx;
      if ((yi == yj && abs(xi - xj) == 1) || (xi == xj && abs(yi - yj) == 1)) v = -J;
    }
    A[idx] = cmk(v, 0.0);
  }
}

// E[r][a] = S[r][N-1-a] - c_r (ascending) and ipr[r][a] = sum_i |U[r][i][N-1-a]|^4
__global__ void ed_spectrum_kernel(const double* S, const cplx* U, const double* shift, int N, int R, double* E,
                                   double* ipr) {
  const long long total = (long long)R * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / N), q = (int)(idx % N);
    const cplx* Ur = U + (size_t)r * N * N;
    double s = 0.0;
    for (int i = 0; i < N; ++i) {
      const double a2 = cabs2(Ur[(size_t)i * N + q]);
      s = fma(a2, a2, s);
    }
    const int a = N - 1 - q;
    E[(size_t)r * N + a] = S[(size_t)r * N + q] - shift[r];
    ipr[(size_t)r * N + a] = s;
  }
}

// bins[r][b] = sum of ipr[r][k] over the states with floor(eps_k / width) = b (the last interval
// also takes eps = 1), eps_k = (E_k - E_min) / (E_max - E_min); one CTA per realisation
__global__ void ed_bins_kernel(const double* E, const double* ipr, int N, int nb, double width, double* bins) {
  const int r = blockIdx.x;
  const double* e = E + (size_t)r * N;
  const double* I = ipr + (size_t)r * N;
  const double emin = e[0], span = e[N - 1] - e[0];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
      const double eps = span > 0.0 ? (e[k] - emin) / span : 0.0;
      const int bk = min((int)(eps / width), nb - 1);
      if (bk == b) s += I[k];
    }
    bins[(size_t)r * nb + b] = s;
  }
}

// out[m] = mean over r of x[r * stride_r + m * stride_m] (summed in order of r)
__global__ void ed_mean_kernel(const double* x, int R, int M, long long stride_r, long long stride_m,
                               double* out) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) s += x[(size_t)r * stride_r + (size_t)m * stride_m];
    out[m] = s / R;
  }
}

// Bo[r][k][j] = U[r][occ_j][k]
__global__ void ed_gather_kernel(const cplx* U, const int* occ, int N, int No, int R, cplx* Bo) {
  const long long total = (long long)R * N * No;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ((long long)N * No));
    const int k = (int)((idx / No) % N), j = (int)(idx % No);
    Bo[idx] = U[(size_t)r * N * N + (size_t)occ[j] * N + k];
  }
}

// W[tb][r][i][q] = U[r][i][q] exp(-i (S[r][q] - c_r) t_tb)
__global__ void ed_phase_kernel(const cplx* U, const double* S, const double* shift, const double* times, int N,
                                int R, int Tb, cplx* W) {
  const long long NN = (long long)N * N, total = (long long)Tb * R * NN;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int tb = (int)(idx / ((long long)R * NN));
    const long long rem = idx % ((long long)R * NN);
    const int r = (int)(rem / NN), q = (int)(rem % N);
    const double ph = -(S[(size_t)r * N + q] - shift[r]) * times[tb];
    double sn, cs;
    sincos(ph, &sn, &cs);
    W[idx] = cmul(U[rem], cmk(cs, sn));
  }
}

// n[row] = sum_j |Phi[row][j]|^2, one warp per row
__global__ void ed_occ_kernel(const cplx* Phi, int No, long long rows, double* n) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
    const cplx* p = Phi + (size_t)row * No;
    double s = 0.0;
    for (int j = lane; j < No; j += 32) s += cabs2(p[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) n[row] = s;
  }
}

// per (time, realisation) block: mean of n over the even and over the odd sites
__global__ void ed_evenodd_kernel(const double* n, const int* par, int N, int ne, int no, double* ev, double* od) {
  const long long b = blockIdx.x;
  const double* x = n + (size_t)b * N;
  double se = 0.0, so = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    if (par[i] > 0) se += x[i];
    else so += x[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    so += __shfl_xor_sync(0xffffffffu, so, o);
  }
  __shared__ double pe[32], po[32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { pe[w] = se; po[w] = so; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += pe[k]; c += po[k]; }
    ev[b] = a / ne;
    od[b] = c / no;
  }
}

struct EdWork {
  cplx *A, *U, *W, *Phi, *Bo, *gwork;
  double *S, *E, *ipr, *bins, *n, *ev, *od, *shift, *fields, *times, *cum, *nev, *nod;
  int *occ, *par, *sweeps;
  unsigned* err;
  void** ptrs;      // Jacobi operand tables [4][R] then GEMM B table [Tb * R]
  size_t gbytes;
  int Tb, nb;
};

int bins_of(double width) { return (int)std::ceil(1.0 / width - 1e-9); }

// times per GEMM block: W and Phi together within ~2 GiB, and at most 65535 GEMM problems
int time_block(int N, int No, int R, int T) {
  const double per = (double)R * ((double)N * N + (double)N * No) * sizeof(cplx);
  const int by_mem = (int)std::min(1e9, (2.0 * (1 << 30)) / per);
  return std::max(1, std::min(std::min(T, by_mem), 65535 / R));
}

size_t carve(Arena& a, EdWork& w, int Lx, int Ly, int R, int T, double width) {
  const int N = Lx * Ly, No = (N + 1) / 2;   // sites with x + y even: ceil(N / 2) on any lattice
  w.Tb = time_block(N, No, R, T);
  w.nb = bins_of(width);
  w.gbytes = jacobi_svd_fits(N, N) ? 0 : jacobi_svd_global_bytes(N, N, R);
  w.A = a.take<cplx>((size_t)R * N * N);
  w.U = a.take<cplx>((size_t)R * N * N);
  w.W = a.take<cplx>((size_t)w.Tb * R * N * N);
  w.Phi = a.take<cplx>((size_t)w.Tb * R * N * No);
  w.Bo = a.take<cplx>((size_t)R * N * No);
  w.gwork = w.gbytes ? a.take<cplx>(w.gbytes / sizeof(cplx) + 1) : nullptr;
  w.S = a.take<double>((size_t)R * N);
  w.E = a.take<double>((size_t)R * N);
  w.ipr = a.take<double>((size_t)R * N);
  w.bins = a.take<double>((size_t)R * w.nb);
  w.n = a.take<double>((size_t)w.Tb * R * N);
  w.ev = a.take<double>((size_t)T * R);
  w.od = a.take<double>((size_t)T * R);
  w.shift = a.take<double>(R);
  w.fields = a.take<double>((size_t)R * N);
  w.times = a.take<double>(T);
  w.cum = a.take<double>(w.nb);
  w.nev = a.take<double>(T);
  w.nod = a.take<double>(T);
  w.occ = a.take<int>(No);
  w.par = a.take<int>(N);
  w.sweeps = a.take<int>(R);
  w.err = a.take<unsigned>(1);
  w.ptrs = a.take<void*>((size_t)4 * R + (size_t)w.Tb * R);
  return a.used;
}

ipeps_status ed_fail(ipeps_status s, const char* msg) {
  set_thread_error(msg);
  return s;
}

ipeps_status ed_validate(const ipeps_ed_params* p) {
  if (!p) return ed_fail(IPEPS_EINVAL, "NULL parameters");
  if (p->Lx < 1 || p->Ly < 1 || (long long)p->Lx * p->Ly < 2 || p->R < 1 || p->R > 65535 || p->T < 1 ||
      !(p->bin_width > 0.0 && p->bin_width <= 1.0) || !std::isfinite(p->J))
    return ed_fail(IPEPS_EINVAL, "bad ED parameters");
  if ((long long)p->Lx * p->Ly > ipeps_ed_max_sites())
    return ed_fail(IPEPS_EUNSUPPORTED, "lattice larger than the device eigensolver accepts");
  return IPEPS_OK;
}

inline int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 8); }

}  // namespace
}  // namespace ipeps

using namespace ipeps;

extern "C" {

int ipeps_ed_max_sites(void) {
  static int cached = 0;
  if (!cached) {
    int n = 2;
    while (jacobi_svd_supported(n + 1, n + 1)) ++n;
    cached = n;
  }
  return cached;
}

ipeps_status ipeps_ed_bytes(const ipeps_ed_params* p, size_t* bytes) {
  if (!bytes) return ed_fail(IPEPS_EINVAL, "NULL output");
  if (ipeps_status s = ed_validate(p)) return s;
  Arena a;
  EdWork w;
  *bytes = carve(a, w, p->Lx, p->Ly, p->R, p->T, p->bin_width) + 256;
  return IPEPS_OK;
}

ipeps_status ipeps_ed_run(const ipeps_ed_params* p, const double* fields, const double* times, double* n_even,
                          double* n_odd, double* cum_ipr, double* spectra, double* ipr, int* sweeps, void* stream) {
  if (ipeps_status s = ed_validate(p)) return s;
  if (!fields || !times || !n_even || !n_odd || !cum_ipr) return ed_fail(IPEPS_EINVAL, "NULL argument");
  const int Lx = p->Lx, Ly = p->Ly, N = Lx * Ly, R = p->R, T = p->T;
  const double J = p->J;
  for (long long k = 0; k < (long long)R * N; ++k)
    if (!std::isfinite(fields[k])) return ed_fail(IPEPS_ENAN, "non-finite field");
  for (int k = 0; k < T; ++k)
    if (!std::isfinite(times[k])) return ed_fail(IPEPS_EINVAL, "non-finite time");
  cudaStream_t st = (cudaStream_t)stream;
  // host-side tables: shifts, Neel sites, parity
  std::vector<double> shift(R);
  for (int r = 0; r < R; ++r) {
    double mn = fields[(size_t)r * N];
    for (int i = 1; i < N; ++i) mn = std::min(mn, fields[(size_t)r * N + i]);
    shift[r] = 4.0 * std::fabs(J) - mn + 1.0;
  }
  std::vector<int> occ, par(N);
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      const int i = x + Lx * y;
      par[i] = (x + y) % 2 == 0 ? 1 : -1;
      if (par[i] > 0) occ.push_back(i);
    }
  const int No = (int)occ.size(), Ne = N - No;
  Arena a;
  EdWork w;
  const size_t bytes = carve(a, w, Lx, Ly, R, T, p->bin_width);
  void* base = nullptr;
  if (cudaMalloc(&base, bytes + 256) != cudaSuccess) {
    cudaGetLastError();
    return ed_fail(IPEPS_ENOMEM, "cudaMalloc of the ED workspace failed");
  }
  a = Arena();
  a.base = (char*)base;
  carve(a, w, Lx, Ly, R, T, p->bin_width);
  const int nb = w.nb, Tb = w.Tb;
  int rc = 0;
  ipeps_status status = IPEPS_OK;
  auto cu = [&](cudaError_t e, const char* what) {
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, what, __FILE__, __LINE__);
  };
  // operand tables: Jacobi A, U, S, V (NULL) per realisation; GEMM B per (time in block, realisation)
  std::vector<const void*> tab((size_t)4 * R + (size_t)Tb * R);
  for (int r = 0; r < R; ++r) {
    tab[r] = w.A + (size_t)r * N * N;
    tab[R + r] = w.U + (size_t)r * N * N;
    tab[2 * R + r] = w.S + (size_t)r * N;
    tab[3 * R + r] = nullptr;
  }
  for (int tb = 0; tb < Tb; ++tb)
    for (int r = 0; r < R; ++r) tab[(size_t)4 * R + (size_t)tb * R + r] = w.Bo + (size_t)r * N * No;
  cu(cudaMemcpyAsync(w.ptrs, tab.data(), sizeof(void*) * tab.size(), cudaMemcpyHostToDevice, st), "ed tables");
  cu(cudaMemcpyAsync(w.shift, shift.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st), "ed shifts");
  cu(cudaMemcpyAsync(w.fields, fields, sizeof(double) * R * N, cudaMemcpyHostToDevice, st), "ed fields");
  cu(cudaMemcpyAsync(w.times, times, sizeof(double) * T, cudaMemcpyHostToDevice, st), "ed times");
  cu(cudaMemcpyAsync(w.occ, occ.data(), sizeof(int) * No, cudaMemcpyHostToDevice, st), "ed sites");
  cu(cudaMemcpyAsync(w.par, par.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st), "ed parity");
  cu(cudaMemsetAsync(w.err, 0, sizeof(unsigned), st), "ed err");
  if (!rc) {
    IPEPS_LAUNCH(K_ED, 0, st,
                 ed_build_kernel<<<blocks_for((long long)R * N * N), 256, 0, st>>>(w.fields, w.shift, Lx, Ly, R, J,
                                                                                   w.A));
    cu(cudaGetLastError(), "ed build");
  }
  if (!rc) {
    SvdDesc d;
    d.m = N; d.n = N; d.batch = R;
    d.A = (const cplx* const*)w.ptrs; d.lda = N;
    d.U = (cplx* const*)(w.ptrs + R); d.ldu = N;
    d.S = (double* const*)(w.ptrs + 2 * R);
    d.V = nullptr; d.ldv = N;
    d.tol = 4e-16 * std::sqrt((double)N); d.max_sweeps = 60; d.err = w.err; d.sweeps_out = w.sweeps;
    d.skip = nullptr; d.gwork = w.gwork; d.gwork_bytes = w.gbytes;
    rc = jacobi_svd(d, st);
  }
  if (!rc) {
    IPEPS_LAUNCH(K_ED, 0, st,
                 ed_spectrum_kernel<<<blocks_for((long long)R * N), 256, 0, st>>>(w.S, w.U, w.shift, N, R, w.E, w.ipr));
    cu(cudaGetLastError(), "ed spectrum");
  }
  if (!rc) {
    IPEPS_LAUNCH(K_ED, 0, st, ed_bins_kernel<<<R, 64, 0, st>>>(w.E, w.ipr, N, nb, p->bin_width, w.bins));
    IPEPS_LAUNCH(K_ED, 0, st, ed_mean_kernel<<<(nb + 127) / 128, 128, 0, st>>>(w.bins, R, nb, nb, 1, w.cum));
    IPEPS_LAUNCH(K_ED, 0, st,
                 ed_gather_kernel<<<blocks_for((long long)R * N * No), 256, 0, st>>>(w.U, w.occ, N, No, R, w.Bo));
    cu(cudaGetLastError(), "ed bins");
  }
  for (int t0 = 0; t0 < T && !rc; t0 += Tb) {
    const int nt = std::min(Tb, T - t0);
    IPEPS_LAUNCH(K_ED, 0, st,
                 ed_phase_kernel<<<blocks_for((long long)nt * R * N * N), 256, 0, st>>>(w.U, w.S, w.shift,
                                                                                      w.times + t0, N, R, nt, w.W));
    cu(cudaGetLastError(), "ed phase");
    if (rc) break;
    GemmDesc g;
    memset(&g, 0, sizeof(g));
    g.M = N; g.N = No; g.K = N; g.batch = nt * R;
    g.alpha = cmk(1.0, 0.0); g.beta = cmk(0.0, 0.0);
    g.A = w.W; g.sA = (long long)N * N; g.lda = N;
    g.Bptr = (const cplx* const*)(w.ptrs + 4 * R); g.ldb = No;
    g.C = w.Phi; g.sC = (long long)N * No; g.ldc = No;
    if ((rc = zgemm_f64(g, st))) break;
    const long long rows = (long long)nt * R * N;
    IPEPS_LAUNCH(K_ED, 0, st, ed_occ_kernel<<<blocks_for(rows * 32), 256, 0, st>>>(w.Phi, No, rows, w.n));
    IPEPS_LAUNCH(K_ED, 0, st,
                 ed_evenodd_kernel<<<nt * R, 256, 0, st>>>(w.n, w.par, N, No, Ne, w.ev + (size_t)t0 * R,
                                                           w.od + (size_t)t0 * R));
    cu(cudaGetLastError(), "ed occupations");
  }
  if (!rc) {
    // means over the realisations: ev / od are [T][R]
    IPEPS_LAUNCH(K_ED, 0, st, ed_mean_kernel<<<(T + 127) / 128, 128, 0, st>>>(w.ev, R, T, 1, R, w.nev));
    cu(cudaGetLastError(), "ed means");
  }
  if (!rc) {
    IPEPS_LAUNCH(K_ED, 0, st, ed_mean_kernel<<<(T + 127) / 128, 128, 0, st>>>(w.od, R, T, 1, R, w.nod));
    cu(cudaGetLastError(), "ed means");
  }
  unsigned e = 0;
  if (!rc) {
    cu(cudaMemcpyAsync(n_even, w.nev, sizeof(double) * T, cudaMemcpyDeviceToHost, st), "ed out");
    cu(cudaMemcpyAsync(n_odd, w.nod, sizeof(double) * T, cudaMemcpyDeviceToHost, st), "ed out");
    cu(cudaMemcpyAsync(cum_ipr, w.cum, sizeof(double) * nb, cudaMemcpyDeviceToHost, st), "ed out");
    if (spectra) cu(cudaMemcpyAsync(spectra, w.E, sizeof(double) * R * N, cudaMemcpyDeviceToHost, st), "ed out");
    if (ipr) cu(cudaMemcpyAsync(ipr, w.ipr, sizeof(double) * R * N, cudaMemcpyDeviceToHost, st), "ed out");
    if (sweeps) cu(cudaMemcpyAsync(sweeps, w.sweeps, sizeof(int) * R, cudaMemcpyDeviceToHost, st), "ed out");
    cu(cudaMemcpyAsync(&e, w.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "ed err");
    cu(cudaStreamSynchronize(st), "ed sync");
  }
  cudaStreamSynchronize(st);
  cudaFree(base);
  if (rc) return (ipeps_status)rc;
  if (e & DEV_NONFINITE) status = ed_fail(IPEPS_ENAN, "non-finite value in the ED eigensolver");
  else if (e & DEV_JACOBI_CAP) status = ed_fail(IPEPS_ENOCONV, "ED Jacobi solve hit its sweep limit");
  return status;
}

}  // extern "C"
