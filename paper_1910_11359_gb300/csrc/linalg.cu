// FP64 dense building blocks (see linalg.cuh).
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "linalg.cuh"
#include "prof.cuh"

namespace cg = cooperative_groups;

namespace ipeps {

// ------------------------------------------------------------------------------------ GEMM
// 16 x 16 output tile per CTA, one complex output per thread, K staged through shared memory in
// chunks of 16.  FP64 issue rate on this part is ~2 DFMA/clk/SM, far below what shared memory can
// feed, so small tiles (little padding waste at N = 32..162) cost nothing in throughput.
constexpr int GT = 16;

__device__ __forceinline__ cplx load_op(const cplx* P, long long ld, int op, int row, int col) {
  // element (row, col) of op(P)
  if (op == OP_N) return P[(long long)row * ld + col];
  cplx v = P[(long long)col * ld + row];
  return op == OP_C ? cconj(v) : v;
}

__global__ void __launch_bounds__(GT * GT) zgemm_kernel(GemmDesc g) {
  const int b = blockIdx.z;
  if (skipped(g.skip, g.skip_mod, b)) return;
  const cplx* A = g.Aptr ? g.Aptr[b] : g.A + (long long)b * g.sA;
  const cplx* B = g.Bptr ? g.Bptr[b] : g.B + (long long)b * g.sB;
  cplx* C = g.Cptr ? g.Cptr[b] : g.C + (long long)b * g.sC;
  __shared__ cplx As[GT][GT + 1];
  __shared__ cplx Bs[GT][GT + 1];
  const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  // a warp holds rows 2w and 2w + 1 of the tile (ty = threadIdx.x / 16)
  const bool row_live = m0 + (ty & ~1) < g.M;
  cplx acc = cmk(0.0, 0.0);
  for (int k0 = 0; k0 < g.K; k0 += GT) {
    {  // A tile As[mm][kk]; for transposed storage let consecutive threads walk the stored row
      int mm, kk;
      if (g.opA == OP_N) { mm = ty; kk = tx; } else { mm = tx; kk = ty; }
      int gm = m0 + mm, gk = k0 + kk;
      As[mm][kk] = (gm < g.M && gk < g.K) ? load_op(A, g.lda, g.opA, gm, gk) : cmk(0.0, 0.0);
    }
    {  // B tile Bs[kk][nn]
      int kk, nn;
      if (g.opB == OP_N) { kk = ty; nn = tx; } else { kk = tx; nn = ty; }
      int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < g.K && gn < g.N) ? load_op(B, g.ldb, g.opB, gk, gn) : cmk(0.0, 0.0);
    }
    __syncthreads();
    // FP64 issue costs the same per warp-instruction whatever the active lanes, so a warp whose two
    // rows both lie beyond M skips the products, and the last chunk stops at K
    if (row_live) {
      if (k0 + GT <= g.K) {
#pragma unroll
        for (int kk = 0; kk < GT; ++kk) cfma(acc, As[ty][kk], Bs[kk][tx]);
      } else {
        for (int kk = 0; kk < g.K - k0; ++kk) cfma(acc, As[ty][kk], Bs[kk][tx]);
      }
    }
    __syncthreads();
  }
  const int gm = m0 + ty, gn = n0 + tx;
  if (gm < g.M && gn < g.N) {
    cplx r = cmul(g.alpha, acc);
    long long o = (long long)gm * g.ldc + gn;
    if (g.beta.x != 0.0 || g.beta.y != 0.0) r = cadd(r, cmul(g.beta, C[o]));
    C[o] = r;
  }
}

int zgemm_f64(const GemmDesc& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return 0;
  if (g.batch > 65535) return cuda_fail(cudaErrorInvalidValue, "zgemm batch", __FILE__, __LINE__);
  dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, g.batch);
  IPEPS_LAUNCH(K_ZGEMM, 8.0 * g.M * g.N * (double)g.K * g.batch, st,
               zgemm_kernel<<<grid, GT * GT, 0, st>>>(g));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------------------------ permute
struct PermArgs {
  int rank;
  long long out_dims[8];
  long long in_stride_of_out_axis[8];
};

__global__ void permute_kernel(const cplx* __restrict__ in, cplx* __restrict__ out, PermArgs a,
                               long long total, int batch, long long s_in, long long s_out,
                               const int* skip, int skip_mod) {
  long long n = total * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    long long b = idx / total, o = idx - b * total;
    if (skipped(skip, skip_mod, (int)b)) continue;
    long long rem = o, off = 0;
    for (int j = a.rank - 1; j >= 0; --j) {
      long long c = rem % a.out_dims[j];
      rem /= a.out_dims[j];
      off += c * a.in_stride_of_out_axis[j];
    }
    out[b * s_out + o] = in[b * s_in + off];
  }
}

int permute_c128(const cplx* in, cplx* out, int rank, const int* dims, const int* perm, int batch,
                 long long s_in, long long s_out, cudaStream_t st, const int* skip, int skip_mod) {
  if (rank < 1 || rank > 8) return cuda_fail(cudaErrorInvalidValue, "permute rank", __FILE__, __LINE__);
  PermArgs a;
  a.rank = rank;
  long long in_stride[8];
  long long s = 1;
  for (int j = rank - 1; j >= 0; --j) { in_stride[j] = s; s *= dims[j]; }
  long long total = s;
  for (int j = 0; j < rank; ++j) {
    a.out_dims[j] = dims[perm[j]];
    a.in_stride_of_out_axis[j] = in_stride[perm[j]];
  }
  long long n = total * batch;
  if (n == 0) return 0;
  int threads = 256;
  long long blocks = std::min<long long>((n + threads - 1) / threads, 152LL * 16);
  IPEPS_LAUNCH(K_PERMUTE, 0, st,
               permute_kernel<<<(unsigned)blocks, threads, 0, st>>>(in, out, a, total, batch, s_in, s_out,
                                                                    skip, skip_mod));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------------------------ Jacobi SVD
constexpr int JCS = 8;          // CTAs per cluster for most blocks (portable cluster size)
constexpr int JCS_TALL = 16;    // tall blocks (m >= 1024) on 16-CTA clusters where the part allows
// Columns whose squared norm is below JTINY take part in no rotation: their squared entries sit in
// or near the subnormal range, where the rotation's phase cannot be formed accurately.
constexpr double JTINY = 1e-250;
constexpr int JTHREADS = 256;

struct JacobiArgs {
  SvdDesc d;
  int np, ra, rw;
  int lpp;                     // lanes per pair in the dot-product phase (power of two, 4..32)
  unsigned long long* flops;   // algorithmic flop counter (dot products + applied rotations)
  unsigned long long* ctr;     // work counters (problems, rounds, sweeps)
};

// Round-robin ("circle") tournament: position 0 fixed, the rest rotate by one each round, so every
// pair of the np (even) columns meets exactly once in np - 1 rounds.
__device__ __forceinline__ int rr_pos(int i, int r, int np) {
  return i == 0 ? 0 : ((i - 1 + r) % (np - 1)) + 1;
}

__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
}

// Rotation of one pair from its Gram entries al = |a_p|^2, be = |a_q|^2, gamma = a_p^+ a_q
// (gr + i gi).  The update a_p <- c a_p - s e a_q, a_q <- s a_p + c e a_q zeroes gamma for
// zeta = (be - al) / 2|gamma|, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2),
// s = c t and e = conj(gamma) / |gamma|.
// FP64 issue is slow on this part, so the fast path forms t in FP32 (the angle only steers the
// iteration; a relative error of 1e-7 in t leaves an off-diagonal of ~1e-7 |gamma| that the next
// sweep removes) while c, s and e are formed in FP64 from that t, so the applied transformation
// is unitary to FP64 rounding.  Column norms outside [1e-70, 1e70] or extreme zeta take the
// all-FP64 path.  Returns 1 when the pair is rotated.
__device__ __forceinline__ int jacobi_rotation(double al, double be, double gr, double gi, double tol,
                                               double* out) {
  const double g2 = fma(gr, gr, gi * gi);
  if (al > 1e-140 && al < 1e140 && be > 1e-140 && be < 1e140) {
    if (!(g2 > tol * tol * (al * be))) return 0;
    const double rg = rsqrt(g2);
    const double zeta = (be - al) * (0.5 * rg);
    if (fabs(zeta) < 1e30) {
      const float zf = (float)zeta, az = fabsf(zf);
      const float tf = az > 1e4f ? 0.5f / zf : copysignf(1.0f, zf) / (az + sqrtf(fmaf(zf, zf, 1.0f)));
      const double t = (double)tf;
      const double c = rsqrt(fma(t, t, 1.0));
      out[0] = c;
      out[1] = c * t;
      out[2] = gr * rg;
      out[3] = -gi * rg;
      return 1;
    }
  }
  // all-FP64 path: rescaled phase, exact angle
  const double g = sqrt(g2 > 0.0 ? g2 : 0.0);
  if (!(al > JTINY && be > JTINY)) return 0;
  const double mg = fmax(fabs(gr), fabs(gi));
  if (!(mg > 0.0)) return 0;
  const double grs = gr / mg, gis = gi / mg;
  const double gn = sqrt(grs * grs + gis * gis);
  const double gabs = mg * gn;                      // |gamma| without underflow
  if (!(gabs > tol * sqrt(al) * sqrt(be))) return 0;
  (void)g;
  const double zeta = (be - al) / (2.0 * gabs);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
  const double c = 1.0 / sqrt(1.0 + t * t);
  out[0] = c;
  out[1] = c * t;
  out[2] = grs / gn;
  out[3] = -gis / gn;
  return 1;
}

template <int CS>
__global__ void __launch_bounds__(JTHREADS) jacobi_kernel(JacobiArgs args) {
  cg::cluster_group cluster = cg::this_cluster();
  const SvdDesc& d = args.d;
  const int rank = (int)cluster.block_rank();
  const int prob = blockIdx.x / CS;
  const int np = args.np, ra = args.ra, rw = args.rw;
  const int npairs = np / 2;
  const int m = d.m, n = d.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = JTHREADS / 32;
  // skipped problems: every CTA of the cluster reads the same flag and leaves before any barrier
  if (skipped(d.skip, d.skip_mod, prob)) return;

  extern __shared__ __align__(16) unsigned char jsm_raw[];
  // the CTA's row slices of the columns: in shared memory, or in its own region of d.gwork
  cplx* colA = d.gwork ? d.gwork + (size_t)blockIdx.x * np * (ra + rw)
                       : reinterpret_cast<cplx*>(jsm_raw);   // colA[j * ra + i]
  cplx* colW = colA + (size_t)np * ra;                      // colW[j * rw + i]
  double* part = d.gwork ? reinterpret_cast<double*>(jsm_raw)
                         : reinterpret_cast<double*>(colW + (size_t)np * rw);   // [2][CS][npairs][4]
  double* rot = part + 2 * CS * npairs * 4;                // [npairs][4]: c, s, er, ei
  int* flags = reinterpret_cast<int*>(rot + npairs * 4);    // [npairs] + any + nonfinite

  const cplx* A = d.A[prob];
  const int a0 = rank * ra, w0 = rank * rw;
  for (int idx = tid; idx < np * ra; idx += JTHREADS) {
    int j = idx / ra, i = idx - j * ra, gi = a0 + i;
    colA[idx] = (j < n && gi < m) ? A[(long long)gi * d.lda + j] : cmk(0.0, 0.0);
  }
  for (int idx = tid; idx < np * rw; idx += JTHREADS) {
    int j = idx / rw, i = idx - j * rw, gi = w0 + i;
    colW[idx] = (gi == j && gi < n) ? cmk(1.0, 0.0) : cmk(0.0, 0.0);
  }
  if (tid == 0) { flags[npairs] = 0; flags[npairs + 1] = 0; }
  __syncthreads();

  const int nrounds = np - 1;
  const int lpp = args.lpp, ppw = 32 / lpp;                 // dot phase: lpp lanes per pair
  const int sub = lane & (lpp - 1), slot = lane / lpp;
  long long gcount = 0;
  __shared__ int nrot_round;
  long long nrot_total = 0;    // rotations applied (tallied by thread 0)
  int sweep = 0;
  bool converged = false;
  for (sweep = 0; sweep < d.max_sweeps; ++sweep) {
    for (int r = 0; r < nrounds; ++r, ++gcount) {
      const int buf = (int)(gcount & 1);
      // slot of this CTA's partial sums inside every CTA's buffer
      const size_t myslot = ((size_t)buf * CS + rank) * npairs * 4;
      // dot products: ppw pairs per warp, lpp lanes per pair, reduced by shuffles within the group
      for (int pb = warp * ppw; pb < npairs; pb += nwarps * ppw) {
        const int p = pb + slot;
        const bool valid = p < npairs;
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
        if (valid) {
          const int cp = rr_pos(p, r, np), cq = rr_pos(np - 1 - p, r, np);
          for (int i = sub; i < ra; i += lpp) {
            cplx x = colA[cp * ra + i], y = colA[cq * ra + i];
            al = fma(x.x, x.x, fma(x.y, x.y, al));
            be = fma(y.x, y.x, fma(y.y, y.y, be));
            gr = fma(x.x, y.x, fma(x.y, y.y, gr));
            gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
          }
        }
        for (int o = lpp >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          gr += __shfl_xor_sync(0xffffffffu, gr, o);
          gi += __shfl_xor_sync(0xffffffffu, gi, o);
        }
        // push the partials into every CTA of the cluster (remote stores do not stall; the
        // cluster barrier below makes them visible), so the reduction reads only local memory
        if (valid)
          for (int q = sub; q < CS; q += lpp) {
            double* dst = cluster.map_shared_rank(part, q) + myslot + p * 4;
            dst[0] = al; dst[1] = be; dst[2] = gr; dst[3] = gi;
          }
      }
      if (tid == 0) nrot_round = 0;
      cluster.sync();
      // decisions: 4 lanes per pair, one Gram component each summed over the CTAs in rank order
      // (so every CTA reaches bit-identical decisions), then gathered by shuffles
      for (int pb = warp * 8; pb < npairs; pb += nwarps * 8) {
        const int p = pb + (lane >> 2), comp = lane & 3;
        double acc = 0.0;
        if (p < npairs)
          for (int q = 0; q < CS; ++q) acc += part[((size_t)buf * CS + q) * npairs * 4 + p * 4 + comp];
        const int base = lane & ~3;
        const double al = __shfl_sync(0xffffffffu, acc, base);
        const double be = __shfl_sync(0xffffffffu, acc, base + 1);
        const double gr = __shfl_sync(0xffffffffu, acc, base + 2);
        const double gi = __shfl_sync(0xffffffffu, acc, base + 3);
        if (p < npairs && comp == 0) {
          int doit = 0;
          if (!(finite_bits(al) && finite_bits(be) && finite_bits(gr) && finite_bits(gi))) {
            flags[npairs + 1] = 1;
          } else {
            double rr[4];
            doit = jacobi_rotation(al, be, gr, gi, d.tol, rr);
            if (doit) {
              rot[p * 4 + 0] = rr[0];
              rot[p * 4 + 1] = rr[1];
              rot[p * 4 + 2] = rr[2];
              rot[p * 4 + 3] = rr[3];
              flags[npairs] = 1;
              atomicAdd(&nrot_round, 1);
            }
          }
          flags[p] = doit;
        }
      }
      __syncthreads();
      if (tid == 0) nrot_total += nrot_round;
      if (flags[npairs + 1]) break;
      // the accumulated right vectors (colW) are rotated only when V is wanted
      const int rows = d.V ? ra + rw : ra;
      for (int idx = tid; idx < npairs * rows; idx += JTHREADS) {
        const int p = idx / rows, i = idx - p * rows;
        if (!flags[p]) continue;
        const int cp = rr_pos(p, r, np), cq = rr_pos(np - 1 - p, r, np);
        cplx* base = i < ra ? colA : colW;
        const int st = i < ra ? ra : rw;
        const int ii = i < ra ? i : i - ra;
        const double c = rot[p * 4 + 0], s = rot[p * 4 + 1];
        const cplx e = cmk(rot[p * 4 + 2], rot[p * 4 + 3]);
        const cplx x = base[cp * st + ii];
        const cplx ey = cmul(e, base[cq * st + ii]);
        base[cp * st + ii] = cmk(c * x.x - s * ey.x, c * x.y - s * ey.y);
        base[cq * st + ii] = cmk(s * x.x + c * ey.x, s * x.y + c * ey.y);
      }
      __syncthreads();
    }
    const bool nonfinite = flags[npairs + 1] != 0;
    const bool any = flags[npairs] != 0;
    __syncthreads();
    if (tid == 0) flags[npairs] = 0;
    __syncthreads();
    if (nonfinite) break;
    if (!any) { converged = true; break; }
  }
  const bool nonfinite_any = flags[npairs + 1] != 0;
  // column norms, reduced over the cluster; the barrier first lets every CTA finish reading the
  // partial-sum buffers of the last round
  cluster.sync();
  double* norms = part;                                       // np doubles fit (8 * npairs >= np)
  for (int j = warp; j < np; j += nwarps) {
    double s = 0.0;
    for (int i = lane; i < ra; i += 32) s += cabs2(colA[j * ra + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) norms[j] = s;
  }
  cluster.sync();
  // rot[] is free now: sigma in rot[0..np), sorted source column in flags[0..np) (both fit)
  double* sig = rot;
  int* order = flags;
  __syncthreads();
  for (int j = tid; j < np; j += JTHREADS) {
    double s = 0.0;
    for (int q = 0; q < CS; ++q) s += cluster.map_shared_rank(norms, q)[j];
    sig[j] = sqrt(s);
  }
  __syncthreads();
  // rank by a key that orders NaN below every norm, so that the ranks form a permutation of
  // [0, n) whatever the data (a NaN compares false both ways and would leave ranks unassigned)
  for (int j = tid; j < n; j += JTHREADS) {
    const double kj = sig[j] == sig[j] ? sig[j] : -1.0;
    int rk = 0;
    for (int k = 0; k < n; ++k) {
      const double kk = sig[k] == sig[k] ? sig[k] : -1.0;
      rk += (kk > kj) || (kk == kj && k < j);
    }
    order[rk] = j;
  }
  __syncthreads();
  if (d.S && rank == 0)
    for (int j = tid; j < n; j += JTHREADS) d.S[prob][j] = sig[order[j]];
  if (d.U) {
    cplx* U = d.U[prob];
    for (int idx = tid; idx < n * ra; idx += JTHREADS) {
      const int j = idx / ra, i = idx - j * ra, gi = a0 + i;
      if (gi >= m) continue;
      const double s = sig[order[j]];
      const cplx v = colA[order[j] * ra + i];
      U[(long long)gi * d.ldu + j] = s > 0.0 ? cscale(v, 1.0 / s) : cmk(0.0, 0.0);
    }
  }
  if (d.V) {
    cplx* V = d.V[prob];
    for (int idx = tid; idx < n * rw; idx += JTHREADS) {
      const int j = idx / rw, i = idx - j * rw, gi = w0 + i;
      if (gi >= n) continue;
      V[(long long)gi * d.ldv + j] = colW[order[j] * rw + i];
    }
  }
  if (tid == 0 && rank == 0) {
    if (args.flops) {
      const double work = 16.0 * m * npairs * (double)gcount + 14.0 * (m + n) * (double)nrot_total;
      atomicAdd(args.flops, (unsigned long long)work);
    }
    if (args.ctr) {
      atomicAdd(args.ctr + CTR_JACOBI_PROBLEMS, 1ull);
      atomicAdd(args.ctr + CTR_JACOBI_ROUNDS, (unsigned long long)gcount);
      atomicAdd(args.ctr + CTR_JACOBI_SWEEPS, (unsigned long long)(sweep + 1));
    }
    if (d.sweeps_out) d.sweeps_out[prob] = sweep + 1;
    if (d.err) {
      if (nonfinite_any) atomicOr(d.err, (unsigned)DEV_NONFINITE);
      else if (!converged) atomicOr(d.err, (unsigned)DEV_JACOBI_CAP);
    }
  }
  cluster.sync();   // no CTA leaves while its shared memory may still be read by the others
}

static void jacobi_layout(int m, int n, int cs, int* np, int* ra, int* rw) {
  *np = n + (n & 1);
  *ra = (m + cs - 1) / cs;
  *rw = (n + cs - 1) / cs;
}

static size_t smem_bytes_cs(int m, int n, int cs) {
  int np, ra, rw;
  jacobi_layout(m, n, cs, &np, &ra, &rw);
  size_t npairs = np / 2;
  return (size_t)np * (ra + rw) * sizeof(cplx) + (2 * (size_t)cs * npairs * 4 + npairs * 4) * sizeof(double) +
         (npairs + 2 + np) * sizeof(int) + 64;
}

// shared memory left when the columns live in global memory: partial sums, rotations, flags
static size_t small_smem_bytes_cs(int m, int n, int cs) {
  int np, ra, rw;
  jacobi_layout(m, n, cs, &np, &ra, &rw);
  const size_t npairs = np / 2;
  return (2 * (size_t)cs * npairs * 4 + npairs * 4) * sizeof(double) + (npairs + 2 + np) * sizeof(int) + 64;
}

static size_t global_bytes_cs(int m, int n, int batch, int cs) {
  int np, ra, rw;
  jacobi_layout(m, n, cs, &np, &ra, &rw);
  return (size_t)batch * cs * np * (ra + rw) * sizeof(cplx);
}

// The public size predicates assume 8-CTA clusters (the conservative choice); a launch on 16-CTA
// clusters needs no more shared memory per CTA and at most jacobi_svd_global_bytes of columns.
size_t jacobi_svd_smem_bytes(int m, int n) { return smem_bytes_cs(m, n, JCS); }

bool jacobi_svd_fits(int m, int n) {
  return m >= n && n >= 1 && smem_bytes_cs(m, n, JCS) <= 200 * 1024;
}

bool jacobi_svd_supported(int m, int n) {
  return m >= n && n >= 1 && small_smem_bytes_cs(m, n, JCS) <= 200 * 1024;
}

size_t jacobi_svd_global_bytes(int m, int n, int batch) {
  return std::max(global_bytes_cs(m, n, batch, JCS), global_bytes_cs(m, n, batch, JCS_TALL));
}

// 16-CTA clusters are a non-portable size: used when the device accepts them for this kernel
// (probed once per process; the library drives one device per process)
static bool tall_clusters_available() {
  static std::once_flag once;
  static int state = 0;
  std::call_once(once, [] {
    if (cudaFuncSetAttribute(jacobi_kernel<JCS_TALL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(jacobi_kernel<JCS_TALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024 + 1024) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = JCS_TALL;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(JCS_TALL);
      cfg.blockDim = dim3(JTHREADS);
      cfg.dynamicSmemBytes = 200 * 1024;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, jacobi_kernel<JCS_TALL>, &cfg) == cudaSuccess &&
          nclusters > 0)
        state = 1;
    }
    cudaGetLastError();
  });
  return state == 1;
}

template <int CS>
static int launch_jacobi(const JacobiArgs& a, size_t smem, int batch, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(jacobi_kernel<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024 + 1024);
  });
  IPEPS_CUDA_TRY(attr_err);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(batch * CS);
  cfg.blockDim = dim3(JTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  IPEPS_LAUNCH(K_JACOBI, 0, st, IPEPS_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_kernel<CS>, a)));
  return 0;
}

int jacobi_svd(const SvdDesc& d, cudaStream_t st) {
  if (d.batch <= 0) return 0;
  if (!jacobi_svd_supported(d.m, d.n))
    return cuda_fail(cudaErrorInvalidValue, "jacobi_svd size", __FILE__, __LINE__);
  const int cs = (d.m >= 1024 && tall_clusters_available()) ? JCS_TALL : JCS;
  JacobiArgs a;
  a.d = d;
  const bool in_smem = smem_bytes_cs(d.m, d.n, cs) <= 200 * 1024;
  if (in_smem) {
    a.d.gwork = nullptr;
  } else if (!d.gwork || d.gwork_bytes < global_bytes_cs(d.m, d.n, d.batch, cs)) {
    return cuda_fail(cudaErrorInvalidValue, "jacobi_svd size", __FILE__, __LINE__);
  }
  jacobi_layout(d.m, d.n, cs, &a.np, &a.ra, &a.rw);
  const size_t smem = in_smem ? smem_bytes_cs(d.m, d.n, cs) : small_smem_bytes_cs(d.m, d.n, cs);
  a.flops = prof_device_flops();
  a.ctr = prof_device_counters();
  // dot-product lanes per pair: about 4 rows per lane, 4..32 lanes
  a.lpp = 4;
  while (a.lpp < 32 && a.lpp * 4 < a.ra) a.lpp *= 2;
  return cs == JCS_TALL ? launch_jacobi<JCS_TALL>(a, smem, d.batch, st)
                        : launch_jacobi<JCS>(a, smem, d.batch, st);
}

}  // namespace ipeps
