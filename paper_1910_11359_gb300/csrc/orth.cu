// Orthonormalisation of batched tall-skinny complex blocks by column-scaled Cholesky QR, and the
// split-K product A^+ B of two such blocks (see orth.cuh).
//
// X (N x k) is first scaled to unit columns (columns below 1e-14 of the largest norm are treated as
// exact zeros and kept out of the factorisation), then orthonormalised by Cholesky QR passes: the
// Gram matrix G = Xh^+ Xh (split over row blocks, the partial sums added in a fixed order so the
// result does not depend on the launch), its Cholesky factor G = R^+ R and R^-1 in one CTA per
// problem, and Q = Xh R^-1 as a batched GEMM.  With OrthDesc::shifted the first pass adds the shift
// 11 (N k + k (k + 1)) u ||Xh||_F^2 to the diagonal, which keeps the factorisation defined for
// Gram matrices that are singular to working precision; the later passes are plain and bring the
// columns to orthonormality at the rounding level (shifted Cholesky QR, Fukaya, Kannan,
// Nakatsukasa, Zhang & Yamamoto, SIAM J. Sci. Comput. 42 (2020)).  A problem whose factorisation
// breaks down, or whose last Gram matrix is still far from the identity, is flagged for the caller.
#include <cmath>
#include <mutex>

#include "orth.cuh"
#include "prof.cuh"

namespace ipeps {

constexpr double kOrthTiny = 1e-14;     // columns below this fraction of the largest count as zero
constexpr int kGramRows = 64;           // rows per split of the A^+ B products
constexpr int GT = 16;

// column norms c_j of X; Xh = X / c_j (zero for columns below kOrthTiny of the largest, whose c_j
// is set to 0)
__global__ void colscale_kernel(const cplx* X, long long sX, int N, int k, double* c, cplx* Xh,
                                const int* skip) {
  const int q = blockIdx.x;
  if (skip && skip[q]) return;
  extern __shared__ double cn[];                 // [k]
  const cplx* x = X + (size_t)q * sX;
  cplx* xh = Xh + (size_t)q * N * k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) cn[j] = 0.0;
  __syncthreads();
  // one warp per column group: lanes walk the rows of a column, partial sums reduced by shuffles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < k; j += nw) {
    double s = 0.0;
    for (int i = lane; i < N; i += 32) s += cabs2(x[(size_t)i * k + j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cn[j] = sqrt(s);
  }
  __syncthreads();
  __shared__ double cmax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int j = 0; j < k; ++j) m = fmax(m, cn[j]);
    cmax = m;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double v = cn[j];
    const bool live = v > 0.0 && v > kOrthTiny * cmax && isfinite(v);
    cn[j] = live ? 1.0 / v : 0.0;
    c[(size_t)q * k + j] = live ? v : 0.0;
  }
  __syncthreads();
  for (long long idx = threadIdx.x; idx < (long long)N * k; idx += blockDim.x)
    xh[idx] = cscale(x[idx], cn[idx % k]);
}

// partial products P[q][p] = A[q][rows of split p]^+ B[q][same rows]  (k x k each); A, B: N x k
// row-major with batch strides sA, sB.  Grid: (tile column, tile row, q * nsplit + p).
__global__ void __launch_bounds__(GT * GT) atb_partial_kernel(const cplx* A, long long sA, const cplx* B,
                                                              long long sB, int N, int k, int nsplit,
                                                              cplx* P, const int* skip) {
  const int q = blockIdx.z / nsplit, p = blockIdx.z % nsplit;
  if (skip && skip[q]) return;
  const cplx* a = A + (size_t)q * sA;
  const cplx* b = B + (size_t)q * sB;
  const int r0 = p * kGramRows, r1 = min(N, r0 + kGramRows);
  __shared__ cplx As[GT][GT + 1];
  __shared__ cplx Bs[GT][GT + 1];
  const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  cplx acc = cmk(0.0, 0.0);
  for (int rr = r0; rr < r1; rr += GT) {
    const int r = rr + ty;
    As[ty][tx] = (r < r1 && i0 + tx < k) ? a[(size_t)r * k + i0 + tx] : cmk(0.0, 0.0);
    Bs[ty][tx] = (r < r1 && j0 + tx < k) ? b[(size_t)r * k + j0 + tx] : cmk(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < GT; ++t) cfmac(acc, As[t][ty], Bs[t][tx]);   // conj(a_ri) b_rj
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  if (i < k && j < k) P[((size_t)q * nsplit + p) * k * k + (size_t)i * k + j] = acc;
}

// C[q] = sum_p P[q][p], added in split order
__global__ void atb_reduce_kernel(const cplx* P, int k, int nsplit, cplx* C, long long sC, const int* skip) {
  const int q = blockIdx.y;
  if (skip && skip[q]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    cplx s = cmk(0.0, 0.0);
    for (int p = 0; p < nsplit; ++p) s = cadd(s, P[((size_t)q * nsplit + p) * k * k + e]);
    C[(size_t)q * sC + e] = s;
  }
}

// 1 / sqrt(d) for d > 0 to FP64 accuracy: an FP32 seed (~23 bits; d is scaled by a power of 4 into
// FP32 range first) refined by two Newton-Raphson steps y <- y (3 - d y^2) / 2, each of which
// doubles the number of correct bits.  A handful of FP64 operations instead of a square root and a
// division, which matters on the factorisation's sequential chain.
__device__ __forceinline__ double rsqrt_nr(double d) {
  int e;
  const double m = frexp(d, &e);                           // d = m 2^e, m in [0.5, 1)
  const int h = e / 2;                                      // d = (m 2^(e - 2h)) 4^h
  const double ms = ldexp(m, e - 2 * h);
  double y = (double)rsqrtf((float)ms);
  y = y * (1.5 - 0.5 * ms * y * y);
  y = y * (1.5 - 0.5 * ms * y * y);
  return ldexp(y, -h);
}

// Cholesky G = R^+ R (R upper triangular) and R^-1 of one k x k problem per CTA, in shared memory;
// G is the sum of the nsplit partial products P[q][p] of atb_partial_kernel.
// Columns with c_j = 0 are decoupled (unit diagonal, zero off-diagonal), so zero columns of Xh stay
// zero in Q.  shift_rel > 0 adds shift_rel * (number of live columns) to the diagonal.  fail[q] is
// set when a pivot is not positive and finite, or when dev_fail > 0 and max |G - I| over the live
// block (how far the input was from orthonormal, written to dev[q]) exceeds dev_fail.  Rinv is
// written row-major (k x k).  R occupies the upper triangle of the shared array; R^-1, also upper
// triangular, is built in its strict lower triangle (transposed) and a separate diagonal.
__global__ void cholinv_kernel(const cplx* P, int nsplit, const double* c, int k, double shift_rel,
                               cplx* Rinv, int* fail, double* dev, double dev_fail, const int* skip) {
  const int q = blockIdx.x;
  if (skip && skip[q]) return;
  extern __shared__ __align__(16) unsigned char chol_smem[];
  cplx* A = reinterpret_cast<cplx*>(chol_smem);            // k x k
  cplx* xd = A + (size_t)k * k;                            // [k] diagonal of R^-1
  const double* cq = c + (size_t)q * k;
  __shared__ int bad;
  __shared__ double s_inv;
  __shared__ double s_dev[32];
  int live = 0;
  for (int j = 0; j < k; ++j) live += cq[j] > 0.0;
  const double shift = shift_rel * live;
  double mydev = 0.0;                                       // max |G - I|^2 over the live block
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, j = idx % k;
    const bool li = cq[i] > 0.0, lj = cq[j] > 0.0;
    cplx v;
    if (li && lj) {
      // G = sum of the split-K partial products, added in split order
      v = cmk(0.0, 0.0);
      for (int p = 0; p < nsplit; ++p) v = cadd(v, P[((size_t)q * nsplit + p) * k * k + idx]);
      mydev = fmax(mydev, cabs2(csub(v, cmk(i == j ? 1.0 : 0.0, 0.0))));
      if (i == j) v = cmk(v.x + shift, 0.0);
    } else {
      v = cmk(i == j ? 1.0 : 0.0, 0.0);
    }
    A[idx] = v;
  }
  for (int o = 16; o > 0; o >>= 1) mydev = fmax(mydev, __shfl_xor_sync(0xffffffffu, mydev, o));
  if ((threadIdx.x & 31) == 0) s_dev[threadIdx.x >> 5] = mydev;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_dev[w]);
    m = sqrt(m);
    dev[q] = m;
    if (dev_fail > 0.0 && !(m <= dev_fail)) bad = 1;
  }
  __syncthreads();
  // right-looking Cholesky: row j of R, then the rank-1 update of the trailing upper triangle; the
  // pivot reciprocals 1 / R_jj are kept in xd[j].y for the back substitution
  for (int j = 0; j < k && !bad; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[(size_t)j * k + j].x;
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
      } else {
        const double inv = rsqrt_nr(d);
        A[(size_t)j * k + j] = cmk(d * inv, 0.0);
        s_inv = inv;
        xd[j] = cmk(0.0, inv);
      }
    }
    __syncthreads();
    if (bad) break;
    for (int l = j + 1 + threadIdx.x; l < k; l += blockDim.x) A[(size_t)j * k + l] = cscale(A[(size_t)j * k + l], s_inv);
    __syncthreads();
    const int m = k - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int l = j + 1 + idx / m, mm = j + 1 + idx % m;
      if (mm < l) continue;
      const cplx rl = A[(size_t)j * k + l], rm = A[(size_t)j * k + mm];
      cplx v = A[(size_t)l * k + mm];
      // A_lm -= conj(R_jl) R_jm
      v.x -= rl.x * rm.x + rl.y * rm.y;
      v.y -= rl.x * rm.y - rl.y * rm.x;
      A[(size_t)l * k + mm] = v;
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) fail[q] = 1;
    return;
  }
  // R^-1 = X by back substitution on the rows of X = I: for j = k-1 .. 0, row j /= R_jj, then every
  // row i < j loses R_ij times row j (only columns l >= j of row j are nonzero).  X_il (l > i) is
  // kept at A[l][i], X_ii in xd[i].
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x)
    if (idx / k > idx % k) A[idx] = cmk(0.0, 0.0);
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double rinv = xd[j].y;                             // 1 / R_jj from the factorisation
    __syncthreads();
    if (threadIdx.x == 0) xd[j] = cmk(rinv, 0.0);            // X_jj = 1 / R_jj
    for (int l = j + 1 + threadIdx.x; l < k; l += blockDim.x) A[(size_t)l * k + j] = cscale(A[(size_t)l * k + j], rinv);
    __syncthreads();
    const int w = k - j;
    for (int idx = threadIdx.x; idx < j * w; idx += blockDim.x) {
      const int i = idx / w, l = j + idx % w;
      const cplx r = A[(size_t)i * k + j];
      const cplx x = l == j ? xd[j] : A[(size_t)l * k + j];
      cplx* dst = &A[(size_t)l * k + i];                   // X_il, l >= j > i
      cplx v = *dst;
      v.x -= r.x * x.x - r.y * x.y;
      v.y -= r.x * x.y + r.y * x.x;
      *dst = v;
    }
    __syncthreads();
  }
  cplx* out = Rinv + (size_t)q * k * k;
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, l = idx % k;
    out[idx] = l == i ? xd[i] : (l > i ? A[(size_t)l * k + i] : cmk(0.0, 0.0));
  }
}

size_t orth_smem_bytes(int k) { return ((size_t)k * k + k) * sizeof(cplx); }

bool orth_supported(int k) { return k >= 1 && orth_smem_bytes(k) <= 200 * 1024; }

size_t orth_work_bytes(int N, int k, int batch) {
  const int nsplit = (N + kGramRows - 1) / kGramRows;
  size_t b = 0;
  auto add = [&](size_t n) { b += (n + 255) & ~(size_t)255; };
  add((size_t)batch * N * k * sizeof(cplx));            // Xh
  add((size_t)batch * N * k * sizeof(cplx));            // ping-pong block
  add((size_t)batch * k * sizeof(double));              // column norms
  add((size_t)batch * nsplit * k * k * sizeof(cplx));   // split-K partials
  add((size_t)batch * k * k * sizeof(cplx));            // R^-1
  add((size_t)batch * sizeof(double));                  // deviation from orthonormality
  return b;
}

int atb_product(const cplx* A, long long sA, const cplx* B, long long sB, int N, int k, int batch,
                cplx* partial, cplx* C, long long sC, const int* skip, cudaStream_t st) {
  const int nsplit = (N + kGramRows - 1) / kGramRows;
  const int tiles = (k + GT - 1) / GT;
  if ((long long)batch * nsplit > 65535) return cuda_fail(cudaErrorInvalidValue, "atb grid", __FILE__, __LINE__);
  IPEPS_LAUNCH(K_ORTH, 8.0 * batch * (double)N * k * k, st,
               atb_partial_kernel<<<dim3(tiles, tiles, batch * nsplit), GT * GT, 0, st>>>(A, sA, B, sB, N, k,
                                                                                        nsplit, partial, skip));
  IPEPS_LAUNCH(K_ORTH, 0, st,
               atb_reduce_kernel<<<dim3((k * k + 255) / 256, batch), 256, 0, st>>>(partial, k, nsplit, C, sC, skip));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

int orth_cqr(const OrthDesc& d, cudaStream_t st) {
  if (d.batch <= 0) return 0;
  if (!orth_supported(d.k)) return cuda_fail(cudaErrorInvalidValue, "orth size", __FILE__, __LINE__);
  const int N = d.N, k = d.k, B = d.batch;
  const int nsplit = (N + kGramRows - 1) / kGramRows;
  char* w = (char*)d.work;
  auto take = [&](size_t n) { char* p = w; w += (n + 255) & ~(size_t)255; return p; };
  cplx* Xh = (cplx*)take((size_t)B * N * k * sizeof(cplx));
  cplx* Xt = (cplx*)take((size_t)B * N * k * sizeof(cplx));
  double* c = (double*)take((size_t)B * k * sizeof(double));
  cplx* part = (cplx*)take((size_t)B * nsplit * k * k * sizeof(cplx));
  cplx* Rinv = (cplx*)take((size_t)B * k * k * sizeof(cplx));
  double* dev = (double*)take((size_t)B * sizeof(double));
  if ((size_t)(w - (char*)d.work) > d.work_bytes) return cuda_fail(cudaErrorInvalidValue, "orth workspace", __FILE__, __LINE__);
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(cholinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  IPEPS_CUDA_TRY(attr_err);
  IPEPS_LAUNCH(K_ORTH, 0, st, colscale_kernel<<<B, 256, k * sizeof(double), st>>>(d.X, d.sX, N, k, c, Xh, d.skip));
  // passes: shifted, plain, plain; Xh -> Xt -> Xh -> Q
  const double shift = 11.0 * ((double)N * k + (double)k * (k + 1)) * 1.1102230246251565e-16;
  cplx* src = Xh;
  const int tiles = (k + GT - 1) / GT;
  for (int pass = 0; pass < d.passes; ++pass) {
    IPEPS_LAUNCH(K_ORTH, 8.0 * B * (double)N * k * k, st,
                 atb_partial_kernel<<<dim3(tiles, tiles, B * nsplit), GT * GT, 0, st>>>(src, (long long)N * k, src,
                                                                                      (long long)N * k, N, k,
                                                                                      nsplit, part, d.skip));
    const bool shifted = d.shifted && pass == 0;
    IPEPS_LAUNCH(K_ORTH, 0, st,
                 cholinv_kernel<<<B, 256, orth_smem_bytes(k), st>>>(part, nsplit, c, k, shifted ? shift : 0.0, Rinv,
                                                                   d.fail, dev,
                                                                   pass + 1 == d.passes ? d.dev_fail : 0.0, d.skip));
    IPEPS_CUDA_TRY(cudaGetLastError());
    cplx* dst = pass + 1 == d.passes ? d.Q : (src == Xh ? Xt : Xh);
    const long long sD = pass + 1 == d.passes ? d.sQ : (long long)N * k;
    GemmDesc g;
    memset(&g, 0, sizeof(g));
    g.M = N; g.N = k; g.K = k; g.batch = B; g.opA = OP_N; g.opB = OP_N;
    g.A = src; g.sA = (long long)N * k; g.lda = k;
    g.B = Rinv; g.sB = (long long)k * k; g.ldb = k;
    g.C = dst; g.sC = sD; g.ldc = k;
    g.alpha = cmk(1.0, 0.0); g.beta = cmk(0.0, 0.0);
    g.skip = d.skip;
    if (int rc = zgemm_f64(g, st)) return rc;
    src = dst;
  }
  return 0;
}

}  // namespace ipeps
