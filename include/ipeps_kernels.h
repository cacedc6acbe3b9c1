/* Building-block entry points of libipeps (FP64 dense kernels), exported for unit tests.
 *
 * These are the kernels the CTMRG / simple-update pipeline is built from; they are not steps of
 * the paper's method on their own (the paper fixes no kernels).  All pointers are DEVICE pointers
 * owned by the caller; complex numbers are interleaved (re, im) doubles; matrices are row-major.
 * Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).
 * Return value: 0 on success, a nonzero ipeps_status code otherwise (see ipeps.h); the text of the
 * last error on the calling thread is available from ipeps_last_error(NULL).
 */
#ifndef IPEPS_KERNELS_H
#define IPEPS_KERNELS_H
#ifdef __cplusplus
extern "C" {
#endif

/* C[b] = op(A[b]) * op(B[b]) for b < batch, strided by sA/sB/sC elements.
 * op: 0 = as stored, 1 = transpose, 2 = conjugate transpose.  op(A) is M x K, op(B) is K x N.
 * FP64 complex, one 16x16 output tile per CTA. */
int ipeps_kernel_zgemm(int M, int N, int K, int batch, int opA, int opB,
                       const double* A, long long lda, long long sA,
                       const double* B, long long ldb, long long sB,
                       double* C, long long ldc, long long sC, void* stream);

/* Allocation-free variant of ipeps_kernel_svd, same arguments and results for every block whose
 * columns fit in the shared memory of one 8-CTA cluster (e.g. 162 x 26, 512 x 40, 256 x 256);
 * taller blocks, which ipeps_kernel_svd serves through an allocated global-memory column buffer,
 * are refused with IPEPS_EUNSUPPORTED.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc (an application allocator owns the
 * device memory, a plug-in only receives pre-allocated buffers, or device allocation is forbidden
 * after start-up).  Instead of allocating its operand pointer tables and error word per call, it
 * uses a fixed array in device global memory (about 33 KB per GPU that loads the library, kept
 * until the process exits), so batch is limited to 1024 problems; larger batches are rejected with
 * IPEPS_EINVAL.  A, U, S, V (and sweeps_out) are still caller-provided device buffers.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share the array and the last
 * call's contents stay in it (the error word is cleared at the start of every call); calls whose
 * GPU work overlaps race on it and must be serialised by the caller.  Synchronises `stream`. */
int ipeps_kernel_svd_noalloc(int m, int n, int batch, const double* A, double* U, double* S,
                             double* V, double tol, int max_sweeps, int* sweeps_out, void* stream);

/* Orthonormal columns spanning those of X[b] (N x k, row-major, contiguous per problem) for
 * b < batch, by column-scaled Cholesky QR: passes >= 2 (the first with a diagonal shift that keeps
 * the factorisation defined, the others plain).  Columns whose norm is below 1e-14 of the largest
 * count as zero and give zero columns of Q.  fail_out: host int[batch] (or NULL) receiving 1 where
 * the factorisation broke down or the last pass still saw the columns off orthonormal by more than
 * 1e-2 (Q is then not usable).  k <= 110.  Allocates its workspace; synchronising. */
int ipeps_kernel_orth(int N, int k, int batch, const double* X, double* Q, int passes, int* fail_out,
                      void* stream);

/* Trotter gate exp(-i h_b delta) of the d = 4 dilated model (J, V, h as in ipeps_params),
 * computed on the device and copied to the HOST buffer out (16 x 16 complex, row index sA*4+sB).
 * Allocates and frees a small device buffer; synchronising. */
int ipeps_kernel_gate(double J, double V, double h, double delta, double* out);

/* Same product as ipeps_kernel_zgemm on the tcgen05 tensor cores in split precision: the complex
 * product is embedded as one real GEMM ([[Ar,-Ai],[Ai,Ar]] [Br;Bi]), every value is split into two
 * BF16 terms hi + lo, the three leading products hi*hi + hi*lo + lo*hi are accumulated in FP32 in
 * tensor memory.  Relative error ~1e-5 of the operand scale.  Allocates and frees its workspace;
 * synchronising; IPEPS_ETIMEOUT if a bounded device-side wait ran out. */
int ipeps_kernel_zgemm_split(int M, int N, int K, int batch, int opA, int opB,
                             const double* A, long long lda, long long sA,
                             const double* B, long long ldb, long long sB,
                             double* C, long long ldc, long long sC, void* stream);

/* The same product with TF32 terms (kind::tf32; two TF32 values per FP64 value, three products):
 * each K tile of 32 TF32 values is accumulated from zero in its own TMEM buffer and the tiles are
 * summed in FP32 registers with round-to-nearest, so the tensor cores' truncating accumulation adds
 * the bias of four MMAs per tile instead of one growing with K.  Relative error (largest over the
 * outputs) ~1e-6 of |a| |b| sqrt(K), growing like the square root of the number of K tiles; BF16x3:
 * ~2e-5.  Arguments, layout, ownership and errors as ipeps_kernel_zgemm_split. */
int ipeps_kernel_zgemm_split_tf32(int M, int N, int K, int batch, int opA, int opB,
                                  const double* A, long long lda, long long sA,
                                  const double* B, long long ldb, long long sB,
                                  double* C, long long ldc, long long sC, void* stream);

/* out = in permuted: out axis j is in axis perm[j] (rank <= 8, dims[] of the input). */
int ipeps_kernel_permute(const double* in, double* out, int rank, const int* dims,
                         const int* perm, int batch, long long s_in, long long s_out, void* stream);

/* Thin SVD A[b] = U[b] diag(S[b]) V[b]^+ of `batch` m x n complex matrices (m >= n), one-sided
 * Jacobi on a thread-block cluster of 8 CTAs.  U: m x n, S: n (descending), V: n x n, all
 * contiguous per problem (strides m*n, n, n*n).  U or V may be NULL.  sweeps_out: int[batch] or
 * NULL.  Returns IPEPS_ENOCONV if a problem hit max_sweeps, IPEPS_ENAN on non-finite input. */
int ipeps_kernel_svd(int m, int n, int batch, const double* A, double* U, double* S, double* V,
                     double tol, int max_sweeps, int* sweeps_out, void* stream);

/* Launch accounting (all handles, all threads).  ipeps_launch_count: kernels launched by the
 * library since it was loaded.  ipeps_profile_enable(1) resets and starts per-class timing: every
 * launch is then bracketed by CUDA events recorded on the stream it is launched on (this adds a
 * little host overhead); ipeps_profile_read synchronises the device and fills, per kernel class
 * (ipeps_profile_classes() entries, names from ipeps_profile_name), the summed event time in ms,
 * the summed algorithmic flops and the number of launches.  Arrays may be NULL. */
unsigned long long ipeps_launch_count(void);
/* Measured FP64 FMA throughput of the current device in TFLOP/s (independent FMA chains on every
 * SM; best of three timed launches).  Allocates a small scratch buffer. */
int ipeps_kernel_fp64_peak(double* tflops_out);
int ipeps_profile_enable(int on);
int ipeps_profile_classes(void);
const char* ipeps_profile_name(int k);
int ipeps_profile_read(double* ms, double* flops, unsigned long long* launches);
/* Executed tensor-pipe flops (2 x rows x columns x depth of the real BF16 GEMMs, padding and the
 * 3-term split included) of the tcgen05 GEMM launches since ipeps_profile_enable(1); the flops that
 * ipeps_profile_read reports for that class are the complex products' algorithmic 8 M N K. */
int ipeps_profile_tc_executed(double* flops_out);
/* Device-side work counters since ipeps_profile_enable(1) (they count whether or not timing is on),
 * out[0..n): Jacobi SVD problems factorised, their rotation rounds and sweeps (summed over
 * problems), subspace-iteration rounds evaluated (summed over projector problems), projector
 * problems whose subspace iteration met its acceptance test, and projector problems handed on at
 * the round cap without meeting it.  Synchronises the device. */
int ipeps_profile_counters(unsigned long long* out, int n);

#ifdef __cplusplus
}
#endif
#endif
