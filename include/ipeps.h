/* libipeps -- iPEPS real-time evolution of the 2D disordered hard-core boson lattice with the
 * disorder carried by an auxiliary spin per site (arXiv:1910.11359, Sec. "Set up for iPEPS").
 *
 * The library owns all device memory of a handle.  Every call takes or returns HOST buffers, which
 * are copied before the call returns; the caller owns them.  Work is issued asynchronously on the
 * CUDA stream given to ipeps_init (borrowed, never destroyed); calls that return data
 * (trunc_err_out, sweeps_out, ipeps_measure, ipeps_corner_spectrum, ipeps_get_*) synchronise it.
 * Errors are reported only through the returned status; no call aborts, throws or traps.  The text
 * of the last error is available from ipeps_last_error.
 *
 * Model (Eq. Hanc in hard-core boson form, V/J = 2 Delta of Eq. Hori):
 *   H = sum_<ij> [ -J (b_i^+ b_j + h.c.) + V n_i n_j ] + h sum_i tau_i n_i,
 * tau_i the auxiliary level operator with eigenvalues 1 - 2 a / (d_A - 1), a = 0 .. d_A - 1
 * (+1, -1 for d_A = 2); local basis s = n d_A + a, d = 2 d_A.  Two-site checkerboard unit cell: A on
 * x + y even, B on x + y odd.
 *
 * Layouts (row-major, complex = interleaved (re, im) doubles):
 *   Gamma tensors  [batch][d][D][D][D][D], leg order (s, up, left, down, right)
 *   lambda         [batch][4][D], bonds named by A's leg (up, left, down, right)
 */
#ifndef IPEPS_H
#define IPEPS_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipeps_ctx* ipeps_h;

typedef enum {
  IPEPS_OK = 0,
  IPEPS_EINVAL = 1,       /* invalid argument or call order */
  IPEPS_ENOMEM = 2,       /* device allocation failed */
  IPEPS_ENOCONV = 3,      /* an iteration hit its limit; results are usable but not converged */
  IPEPS_ENAN = 4,         /* a non-finite value was produced */
  IPEPS_ECUDA = 5,        /* a CUDA runtime call failed */
  IPEPS_ETIMEOUT = 6,     /* a device-side bounded wait ran out */
  IPEPS_EBUSY = 7,        /* handle in use */
  IPEPS_EUNSUPPORTED = 8  /* valid request this build does not implement */
} ipeps_status;

enum { IPEPS_FP64 = 0, IPEPS_SPLIT_BF16X3 = 1, IPEPS_SPLIT_TF32X3 = 2 };

typedef struct {
  int batch;                /* independent instances sharing the shapes below (>= 1) */
  int d_A;                  /* auxiliary levels = number of disorder values, 2..5 (field levels
                               spaced uniformly in [-h, h], Sec. "Set up for iPEPS"); d = 2 d_A;
                               d_A > 2 needs D^2 >= d */
  int D;                    /* PEPS bond dimension (>= 2) */
  int chi;                  /* environment bond dimension (>= D^2, Appendix) */
  int trotter_order;        /* 1 or 2 */
  double dt;                /* Trotter step */
  int precision;            /* IPEPS_FP64; IPEPS_SPLIT_BF16X3 or IPEPS_SPLIT_TF32X3: the large
                               contractions on the tcgen05 tensor cores as 3-term split products
                               (two BF16 / TF32 terms per value, FP32 accumulation, per K tile for
                               TF32; relative error ~2e-5 / ~1e-6), projectors, simple update and
                               readout in FP64 */
  unsigned long long seed;  /* seeds random starting vectors of iterative solvers */
  const double* J;          /* [batch] hopping, host, copied */
  const double* V;          /* [batch] nearest-neighbour interaction, host, copied */
  const double* h;          /* [batch] disorder strength, host, copied */
  double ctm_cut_rel;       /* CTMRG projector truncation: singular values of the product of the two
                               half-systems below ctm_cut_rel times the largest are dropped
                               (<= 0 selects 1e-10) */
  int projector_svd;        /* 0 = automatic, 1 = full Jacobi SVD of the chi D^2 x chi D^2 product,
                               2 = top-(chi+8) subspace iteration */
} ipeps_params;

typedef struct {
  double t;                 /* simulated time of the measured state */
  double nA, nB;            /* disorder-averaged occupations of the two sublattices */
  double imbalance;         /* I = nA - nB (Sec. "Results for interacting case") */
  double tauzA, tauzB;      /* auxiliary polarisation (conserved, 0 for |+>) */
  double energy;            /* energy per site */
  double purityA;           /* Tr rho_A^2 / (Tr rho_A)^2 of the one-site RDM of A */
  double trunc_err_acc;     /* accumulated discarded weight of the simple update (A's bonds) */
  int ctm_sweeps;           /* sweeps of the last ctmrg_converge */
  double ctm_delta;         /* final corner-spectrum change of the last ctmrg_converge */
  double renyi1A;           /* Renyi entropies S_1 (von Neumann), S_1/2, S_2 of the physical one-site */
  double renyi_halfA;       /* RDM of A, the auxiliary traced out (Sec. "Results for interacting      */
  double renyi2A;           /* case"; at most ln d_p = ln 2)                                           */
} ipeps_obs;

/* Create a handle with `batch` instances in the CDW (x) |+> product state (Sec. "Set up for iPEPS",
 * Initialization, Fig. 1: a D = 1 iPEPS, zero-padded to D) and build the Trotter gates
 * exp(-i h_b delta).  cuda_stream: a cudaStream_t (NULL = legacy default stream). */
ipeps_status ipeps_init(const ipeps_params* p, void* cuda_stream, ipeps_h* out);

/* Replace the site tensors (host arrays, layouts above).  lambda may be NULL: all weights 1, so the
 * tensors are contracted as given.  The environment is kept as a warm start. */
ipeps_status ipeps_set_tensors(ipeps_h h, const double* gamma_A, const double* gamma_B,
                               const double* lambda);

/* n_steps Trotter steps of the simple update (Sec. "Set up for iPEPS", Quench; Appendix): per step
 * the bond updates R, U, L, D (first order) or R, U, L (dt/2), D (dt), L, U, R (dt/2) (second
 * order), each a two-site gate followed by a truncated SVD back to D.  trunc_err_out: host
 * double[batch] receiving the accumulated discarded weight (Sec. "Results for interacting case"),
 * or NULL (then the call does not synchronise). */
ipeps_status ipeps_trotter_step(ipeps_h h, int n_steps, double* trunc_err_out);

/* CTMRG environment of the current tensors (Sec. "Set up for iPEPS", Readout; Appendix: chi >= D^2,
 * "sufficiently well converged").  Directional moves with full 2x2-block projectors; per instance,
 * sweeps until the normalised corner spectra change by less than tol, or until that change has
 * stalled at its rounding floor (no factor-2 improvement of its best value for 10 sweeps while that
 * best and the current change are below 1e-7, the current one within 4x of the best); converged
 * instances stop updating; at most max_sweeps sweeps.  tol <= 0 runs exactly max_sweeps sweeps.  The
 * split precisions leave a noise floor in the spectra: with IPEPS_SPLIT_BF16X3 a positive tol below
 * 1e-7 is raised to 1e-7 and the stall threshold is 1e-5; with IPEPS_SPLIT_TF32X3 they are 1e-8 and
 * 1e-6.  The first call starts from the traced
 * double layers, later calls from the previous environment.  sweeps_out: host int[batch] or NULL;
 * delta_out: host double[batch] or NULL (last change).  Returns IPEPS_ENOCONV when an instance
 * reached max_sweeps without converging (its environment is still usable).  Once every projector
 * has been warm-started (after the first sweep from a fresh environment), the remaining sweeps run
 * as one CUDA graph in which the device decides when to stop (conditional WHILE nodes over the
 * sweeps and over each projector's subspace rounds); the results are those of the eager loop. */
ipeps_status ctmrg_converge(ipeps_h h, double tol, int max_sweeps, int* sweeps_out, double* delta_out);

/* enable != 0 (the default): ctmrg_converge uses the convergence graph described above; 0: every
 * sweep is issued from the host, with a readback of the converged flags after each.  Launch timing
 * (ipeps_profile_enable) always uses the host loop. */
ipeps_status ipeps_set_graphs(ipeps_h h, int enable);

/* Discard the environment; the next ctmrg_converge starts from the traced double layers. */
ipeps_status ctmrg_reset(ipeps_h h);

/* Observables from the environment of the last ctmrg_converge (Sec. "Set up for iPEPS", Readout:
 * disorder-averaged local expectation values with the auxiliaries traced out).  out: host
 * ipeps_obs[batch]. */
ipeps_status ipeps_measure(ipeps_h h, ipeps_obs* out);

/* Normalised singular values s / s_1 of corner `corner` (0..3 = C1..C4) at unit-cell position
 * pos = x + 2 y of instance `inst`; sv_out: host double[chi]. */
ipeps_status ipeps_corner_spectrum(ipeps_h h, int inst, int pos, int corner, double* sv_out);

/* Copy out / replace the CTM environment of instance `inst` (Appendix: the corner and edge
 * fixed-point tensors of CTMRG).  Host buffers, interleaved complex doubles:
 *   C [4][4][chi][chi]       corners C1..C4 at unit-cell position pos = x + 2 y,
 *                            C1[c_T4, c_T1], C2[c_T1, c_T2], C3[c_T2, c_T3], C4[c_T3, c_T4]
 *   T [4][4][chi][D^2][chi]  edges T1..T4 at pos, T1[left, k, right], T2[up, k, down],
 *                            T3[right, k, left], T4[down, k, up], k = ket * D + bra
 * (each index joins the clockwise neighbour's: the last index of C1 is the first of T1, and so on).
 * ipeps_get_env needs an environment (a previous ctmrg_converge or ipeps_set_env) and returns
 * IPEPS_EINVAL otherwise.  ipeps_set_env makes the given tensors the environment of `inst` (the
 * other instances keep theirs, or get the traced start when there was no environment yet); the
 * next ctmrg_converge and ipeps_measure start from it.  Both synchronise the stream. */
ipeps_status ipeps_get_env(ipeps_h h, int inst, double* C_out, double* T_out);
ipeps_status ipeps_set_env(ipeps_h h, int inst, const double* C_in, const double* T_in);

/* Copy out the bond weights (host double[batch][4][D]) / site tensors (host, layouts above). */
ipeps_status ipeps_get_lambda(ipeps_h h, double* lambda_out);
ipeps_status ipeps_get_tensors(ipeps_h h, double* gamma_A, double* gamma_B);

/* Device bytes a handle with these parameters allocates (for admission by memory footprint). */
ipeps_status ipeps_footprint_bytes(const ipeps_params* p, size_t* bytes);

/* Release all device memory of the handle (synchronises its stream). */
ipeps_status ipeps_destroy(ipeps_h h);

/* Text of the last error of the handle (or of the calling thread when h is NULL). */
const char* ipeps_last_error(ipeps_h h);

#ifdef __cplusplus
}
#endif
#endif
