/* libipeps -- free-fermion exact diagonalisation workload (arXiv:1910.11359, Sec. "Set up for
 * non-interacting fermions"; Sec. "Results", non-interacting case, Eq. IPR, Fig. 2-4).
 *
 * R disorder realisations of the single-particle Hamiltonian on an open Lx x Ly square lattice,
 *   H_ij = -J (i, j nearest neighbours),  H_ii = h_i,   site i = x + Lx y,
 * each diagonalised on the device (one-sided Jacobi of H + c I, c chosen so that H + c I is
 * positive definite: its singular vectors are then the eigenvectors of H and E = sigma - c).
 * From the eigensystems:
 *   - the Neel state (sites with x + y even occupied) evolved in the single-particle sector,
 *     n_i(t) = sum over occupied j of |[V exp(-i E t) V^T]_ij|^2, and the mean occupation of the
 *     even and of the odd sites, averaged over the realisations (Fig. 2);
 *   - the inverse participation ratio of every eigenvector, I_k = sum_i |V_ik|^4 (Eq. IPR), and
 *     its sums over the intervals of width bin_width of the rescaled spectrum
 *     eps = (E - E_min) / (E_max - E_min) (eps = 1 in the last interval), averaged over the
 *     realisations (Fig. 4);
 *   - the spectra (Fig. 3).
 * The fields h_i are inputs (the random draws of the disorder are made by the caller).
 *
 * All buffers are HOST buffers owned by the caller; the call allocates and frees its own device
 * workspace, runs on `stream` (a cudaStream_t, NULL = legacy default stream) and synchronises it.
 * Errors: IPEPS_EINVAL for bad sizes or NULL required pointers, IPEPS_EUNSUPPORTED when
 * N = Lx Ly exceeds ipeps_ed_max_sites() (the Jacobi kernel's size limit), IPEPS_ENOMEM,
 * IPEPS_ENAN (non-finite fields), IPEPS_ENOCONV (a Jacobi solve hit its sweep cap; outputs are
 * written), IPEPS_ECUDA. */
#ifndef IPEPS_ED_H
#define IPEPS_ED_H
#include <stddef.h>

#include "ipeps.h"
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int Lx, Ly;          /* lattice, N = Lx * Ly sites, 2 <= N <= ipeps_ed_max_sites() */
  int R;               /* realisations, >= 1 */
  double J;            /* hopping amplitude */
  int T;               /* number of times, >= 1 */
  double bin_width;    /* width of the eps intervals, in (0, 1]; ceil(1 / bin_width) intervals */
} ipeps_ed_params;

/* Largest N = Lx Ly the device eigensolver accepts. */
int ipeps_ed_max_sites(void);

/* Device bytes ipeps_ed_run allocates for these parameters. */
ipeps_status ipeps_ed_bytes(const ipeps_ed_params* p, size_t* bytes);

/* fields: [R][N] on-site fields; times: [T].  Outputs: n_even, n_odd: [T] realisation-averaged
 * mean occupations of the even / odd sites; cum_ipr: [ceil(1 / bin_width)] realisation-averaged
 * interval sums of the IPR; spectra: [R][N] eigenvalues ascending, or NULL; ipr: [R][N] the IPR of
 * the eigenvector of each of those eigenvalues, or NULL; sweeps: [R] Jacobi sweeps used, or NULL. */
ipeps_status ipeps_ed_run(const ipeps_ed_params* p, const double* fields, const double* times,
                          double* n_even, double* n_odd, double* cum_ipr, double* spectra, double* ipr,
                          int* sweeps, void* stream);

#ifdef __cplusplus
}
#endif
#endif
