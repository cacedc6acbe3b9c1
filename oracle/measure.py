"""Reduced density matrices and observables from a converged CTM environment (FP64, plain NumPy).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Paper: Sec. "Set up for iPEPS" (Readout): local expectation values of |Psi(t)> are exact disorder
averages, E<O(t)> = <Psi(t)|O|Psi(t)>, with the auxiliaries traced out; CTMRG supplies the effective
environment.  Sec. "Results for interacting case": the imbalance is the difference of the particle
numbers on the two sublattices, I = n_A - n_B.

Index conventions are those of ``oracle/ctmrg.py``.  Site A is read at unit-cell position (0, 0),
site B at (1, 0).

Quantities:
  rho1        one-site RDM rho[s, s'] = sum psi_s psi*_s' (d x d), unnormalised
  rho2_h/v    two-site RDMs rho[s, s', v, v'] on a horizontal / vertical bond
  norm_site   CTM norm per site kappa = Z(1x1) Z(0x0) / (Z(1x0) Z(0x1)) -- closed networks of the
              environment around one site with the site, with nothing, with only the row, with only
              the column.  Gauge-invariant only for a translation-invariant environment (A = B),
              where the two chi-legs of each edge tensor sit on equivalent cuts; used for the Ising
              pin, not reported for the checkerboard state.
  purity      Tr(rho^2) / Tr(rho)^2 of the one-site RDM (Renyi-2 entropy = -ln purity).
  renyi       Renyi entropies S_1, S_1/2, S_2 of the physical one-site RDM (auxiliary traced out).

Parity: pinned by tests/test_oracle_ctmrg.py (Ising magnetisation, bond energy and free energy;
dimer states; brute-force tori) and tests/test_oracle_evolve.py (J = 0, short-time closed form,
exact diagonalisation of an 8-site cluster).
"""
import functools

import numpy as np

from .ctmrg import double_layer, double_layer_open
from .model import bond_hamiltonian, local_ops

ein = functools.partial(np.einsum, optimize=True)


def rho1(A, env, p):
    """One-site RDM at unit-cell position p for site tensor A (legs s, u, l, d, r)."""
    C, T = env.C, env.T
    ao = double_layer_open(A)
    top = ein('ac,cue,ef->auf', C[0][p], T[0][p], C[1][p])
    bottom = ein('ab,bkc,cd->akd', C[2][p], T[2][p], C[3][p])
    return ein('auf,frg,gkh,hla,stulkr->st', top, T[1][p], bottom, T[3][p], ao)


def rho2_h(A1, A2, env, p, q):
    """Two-site RDM on the horizontal bond p -> q = p + x; returns rho[s, s', v, v']."""
    C, T = env.C, env.T
    ao1, ao2 = double_layer_open(A1), double_layer_open(A2)
    left = ein('ab,buc,hla,gh,ekg,stulkr->stcre', C[0][p], T[0][p], T[3][p], C[3][p], T[2][p], ao1)
    right = ein('cuf,fi,irj,jm,mke,vwulkr->vwcle', T[0][q], C[1][q], T[1][q], C[2][q], T[2][q], ao2)
    return ein('stcre,vwcre->stvw', left, right)


def rho2_v(A1, A2, env, p, q):
    """Two-site RDM on the vertical bond p -> q = p + y; returns rho[s, s', v, v']."""
    C, T = env.C, env.T
    ao1, ao2 = double_layer_open(A1), double_layer_open(A2)
    up = ein('ab,buc,cf,frg,hla,stulkr->sthkg', C[0][p], T[0][p], C[1][p], T[1][p], T[3][p], ao1)
    low = ein('ilh,grj,jm,mkn,ni,vwulkr->vwhug', T[3][q], T[1][q], C[2][q], T[2][q], C[3][q], ao2)
    return ein('sthkg,vwhkg->stvw', up, low)


def norm_site(A, env, p):
    """CTM norm per site kappa at position p (meaningful for translation-invariant environments)."""
    C, T = env.C, env.T
    a = double_layer(A)
    top = ein('ac,cue,ef->auf', C[0][p], T[0][p], C[1][p])
    bottom = ein('ab,bkc,cd->akd', C[2][p], T[2][p], C[3][p])
    z11 = ein('auf,frg,gkh,hla,ulkr->', top, T[1][p], bottom, T[3][p], a)
    z00 = ein('ab,bc,cd,da->', C[0][p], C[1][p], C[2][p], C[3][p])
    z10 = ein('ab,bkc,cf,fg,gkh,ha->', C[0][p], T[0][p], C[1][p], C[2][p], T[2][p], C[3][p])
    z01 = ein('ab,bc,ckd,de,ef,fka->', C[0][p], C[1][p], T[1][p], C[2][p], C[3][p], T[3][p])
    return z11 * z00 / (z10 * z01)


def expect1(rho, O):
    """<O> = Tr(O rho) / Tr(rho) for rho[s, s'] = psi_s psi*_s'."""
    return np.einsum('ts,st->', O, rho) / np.trace(rho)


def expect2(rho, O):
    """<O> for a two-site operator O on index sA * d + sB and rho[s, s', v, v']."""
    d = rho.shape[0]
    O4 = O.reshape(d, d, d, d)                     # [s', v', s, v]
    num = np.einsum('twsv,stvw->', O4, rho)
    den = np.einsum('ssvv->', rho)
    return num / den


def physical_rdm(rho, d_A):
    """One-site RDM of the physical boson alone: the auxiliary level traced out of rho[s, s'] with
    s = n * d_A + a, normalised to unit trace (2 x 2)."""
    dp = rho.shape[0] // d_A
    r = np.einsum('iaja->ij', rho.reshape(dp, d_A, dp, d_A))
    return r / np.trace(r)


def renyi(rho_phys, alpha):
    """Renyi entropy S_alpha = ln(Tr rho^alpha) / (1 - alpha) of a normalised density matrix; the
    von Neumann entropy -Tr rho ln rho for alpha = 1 (Sec. "Results for interacting case": Renyi
    entropies of the one-site RDM of the physical site, bounded by ln d_p)."""
    p = np.clip(np.linalg.eigvalsh(0.5 * (rho_phys + rho_phys.conj().T)), 0.0, None)
    p = p[p > 0]
    if alpha == 1.0:
        return float(-np.sum(p * np.log(p)))
    return float(np.log(np.sum(p ** alpha)) / (1.0 - alpha))


def observables(A, B, env, J, V, h, d_A=2):
    """Observables of the checkerboard state (A at (0,0), B at (1,0)); all real FP64."""
    b, n, tau, _ = local_ops(d_A)
    pA, pB = (0, 0), (1, 0)
    rA, rB = rho1(A, env, pA), rho1(B, env, pB)
    nA, nB = expect1(rA, n).real, expect1(rB, n).real
    tzA, tzB = expect1(rA, tau).real, expect1(rB, tau).real
    tnA, tnB = expect1(rA, tau @ n).real, expect1(rB, tau @ n).real
    hb = bond_hamiltonian(J, V, 0.0, d_A)          # hopping + interaction only
    e_bonds = 0.0
    e_bonds += expect2(rho2_h(A, B, env, (0, 0), (1, 0)), hb).real
    e_bonds += expect2(rho2_h(B, A, env, (1, 0), (0, 0)), hb).real
    e_bonds += expect2(rho2_v(A, B, env, (0, 0), (0, 1)), hb).real
    e_bonds += expect2(rho2_v(B, A, env, (0, 1), (0, 0)), hb).real
    energy = 0.5 * (e_bonds + h * (tnA + tnB))
    purA = (np.einsum('st,ts->', rA, rA) / np.trace(rA) ** 2).real
    pA = physical_rdm(rA, d_A)
    return dict(nA=nA, nB=nB, imbalance=nA - nB, imbalance_rel=(nA - nB) / (nA + nB),
                tauzA=tzA, tauzB=tzB, energy=energy, purityA=purA,
                renyi1A=renyi(pA, 1.0), renyi_halfA=renyi(pA, 0.5), renyi2A=renyi(pA, 2.0))
