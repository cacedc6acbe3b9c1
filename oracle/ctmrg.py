"""Directional CTMRG with full 2x2-block projectors, explicit double layer (FP64, plain NumPy).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Paper: Sec. "Set up for iPEPS" (Readout) and the Appendix use CTMRG (Orus & Vidal, PRB 80, 094403
(2009); Orus, PRB 85, 205117 (2012); Nishino & Okunishi 1996/97) to contract the infinite lattice
around a site into fixed-point corner and edge tensors, with environment dimension chi >= D^2,
"sufficiently well converged".  The projectors follow Corboz, Rice & Troyer, PRL 113, 046402 (2014):
from the four enlarged corners Q1..Q4 of a 2x2 block, R = Q3 Q4 (lower half) and R~ = Q1 Q2 (upper
half) are contracted over the bond to be truncated, M = R R~ = U S V^+, and

    P = R~ V S^{-1/2}   (attached to the lower side of the cut)
    P~ = S^{-1/2} U^+ R (attached to the upper side of the cut)

so that P~ P = 1 and R P P~ R~ is the best rank-chi approximation of M.

Unit cell Lx x Ly (here 2 x 2 with A on x+y even, B on x+y odd).  Coordinates: x grows to the
right, y grows downwards.

Tensor conventions (every environment index order follows the clockwise walk around the site
C1 -> T1 -> C2 -> T2 -> C3 -> T3 -> C4 -> T4 -> C1; the last index of each tensor joins the first
index of the next; chi indices first/last, the D^2 index in the middle):

    C1[c_T4, c_T1]      T1[left, k_U, right]
    C2[c_T1, c_T2]      T2[up,   k_R, down]
    C3[c_T2, c_T3]      T3[right, k_D, left]
    C4[c_T3, c_T4]      T4[down, k_L, up]

    double layer a[U, L, D, R], each index (ket, bra) -> ket * D + bra, dimension D^2.

A 90-degree counter-clockwise rotation of the lattice maps site (x, y) to (y, -x), the site tensor
to a.transpose(3, 0, 1, 2), and the environment (C1..C4, T1..T4) to (C2, C3, C4, C1; T2, T3, T4, T1)
with no index permutation -- so one left move plus rotations gives all four directional moves.

Degenerate singular values at the cut are kept or dropped as whole multiplets; singular values
below cut_rel of the largest are dropped (pseudo-inverse); the kept rank is zero-padded to chi.  The
paper fixes no cutoff; the default PROJ_CUT_REL = 1e-10 keeps the early-time physics (a cutoff of
1e-6 biases I(t = 0.01) by 6e-7).  Rounding in the singular vectors of M is amplified by about
eps s_1 / (s_K gap) in the projectors, so when the cut falls in a cluster of tiny singular values the
fixed point depends on rounding (D = 2 quench workload, t >= 0.7: 1e-8 shifts under a 1e-15 change of the
gates); a larger cutoff such as 1e-6 removes that sensitivity.

Parity: pinned by tests/test_oracle_ctmrg.py (Ising PEPS against Onsager/Yang, exact dimer states,
brute-force contraction of small periodic tori, product states at chi = 1, rotation invariance).
"""
import functools

import numpy as np

from .su import DEGEN_RTOL, TINY_REL, truncation_rank

# every contraction below is a pairwise (or three-operand) einsum; optimize=True lets NumPy hand
# each pairwise step to BLAS and changes nothing but speed
ein = functools.partial(np.einsum, optimize=True)

PROJ_CUT_REL = 1e-10
# Multiplets at the chi cut (C8 reading): a computed singular value of M is accurate to about
# eps * s_1 in absolute terms, so for values below ~1e-5 s_1 a relative gap of 1e-10 lies inside the
# rounding noise; two values whose absolute gap is below PROJ_DEGEN_ABS * s_1 also count as one
# multiplet, so that the decision does not depend on rounding.
PROJ_DEGEN_ABS = 1e-11


# ----------------------------------------------------------------------------- double layer
def double_layer(A):
    """a[(u u'), (l l'), (d d'), (r r')] = sum_s A[s,u,l,d,r] conj(A[s,u',l',d',r'])."""
    D = A.shape[1]
    a = ein('suldr,svmew->uvlmderw', A, A.conj())
    return a.reshape(D * D, D * D, D * D, D * D)


def double_layer_open(A):
    """Open double layer ao[s, s', U, L, D, R] (physical ket/bra indices kept)."""
    D = A.shape[1]
    ao = ein('suldr,tvmew->stuvlmderw', A, A.conj())
    return ao.reshape(A.shape[0], A.shape[0], D * D, D * D, D * D, D * D)


def _trace_pair(a, D, axes):
    """Trace the ket/bra pair of each leg in ``axes`` of a double-layer tensor; keep the rest."""
    t = a.reshape([D, D] * 4)
    letters = 'abcdefgh'
    spec_in = ''
    spec_out = ''
    for leg in range(4):
        k, b = letters[2 * leg], letters[2 * leg + 1]
        if leg in axes:
            spec_in += k + k
        else:
            spec_in += k + b
            spec_out += k + b
    out = ein(spec_in + '->' + spec_out, t)
    return out.reshape([D * D] * (4 - len(axes)))


# ----------------------------------------------------------------------------- environment
class Env:
    """Corner and edge tensors per unit-cell site: C[i][(x, y)], T[i][(x, y)], i = 0..3 (C1..C4)."""

    def __init__(self, Lx, Ly, C, T):
        self.Lx, self.Ly = Lx, Ly
        self.C, self.T = C, T

    def copy(self):
        return Env(self.Lx, self.Ly, [dict((k, v.copy()) for k, v in c.items()) for c in self.C],
                   [dict((k, v.copy()) for k, v in t.items()) for t in self.T])


def _pad(t, shape):
    out = np.zeros(shape, dtype=np.complex128)
    out[tuple(slice(0, n) for n in t.shape)] = t
    return out


def init_env(a, Lx, Ly, chi, D):
    """Initial environment: each outward ket/bra leg pair of the neighbouring double layer traced,
    giving chi_init = D^2, zero-padded to chi.  a[(x, y)] are the double layers."""
    if chi < D * D:
        raise ValueError("chi must be >= D^2")
    D2 = D * D
    C = [{}, {}, {}, {}]
    T = [{}, {}, {}, {}]
    for x in range(Lx):
        for y in range(Ly):
            def at(dx, dy):
                return a[((x + dx) % Lx, (y + dy) % Ly)]
            # corners: keep the two inner legs, ordered clockwise
            C[0][(x, y)] = _pad(_trace_pair(at(-1, -1), D, (0, 1)), (chi, chi))   # [D, R]
            c2 = _trace_pair(at(1, -1), D, (0, 3))                                # [L, D]
            C[1][(x, y)] = _pad(c2, (chi, chi))
            c3 = _trace_pair(at(1, 1), D, (2, 3))                                 # [U, L]
            C[2][(x, y)] = _pad(c3, (chi, chi))
            c4 = _trace_pair(at(-1, 1), D, (1, 2))                                # [U, R]
            C[3][(x, y)] = _pad(c4.T, (chi, chi))                                 # [R, U]
            # edges
            t1 = _trace_pair(at(0, -1), D, (0,))                                  # [L, D, R]
            T[0][(x, y)] = _pad(t1, (chi, D2, chi))
            t2 = _trace_pair(at(1, 0), D, (3,))                                   # [U, L, D]
            T[1][(x, y)] = _pad(t2, (chi, D2, chi))
            t3 = _trace_pair(at(0, 1), D, (2,))                                   # [U, L, R]
            T[2][(x, y)] = _pad(np.transpose(t3, (2, 0, 1)), (chi, D2, chi))      # [R, U, L]
            t4 = _trace_pair(at(-1, 0), D, (1,))                                  # [U, D, R]
            T[3][(x, y)] = _pad(np.transpose(t4, (1, 2, 0)), (chi, D2, chi))      # [D, R, U]
    return Env(Lx, Ly, C, T)


def rotate(a, env):
    """Rotate the whole network by 90 degrees counter-clockwise: (x, y) -> (y, -x)."""
    Lx, Ly = env.Lx, env.Ly

    def np_(p):
        return (p[1] % Ly, (-p[0]) % Lx)

    a2 = {np_(p): np.transpose(t, (3, 0, 1, 2)) for p, t in a.items()}
    C2 = [{np_(p): t for p, t in env.C[(i + 1) % 4].items()} for i in range(4)]
    T2 = [{np_(p): t for p, t in env.T[(i + 1) % 4].items()} for i in range(4)]
    return a2, Env(Ly, Lx, C2, T2)


# ----------------------------------------------------------------------------- enlarged corners
def corner_q1(C1, T1, T4, a):
    """Q1[(e4, kD), (e1, kR)] = C1[c4,c1] T1[c1,kU,e1] T4[e4,kL,c4] a[kU,kL,kD,kR]."""
    x = ein('pc,cue->pue', C1, T1)
    x = ein('flp,pue->fleu', T4, x)
    x = ein('fleu,ulkr->fker', x, a)
    chi, D2 = C1.shape[0], a.shape[0]
    return x.reshape(chi * D2, chi * D2)


def corner_q2(T1, C2, T2, a):
    """Q2[(e1, kL), (e2, kD)] = T1[e1,kU,c1] C2[c1,c2] T2[c2,kR,e2] a[kU,kL,kD,kR]."""
    x = ein('euc,cp->eup', T1, C2)
    x = ein('eup,prf->eurf', x, T2)
    x = ein('eurf,ulkr->elfk', x, a)
    chi, D2 = C2.shape[0], a.shape[0]
    return x.reshape(chi * D2, chi * D2)


def corner_q3(T2, C3, T3, a):
    """Q3[(e2, kU), (e3, kL)] = T2[e2,kR,c2] C3[c2,c3] T3[c3,kD,e3] a[kU,kL,kD,kR]."""
    x = ein('erc,cp->erp', T2, C3)
    x = ein('erp,pkf->erkf', x, T3)
    x = ein('erkf,ulkr->eufl', x, a)
    chi, D2 = C3.shape[0], a.shape[0]
    return x.reshape(chi * D2, chi * D2)


def corner_q4(T3, C4, T4, a):
    """Q4[(e3, kR), (e4, kU)] = T3[e3,kD,c3] C4[c3,c4] T4[c4,kL,e4] a[kU,kL,kD,kR]."""
    x = ein('ekc,cp->ekp', T3, C4)
    x = ein('ekp,plf->eklf', x, T4)
    x = ein('eklf,ulkr->erfu', x, a)
    chi, D2 = C4.shape[0], a.shape[0]
    return x.reshape(chi * D2, chi * D2)


# ----------------------------------------------------------------------------- projectors
def cut_margin(s, chi, cut_rel=PROJ_CUT_REL, degen_rtol=DEGEN_RTOL, degen_abs=PROJ_DEGEN_ABS):
    """How far, in decades, the multiplet decisions at the chi cut lie from their thresholds.

    For every pair (s[K-1], s[K]) the multiplet rule examines while it moves the cut down, with
    s[K] above the cutoff (below it the cutoff decides anyway), the decision is "relative gap <
    degen_rtol or absolute gap < degen_abs * s_1"; its margin is |log10| of the ratio of the deciding
    threshold to the gap.  Returns the smallest margin (inf when no such pair exists).  A small
    margin means the decision can go either way under rounding (C8)."""
    m = np.inf
    K = min(chi, len(s))
    if not s[0] > 0:
        return m
    while 1 < K < len(s) and s[K] > max(TINY_REL, cut_rel) * s[0]:
        rel = max(s[K - 1] / s[K] - 1.0, 1e-300)
        ab = max((s[K - 1] - s[K]) / s[0], 1e-300)
        d = max(np.log10(degen_rtol / rel), np.log10(degen_abs / ab))   # > 0: multiplet
        m = min(m, abs(d))
        if d <= 0:
            break
        K -= 1
    return m


def projectors(R, Rt, chi, cut_rel=PROJ_CUT_REL, log=None):
    """Full-SVD projectors for the bond joining R (columns) and R~ (rows); returns (P, P~, s).

    s is the full singular spectrum of M = R R~ (for diagnostics).  When ``log`` is a list it
    receives (cut_margin() of this cut, s_K / s_1 for the largest value the multiplet rule moved
    out of the kept set where the cutoff would have kept it, else 0)."""
    M = R @ Rt
    U, s, Vh = np.linalg.svd(M)
    K = truncation_rank(s, chi, degen_abs=PROJ_DEGEN_ABS)
    if log is not None:
        moved = s[0] > 0 and K < min(chi, len(s)) and s[K] > cut_rel * s[0]
        log.append((cut_margin(s, chi, cut_rel), float(s[K] / s[0]) if moved else 0.0))
    K = min(K, int(np.sum(s > cut_rel * s[0]))) if s[0] > 0 else 0
    K = max(K, 1) if s[0] > 0 else 0
    N = R.shape[1]
    P = np.zeros((N, chi), dtype=np.complex128)
    Pt = np.zeros((chi, N), dtype=np.complex128)
    if K > 0:
        isq = 1.0 / np.sqrt(s[:K])
        P[:, :K] = (Rt @ Vh[:K].conj().T) * isq[None, :]
        Pt[:K] = (U[:, :K].conj().T @ R) * isq[:, None]
    return P, Pt, s


def _normalize(t):
    m = np.max(np.abs(t))
    return t / m if m > 0 else t


def left_move(a, env, x, chi, cut_rel=PROJ_CUT_REL, log=None):
    """Absorb column x into the left environment of column x+1 (all rows)."""
    Lx, Ly = env.Lx, env.Ly
    C, T = env.C, env.T
    xp = (x + 1) % Lx
    D2 = a[(0, 0)].shape[0]
    P, Pt = {}, {}
    for y in range(Ly):
        yp = (y + 1) % Ly
        q1 = corner_q1(C[0][(x, y)], T[0][(x, y)], T[3][(x, y)], a[(x, y)])
        q2 = corner_q2(T[0][(xp, y)], C[1][(xp, y)], T[1][(xp, y)], a[(xp, y)])
        q3 = corner_q3(T[1][(xp, yp)], C[2][(xp, yp)], T[2][(xp, yp)], a[(xp, yp)])
        q4 = corner_q4(T[2][(x, yp)], C[3][(x, yp)], T[3][(x, yp)], a[(x, yp)])
        R = q3 @ q4       # rows: bond Q2|Q3, columns: the cut (bond Q4|Q1)
        Rt = q1 @ q2      # rows: the cut, columns: bond Q2|Q3
        P[y], Pt[y], _ = projectors(R, Rt, chi, cut_rel, log)
    newC1, newT4, newC4 = {}, {}, {}
    for y in range(Ly):
        ym = (y - 1) % Ly
        c1t1 = ein('pc,cue->pue', C[0][(x, y)], T[0][(x, y)]).reshape(chi * D2, chi)
        newC1[y] = Pt[ym] @ c1t1
        t4a = ein('flp,ulkr->fkrpu', T[3][(x, y)], a[(x, y)]).reshape(chi * D2, D2, chi * D2)
        newT4[y] = ein('cm,mkn,nf->ckf', Pt[y], t4a, P[ym])
        t3c4 = ein('ekc,cp->epk', T[2][(x, y)], C[3][(x, y)]).reshape(chi, chi * D2)
        newC4[y] = t3c4 @ P[y]
    for y in range(Ly):
        C[0][(xp, y)] = _normalize(newC1[y])
        T[3][(xp, y)] = _normalize(newT4[y])
        C[3][(xp, y)] = _normalize(newC4[y])


def sweep(a, env, chi, cut_rel=PROJ_CUT_REL, log=None):
    """One CTMRG sweep: left, top, right and bottom moves, each over every column (16 projector
    computations on the 2x2 cell, always in the same order)."""
    for _ in range(4):
        for x in range(env.Lx):
            left_move(a, env, x, chi, cut_rel, log)
        a, env = rotate(a, env)
    return env


def corner_spectra(env, chi):
    """Normalised singular values of every corner, zero-padded to chi: dict (i, x, y) -> array."""
    out = {}
    for i in range(4):
        for p, c in env.C[i].items():
            s = np.linalg.svd(c, compute_uv=False)
            v = np.zeros(chi)
            if s[0] > 0:
                v[:len(s)] = s / s[0]
            out[(i, p)] = v
    return out


def spectra_delta(s_new, s_old):
    """Convergence number: max over corners of the 2-norm change of the normalised spectrum."""
    return max(np.linalg.norm(s_new[k] - s_old[k]) for k in s_new)


STALL_WINDOW = 10      # sweeps without a factor-2 improvement of the best delta
STALL_MAX = 1e-7       # ... counted as a stall only while the best and the current delta are below this
STALL_GROWTH = 4.0     # ... and while the current delta is within this factor of the best one


def ctmrg(a, env, chi, tol=1e-10, max_sweeps=200, min_sweeps=1, cut_rel=PROJ_CUT_REL,
          stall_window=STALL_WINDOW, stall_max=STALL_MAX, log=None):
    """Sweep until the corner spectra change by less than ``tol``; returns (env, sweeps, delta).

    The paper asks for a "sufficiently well-converged" environment (Appendix).  Reading: stop at
    delta < tol, or when delta has stalled at its rounding floor -- no factor-2 improvement of the
    best delta for ``stall_window`` sweeps while that best is already below ``stall_max`` and the
    current delta still sits at that floor (below ``stall_max`` and within a factor
    ``STALL_GROWTH`` of the best).  A delta that grows again after coming close to a fixed point
    means the run is leaving an unstable fixed point, not sitting at a rounding floor; such a run
    goes on sweeping.  With tol <= 0 exactly max_sweeps sweeps run (no stall test)."""
    prev = corner_spectra(env, chi)
    delta = np.inf
    best, since = np.inf, 0
    n = 0
    for n in range(1, max_sweeps + 1):
        env = sweep(a, env, chi, cut_rel, log)
        cur = corner_spectra(env, chi)
        delta = spectra_delta(cur, prev)
        prev = cur
        if n >= min_sweeps and delta < tol:
            break
        if delta < 0.5 * best:
            best, since = delta, 0
        else:
            since += 1
        if (tol > 0 and since >= stall_window and best < stall_max and delta < stall_max
                and delta <= STALL_GROWTH * best):
            break
    return env, n, delta


def checkerboard(A, B):
    """Site tensors of the 2x2 unit cell: A on x + y even, B on x + y odd."""
    return {(x, y): (A if (x + y) % 2 == 0 else B) for x in range(2) for y in range(2)}
