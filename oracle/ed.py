"""Free-fermion exact diagonalisation (paper Sec. "Set up for non-interacting fermions"; Sec.
"Results", non-interacting case, Fig. 2-4).  TEST INFRASTRUCTURE ONLY (see the package header).

The non-interacting limit of the lattice model on a finite L_x x L_y square lattice: one particle
hops with amplitude J between nearest neighbours and feels the on-site field h_i of its site,

    H_ij = -J  (i, j nearest neighbours),     H_ii = h_i,

with open boundaries (the paper's finite systems; it does not state the boundary condition).  The
fields are drawn outside (inputs.ed_fields): continuous, uniform in [-h, h], or discrete with s
equally spaced levels in [-h, h] (the paper's spin-1 case is s = 3).  Site index i = x + L_x y.

Because the dynamics stays in the single-particle sector, the many-fermion Neel state (every site
with x + y even occupied) evolves through the single-particle propagator U(t) = exp(-i H t):

    n_i(t) = sum over occupied j of |U(t)_ij|^2,    U(t) = V diag(exp(-i E_k t)) V^T

from the eigen-decomposition H = V diag(E) V^T (LAPACK eigh).  The readouts are the mean particle
number on the even and on the odd sites (Fig. 2).

Localisation of the eigenvectors (Eq. IPR): I_k = sum_i |<i|E_k>|^4; the spectrum is rescaled to
eps_k = (E_k - E_min) / (E_max - E_min) in [0, 1] and the I_k of the states in each interval of
width 0.05 are summed (the cumulative IPR, Fig. 4), per realisation; realisations are averaged.
There are ceil(1 / width) intervals and eps = 1 belongs to the last one.

Pins (tests/test_oracle_ed.py): J = 0 (site eigenvectors, IPR 1, frozen occupations), the clean
chain and clean rectangle (closed-form spectrum and IPR), the short-time law
n_odd = J^2 t^2 (bonds) / (odd sites) + O(t^4), particle-number conservation, and a many-body
brute force on a 2 x 3 lattice (3 fermions, the full 20-state Fock sector with fermion signs).
"""
import numpy as np


def hamiltonian(Lx, Ly, J, fields):
    """Single-particle Hamiltonian, open boundaries, site i = x + Lx y."""
    N = Lx * Ly
    H = np.diag(np.asarray(fields, dtype=np.float64)).copy()
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            if x + 1 < Lx:
                H[i, i + 1] = H[i + 1, i] = -J
            if y + 1 < Ly:
                H[i, i + Lx] = H[i + Lx, i] = -J
    return H


def neel_sites(Lx, Ly):
    """Occupied sites of the Neel state: x + y even."""
    return np.array([x + Lx * y for y in range(Ly) for x in range(Lx) if (x + y) % 2 == 0])


def parity(Lx, Ly):
    """+1 on even sites (x + y even), -1 on odd ones."""
    return np.array([1 if (x + y) % 2 == 0 else -1 for y in range(Ly) for x in range(Lx)])


def eigensystem(H):
    """E ascending, V[:, k] the eigenvector of E[k] (LAPACK eigh)."""
    return np.linalg.eigh(H)


def occupations(E, V, occ, times):
    """n_i(t) for every time: [len(times)][N]."""
    out = []
    Vo = V[occ, :]                                   # rows of the occupied sites
    for t in times:
        U = (V * np.exp(-1j * E * t)) @ Vo.T         # U[:, j] = exp(-iHt) e_j, j occupied
        out.append(np.sum(np.abs(U) ** 2, axis=1))
    return np.array(out)


def even_odd(n, Lx, Ly):
    """Mean occupation over the even and over the odd sites of each row of n."""
    p = parity(Lx, Ly)
    return n[:, p > 0].mean(axis=1), n[:, p < 0].mean(axis=1)


def ipr(V):
    """I_k = sum_i |V_ik|^4 for every eigenvector."""
    return np.sum(np.abs(V) ** 4, axis=0)


def cumulative_ipr(E, I, width=0.05):
    """Sum of I_k over the states in each interval of the rescaled spectrum (1 / width bins)."""
    nb = int(np.ceil(1.0 / width - 1e-9))          # intervals covering [0, 1]
    span = E[-1] - E[0] if len(E) > 1 else 0.0
    eps = (E - E[0]) / span if span > 0 else np.zeros_like(E)
    b = np.minimum((eps / width).astype(int), nb - 1)
    out = np.zeros(nb)
    np.add.at(out, b, I)
    return out


def run(Lx, Ly, J, fields, times, width=0.05):
    """All readouts for a batch of realisations fields[R][N]: the realisation-averaged even / odd
    occupations [T] each, the averaged cumulative IPR [1 / width], and per realisation the
    spectrum [R][N] and the IPRs [R][N]."""
    occ = neel_sites(Lx, Ly)
    ev, od, cum, spec, iprs = [], [], [], [], []
    for f in np.atleast_2d(fields):
        E, V = eigensystem(hamiltonian(Lx, Ly, J, f))
        n = occupations(E, V, occ, times)
        e, o = even_odd(n, Lx, Ly)
        I = ipr(V)
        ev.append(e); od.append(o); cum.append(cumulative_ipr(E, I, width))
        spec.append(E); iprs.append(I)
    return dict(n_even=np.mean(ev, axis=0), n_odd=np.mean(od, axis=0), cum_ipr=np.mean(cum, axis=0),
                spectra=np.array(spec), ipr=np.array(iprs))
