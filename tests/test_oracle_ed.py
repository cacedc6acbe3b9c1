"""Pins of the free-fermion ED oracle (oracle/ed.py) against closed forms and a many-body brute
force, so that a dropped term, a wrong sign or index, or a transposed eigenvector matrix fails."""
import itertools

import numpy as np
import pytest

from inputs import ed_fields
from oracle import ed


def test_zero_hopping_sites_are_eigenvectors():
    """J = 0: every eigenvector is a site vector (IPR 1), occupations never change, so the even
    sites stay full and the odd ones empty; the cumulative IPR counts the states per interval."""
    f = ed_fields(6, 2, 4.0, 0, seed=3)
    out = ed.run(6, 6, 0.0, f, [0.0, 0.7, 3.0])
    assert np.allclose(out["ipr"], 1.0, atol=1e-14)
    assert np.allclose(out["n_even"], 1.0, atol=1e-14) and np.allclose(out["n_odd"], 0.0, atol=1e-14)
    assert abs(out["cum_ipr"].sum() - 36.0) < 1e-12


@pytest.mark.parametrize("L", [6, 8, 12])
def test_clean_chain_closed_form(L):
    """h = 0 chain of L sites (L even): E_a = -2J cos(pi a / (L + 1)) and every eigenvector
    sqrt(2 / (L + 1)) sin(pi a i / (L + 1)) has IPR 3 / (2 (L + 1))."""
    J = 1.3
    E, V = ed.eigensystem(ed.hamiltonian(L, 1, J, np.zeros(L)))
    a = np.arange(1, L + 1)
    assert np.allclose(E, np.sort(-2 * J * np.cos(np.pi * a / (L + 1))), atol=1e-13)
    assert np.allclose(ed.ipr(V), 1.5 / (L + 1), atol=1e-13)


def test_clean_rectangle_spectrum():
    """h = 0 on a 5 x 4 rectangle: E = -2J (cos(pi a / 6) + cos(pi b / 5)), a = 1..5, b = 1..4."""
    E, _ = ed.eigensystem(ed.hamiltonian(5, 4, 1.0, np.zeros(20)))
    ref = np.sort([-2 * (np.cos(np.pi * a / 6) + np.cos(np.pi * b / 5))
                   for a in range(1, 6) for b in range(1, 5)])
    assert np.allclose(E, ref, atol=1e-13)


def test_short_time_law_and_conservation():
    """n_odd(t) = J^2 t^2 (bonds) / (odd sites) + O(t^4), n_even = 1 - J^2 t^2 (bonds) / (even
    sites) + O(t^4) whatever the fields; the particle number is conserved at every time."""
    Lx, Ly, J = 5, 4, 0.9
    f = ed_fields(5, 1, 3.0, 0, seed=1)[0][:Lx * Ly]
    E, V = ed.eigensystem(ed.hamiltonian(Lx, Ly, J, f))
    occ = ed.neel_sites(Lx, Ly)
    bonds = (Lx - 1) * Ly + Lx * (Ly - 1)
    n_even_sites = len(occ)
    n_odd_sites = Lx * Ly - n_even_sites
    t = 1e-3
    n = ed.occupations(E, V, occ, [t, 0.8, 2.5])
    e, o = ed.even_odd(n, Lx, Ly)
    assert abs(o[0] - J * J * t * t * bonds / n_odd_sites) < 1e-10
    assert abs(e[0] - (1 - J * J * t * t * bonds / n_even_sites)) < 1e-10
    assert np.allclose(n.sum(axis=1), len(occ), atol=1e-12)


def _many_body_occupations(Lx, Ly, J, fields, times):
    """Brute force: the Neel state in the fixed-particle-number Fock sector, with fermionic signs
    (Jordan-Wigner order = site index), evolved by the many-body Hamiltonian sum H_ij c_i^+ c_j."""
    h1 = ed.hamiltonian(Lx, Ly, J, fields)
    N = Lx * Ly
    occ = set(ed.neel_sites(Lx, Ly).tolist())
    basis = [s for s in itertools.combinations(range(N), len(occ))]
    index = {s: k for k, s in enumerate(basis)}
    Hm = np.zeros((len(basis), len(basis)))
    for k, s in enumerate(basis):
        ss = set(s)
        for i in range(N):
            for j in range(N):
                if h1[i, j] == 0.0:
                    continue
                if i == j:
                    if i in ss:
                        Hm[k, k] += h1[i, i]
                    continue
                if j not in ss or i in ss:
                    continue
                # c_i^+ c_j |s>: sign (-1)^(occupied sites strictly between i and j)
                lo, hi = min(i, j), max(i, j)
                sign = (-1) ** sum(1 for q in ss if lo < q < hi)
                t_state = tuple(sorted((ss - {j}) | {i}))
                Hm[index[t_state], k] += sign * h1[i, j]
    psi0 = np.zeros(len(basis), dtype=complex)
    psi0[index[tuple(sorted(occ))]] = 1.0
    w, U = np.linalg.eigh(Hm)
    out = []
    for t in times:
        psi = U @ (np.exp(-1j * w * t) * (U.conj().T @ psi0))
        p = np.abs(psi) ** 2
        out.append([sum(p[k] for k, s in enumerate(basis) if i in s) for i in range(N)])
    return np.array(out)


def test_many_body_brute_force_2x3():
    """Single-particle occupations equal the many-fermion evolution on a 3 x 2 lattice (3 fermions,
    20 Fock states, fermion signs included), with disorder, at several times."""
    Lx, Ly = 3, 2
    f = np.array([0.7, -1.1, 0.3, 1.9, -0.4, 0.05])
    times = [0.0, 0.37, 1.2, 4.0]
    mb = _many_body_occupations(Lx, Ly, 1.0, f, times)
    E, V = ed.eigensystem(ed.hamiltonian(Lx, Ly, 1.0, f))
    sp = ed.occupations(E, V, ed.neel_sites(Lx, Ly), times)
    assert np.allclose(sp, mb, atol=1e-12)


def test_cumulative_ipr_bins():
    """Interval sums: the total over the intervals is the total IPR; E_max lands in the last
    interval, E_min in the first; a state at eps = 0.5 lands in interval 10."""
    E = np.array([-2.0, -1.0, 0.0, 0.5, 2.0])
    I = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    c = ed.cumulative_ipr(E, I)
    assert len(c) == 20 and abs(c.sum() - 1.5) < 1e-15
    assert c[0] == 0.1 and c[19] == 0.5 and c[10] == 0.3 and c[5] == 0.2
    assert c[12] == 0.4          # eps = 2.5 / 4 = 0.625 -> interval 12


def test_ed_fields_recipe():
    """The seeded on-site fields: continuous ones uniform in [-h, h]; discrete ones only the levels
    -h + 2 h k / (s - 1), all of them used, each with frequency near 1 / s; reproducible by seed."""
    c = ed_fields(20, 50, 4.0, 0, seed=2)
    assert c.shape == (50, 400) and c.min() >= -4.0 and c.max() <= 4.0
    assert abs(c.mean()) < 0.05 and abs(c.var() - 16.0 / 3.0) < 0.1
    d = ed_fields(20, 50, 10.0, 3, seed=2)
    vals, counts = np.unique(d, return_counts=True)
    assert np.allclose(vals, [-10.0, 0.0, 10.0])
    assert np.all(np.abs(counts / d.size - 1.0 / 3.0) < 0.01)
    assert np.array_equal(ed_fields(6, 3, 1.0, 0, seed=9), ed_fields(6, 3, 1.0, 0, seed=9))
