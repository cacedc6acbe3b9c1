"""Exact dynamics of the disordered hard-core boson model on the 8-site tilted square cluster.

Cluster: the square lattice modulo the vectors (2, 2) and (2, -2) -- 8 sites, each with four
distinct nearest neighbours, bipartite (the checkerboard survives the periodic identification).
A plain 2 x 4 torus would double the bonds across its width-2 direction, which changes the
O(t^2) coefficient of the imbalance; the tilted cluster keeps the infinite lattice's local
structure up to loops that wrap the torus.

The exact disorder average of the dilated model equals the uniform mean over all d_A^8 auxiliary
configurations of the plain boson model with fields h tau_i, tau_i in the d_A levels
1 - 2 a / (d_A - 1) (+1, -1 for d_A = 2; +1, 0, -1 for d_A = 3) (Sec. "Set up for iPEPS", Readout).
Each configuration is evolved from the CDW (4 particles on sublattice A) in the 70-dimensional
N = 4 sector by exact eigendecomposition.
"""
import itertools

import numpy as np


def cluster():
    def canon(p):
        x, y = p
        m = int(np.floor((x + y) / 4.0))
        n = int(np.floor((x - y) / 4.0))
        return (x - 2 * m - 2 * n, y - 2 * m + 2 * n)

    sites = sorted({canon((x, y)) for x in range(-4, 5) for y in range(-4, 5)})
    assert len(sites) == 8
    index = {s: i for i, s in enumerate(sites)}
    bonds = set()
    for s in sites:
        nbrs = {canon((s[0] + dx, s[1] + dy)) for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1))}
        assert len(nbrs) == 4
        for t in nbrs:
            bonds.add(tuple(sorted((index[s], index[t]))))
    assert len(bonds) == 16
    sub = [(s[0] + s[1]) % 2 for s in sites]        # 0 = A (occupied initially), 1 = B
    return sites, sorted(bonds), sub


def imbalance(J, V, h, times, d_A=2):
    sites, bonds, sub = cluster()
    L = len(sites)
    basis = [c for c in itertools.combinations(range(L), L // 2)]
    idx = {c: i for i, c in enumerate(basis)}
    nb = len(basis)
    occ = np.array([[1.0 if i in c else 0.0 for i in range(L)] for c in basis])
    Hkin = np.zeros((nb, nb))
    Hint = np.zeros(nb)
    for k, c in enumerate(basis):
        cs = set(c)
        for i, j in bonds:
            Hint[k] += V * occ[k, i] * occ[k, j]
            for a, b in ((i, j), (j, i)):
                if a in cs and b not in cs:
                    new = tuple(sorted((cs - {a}) | {b}))
                    Hkin[idx[new], k] += -J
    psi0 = np.zeros(nb)
    psi0[idx[tuple(i for i in range(L) if sub[i] == 0)]] = 1.0
    A = np.array([i for i in range(L) if sub[i] == 0])
    B = np.array([i for i in range(L) if sub[i] == 1])
    out = np.zeros(len(times))
    levels = [1.0 - 2.0 * a / (d_A - 1) for a in range(d_A)]
    for taus in itertools.product(levels, repeat=L):
        H = Hkin + np.diag(Hint + h * occ @ np.array(taus))
        w, W = np.linalg.eigh(H)
        c0 = W.T @ psi0
        for it, t in enumerate(times):
            psi = W @ (np.exp(-1j * w * t) * c0)
            n = (np.abs(psi) ** 2) @ occ
            out[it] += n[A].mean() - n[B].mean()
    return out / d_A ** L
