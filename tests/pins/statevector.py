"""Brute-force PEPS state vector on a small periodic L x L torus (plain einsum over all bonds).

Independent of oracle/ and of the transfer-matrix helper: the amplitude psi(s) is the contraction
of all site tensors A[s, u, l, d, r] with (x, y).r joined to (x+1, y).l and (x, y).d to (x, y+1).u.
"""
import string

import numpy as np


def psi_torus(T, L):
    letters = iter(string.ascii_letters)
    hb = {(x, y): next(letters) for x in range(L) for y in range(L)}
    vb = {(x, y): next(letters) for x in range(L) for y in range(L)}
    phys = {(x, y): next(letters) for x in range(L) for y in range(L)}
    specs, ops = [], []
    for y in range(L):
        for x in range(L):
            specs.append(phys[(x, y)] + vb[(x, (y - 1) % L)] + hb[((x - 1) % L, y)]
                         + vb[(x, y)] + hb[(x, y)])
            ops.append(T[(x, y)])
    out = ''.join(phys[(x, y)] for y in range(L) for x in range(L))
    return np.einsum(','.join(specs) + '->' + out, *ops, optimize=True)


def one_site(T, L, O, p):
    """<psi|O_p|psi>/<psi|psi> with O[t, s] acting as sum_t,s |t><t|O|s><s|."""
    psi = psi_torus(T, L)
    d = psi.shape[0]
    m = np.moveaxis(psi, p[1] * L + p[0], 0).reshape(d, -1)
    return np.einsum('ts,sk,tk->', O, m, m.conj()) / np.vdot(m, m)
