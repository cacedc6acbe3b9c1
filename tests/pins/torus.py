"""Exact contraction of a PEPS norm network on a periodic L x L torus by row transfer matrices.

Independent of oracle/: site tensors A[s, u, l, d, r], checkerboard (A on x + y even).  Sites are
listed row by row; a row transfer matrix maps the L up-legs (ket x bra) to the L down-legs.
Used for the pin "CTMRG matches brute-force contraction of a small periodic PEPS".
"""
import numpy as np


def _dl(A, Oket=None):
    """Double layer with an optional operator sandwiched: sum_{s,s'} A[s] O[s', s] conj(A[s'])."""
    d, D = A.shape[0], A.shape[1]
    if Oket is None:
        Oket = np.eye(d)
    t = np.einsum('suldr,ts,tvmew->uvlmderw', A, Oket, A.conj())
    return t.reshape(D * D, D * D, D * D, D * D)


def _row(tensors):
    """Row transfer matrix from L double layers [U, L, D, R] with periodic horizontal bonds."""
    t = tensors[0]                                  # [u0, l0, d0, r0]
    D2 = t.shape[0]
    acc = t.transpose(1, 0, 2, 3)                   # [l0, u0, d0, r]
    acc = acc.reshape(D2, D2, D2, D2)
    ups, downs = 1, 1
    acc = acc.reshape(D2, D2, D2, D2)               # [l0, U, Dn, r]
    for t in tensors[1:]:
        # acc[l0, U, Dn, r] x t[u, r, d, r'] -> [l0, U u, Dn d, r']
        acc = np.einsum('aUDr,urdz->aUuDdz', acc, t)
        s = acc.shape
        acc = acc.reshape(s[0], s[1] * s[2], s[3] * s[4], s[5])
    acc = np.einsum('aUDa->UD', acc)                # close the periodic bond
    return acc


def expectation(A, B, L, ops):
    """<prod O> on the L x L torus; ops maps (x, y) -> d x d operator (others identity)."""
    rows = []
    for y in range(L):
        ts = []
        for x in range(L):
            site = A if (x + y) % 2 == 0 else B
            ts.append(_dl(site, ops.get((x, y))))
        rows.append(_row(ts))
    M = rows[0]
    for r in rows[1:]:
        M = M @ r
    return np.trace(M)


def one_site(A, B, L, O, p=(0, 0)):
    return expectation(A, B, L, {p: O}) / expectation(A, B, L, {})


def two_site(A, B, L, O1, O2, p, q):
    return expectation(A, B, L, {p: O1, q: O2}) / expectation(A, B, L, {})
