"""Pins for the Renyi entropies of the physical one-site RDM (oracle/measure.py).

The paper reads out Renyi entropies of the one-site reduced density matrix of the physical site
(Sec. "Results for interacting case"), bounded by ln d_p = ln 2.  Particle number is conserved by
every gate and the CDW start has a definite number on every site, so the physical one-site RDM is
diagonal in the occupation basis: rho_phys = diag(1 - n_A, n_A).  Its entropies are then fixed by
the independently measured occupation n_A through the binary-entropy closed forms

    S_1   = -p ln p - (1 - p) ln(1 - p),
    S_1/2 = 2 ln(sqrt(p) + sqrt(1 - p)),
    S_2   = -ln(p^2 + (1 - p)^2),          p = n_A.

A mistake in the auxiliary trace (tracing the occupation instead of the level, or the wrong index
order of s = n d_A + a) or in the entropy formula breaks this identity.  J = 0 keeps the product
state: every entropy is 0.  A maximally mixed qubit gives ln 2 for every alpha.
"""
import numpy as np
import pytest

from oracle import evolve, measure


def _binary(p):
    q = 1.0 - p
    s1 = -sum(x * np.log(x) for x in (p, q) if x > 0)
    return dict(renyi1A=s1, renyi_halfA=2 * np.log(np.sqrt(p) + np.sqrt(q)),
                renyi2A=-np.log(p * p + q * q))


@pytest.mark.parametrize("d_A", [2, 3])
def test_entropies_follow_the_occupation(d_A):
    p = dict(J=1.0, V=1.0, h=5.0, D=2, chi=8, order=2, dt=0.02, t_max=0.2, meas_every=0.05, d_A=d_A)
    out = evolve.run(p, tol=1e-11)
    grew = False
    for o in out:
        want = _binary(o["nA"])
        for k, v in want.items():
            assert abs(o[k] - v) < 1e-10, (o["t"], k, o[k], v)
            assert -1e-14 <= o[k] <= np.log(2) + 1e-12
        grew = grew or o["renyi1A"] > 1e-3
    assert grew                                       # the evolution entangles the site


def test_zero_hopping_keeps_product_state():
    p = dict(J=0.0, V=1.0, h=5.0, D=2, chi=8, order=1, dt=0.05, t_max=0.2, meas_every=0.1)
    for o in evolve.run(p, tol=1e-11):
        assert abs(o["renyi1A"]) < 1e-14 and abs(o["renyi_halfA"]) < 1e-14 and abs(o["renyi2A"]) < 1e-14


def test_maximally_mixed_and_pure_qubit():
    d_A = 2
    rho = np.kron(np.eye(2) / 2, np.eye(d_A) / d_A)      # s = n * d_A + a
    r = measure.physical_rdm(rho, d_A)
    for a in (1.0, 0.5, 2.0):
        assert abs(measure.renyi(r, a) - np.log(2)) < 1e-14
    pure = np.zeros((4, 4))
    pure[2, 2] = 1.0                                     # n = 1, a = 0
    assert np.allclose(measure.physical_rdm(pure, d_A), [[0, 0], [0, 1]])
    for a in (1.0, 0.5, 2.0):
        assert abs(measure.renyi(measure.physical_rdm(pure, d_A), a)) < 1e-14
