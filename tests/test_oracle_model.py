"""Pins for oracle/model.py: operators, bond Hamiltonian and Trotter gate.

The gate is checked against the closed-form exponential of its 2x2 one-particle block and the
diagonal phases of the empty / doubly-occupied pairs, for every auxiliary configuration, plus
unitarity, the group property and the conservation laws of the dilated model (Sec. "Set up for
iPEPS", Eq. Hanc; the tau operators commute with H, particle number is conserved).
"""
import numpy as np
import pytest

from oracle import model


@pytest.mark.parametrize("d_A", [2, 3])
def test_local_operators(d_A):
    b, n, tau, I = model.local_ops(d_A)
    d = 2 * d_A
    assert np.allclose(b @ b, 0)                      # hard core
    assert np.allclose(np.diag(n).real, [0] * d_A + [1] * d_A)
    assert np.allclose(b.conj().T @ b + b @ b.conj().T, I)  # single-mode hard-core anticommutator
    lv = np.diag(tau).real[:d_A]
    assert lv[0] == 1.0 and lv[-1] == -1.0            # field levels span [-h, h]
    assert np.allclose(np.diff(lv), -2.0 / (d_A - 1))


def _closed_form_gate(J, V, h, delta, tA, tB):
    """Gate on the (n_A, n_B) pair for fixed auxiliary levels tA, tB, written out by hand.

    |00>: no energy.  |11>: V + (h/4)(tA + tB).  {|10>, |01>}: H2 = [[eA, -J], [-J, eB]] with
    eA = h tA / 4, eB = h tB / 4; exp(-i H2 delta) = e^{-i m delta} (cos(w delta) - i sin(w delta)
    (H2 - m) / w), m = (eA + eB)/2, w = sqrt(((eA - eB)/2)^2 + J^2)."""
    eA, eB = h * tA / 4, h * tB / 4
    m = 0.5 * (eA + eB)
    w = np.sqrt((0.5 * (eA - eB)) ** 2 + J ** 2)
    H2 = np.array([[eA, -J], [-J, eB]], dtype=complex)
    if w > 0:
        blk = np.exp(-1j * m * delta) * (np.cos(w * delta) * np.eye(2)
                                         - 1j * np.sin(w * delta) / w * (H2 - m * np.eye(2)))
    else:
        blk = np.exp(-1j * m * delta) * np.eye(2)
    return {"00": 1.0, "11": np.exp(-1j * (V + eA + eB) * delta), "1p": blk}


@pytest.mark.parametrize("J,V,h,delta", [(1.0, 1.0, 5.0, 0.02), (0.7, 0.0, 10.0, 0.05),
                                         (-1.3, 2.0, 1.0, 0.1), (0.0, 1.0, 3.0, 0.3)])
def test_gate_closed_form(J, V, h, delta):
    d_A = 2
    d = 4
    U = model.gate(J, V, h, delta, d_A).reshape(d, d, d, d)   # [sA', sB', sA, sB]
    levels = [1.0, -1.0]
    for aA in range(d_A):
        for aB in range(d_A):
            ref = _closed_form_gate(J, V, h, delta, levels[aA], levels[aB])
            s00 = (0 * d_A + aA, 0 * d_A + aB)
            s11 = (1 * d_A + aA, 1 * d_A + aB)
            s10 = (1 * d_A + aA, 0 * d_A + aB)
            s01 = (0 * d_A + aA, 1 * d_A + aB)
            assert abs(U[s00 + s00] - ref["00"]) < 1e-14
            assert abs(U[s11 + s11] - ref["11"]) < 1e-14
            blk = np.array([[U[s10 + s10], U[s10 + s01]], [U[s01 + s10], U[s01 + s01]]])
            assert np.max(np.abs(blk - ref["1p"])) < 1e-14


@pytest.mark.parametrize("d_A", [2, 3])
def test_gate_unitary_and_conserving(d_A):
    b, n, tau, I = model.local_ops(d_A)
    U = model.gate(1.0, 1.0, 5.0, 0.05, d_A)
    d2 = U.shape[0]
    assert np.max(np.abs(U.conj().T @ U - np.eye(d2))) < 1e-14
    N = np.kron(n, I) + np.kron(I, n)
    for Op in (N, np.kron(tau, I), np.kron(I, tau)):
        assert np.max(np.abs(U @ Op - Op @ U)) < 1e-14
    # group property exp(-iH a) exp(-iH b) = exp(-iH (a+b)); identity at zero time
    Ua = model.gate(1.0, 1.0, 5.0, 0.02, d_A)
    Ub = model.gate(1.0, 1.0, 5.0, 0.03, d_A)
    assert np.max(np.abs(Ua @ Ub - U)) < 1e-13
    assert np.max(np.abs(model.gate(1.0, 1.0, 5.0, 0.0, d_A) - np.eye(d2))) < 1e-15


def test_bond_hamiltonian_site_sum():
    """Each of the four bonds touching a site carries h/4 of that site's field term, so that the
    four bonds together give h tau n once per site."""
    b, n, tau, I = model.local_ops(2)
    h = 2.0
    hb = model.bond_hamiltonian(0.0, 0.0, h, 2)
    assert np.allclose(hb, (h / 4) * (np.kron(tau @ n, I) + np.kron(I, tau @ n)))
    # hopping and interaction parts
    hJ = model.bond_hamiltonian(1.0, 0.0, 0.0, 2) - model.bond_hamiltonian(0.0, 0.0, 0.0, 2)
    bd = b.conj().T
    assert np.allclose(hJ, -(np.kron(bd, b) + np.kron(b, bd)))
    hV = model.bond_hamiltonian(0.0, 1.0, 0.0, 2)
    assert np.allclose(hV, np.kron(n, n))


def test_initial_state():
    GA, GB, lam = model.initial_tensors(3, 2)
    b, n, tau, I = model.local_ops(2)
    a = GA[:, 0, 0, 0, 0]
    c = GB[:, 0, 0, 0, 0]
    assert abs(np.vdot(a, n @ a) - 1) < 1e-15 and abs(np.vdot(c, n @ c)) < 1e-15
    assert abs(np.vdot(a, tau @ a)) < 1e-15 and abs(np.vdot(c, tau @ c)) < 1e-15
    assert abs(np.vdot(a, a) - 1) < 1e-15
    assert np.count_nonzero(GA) == 2 and np.count_nonzero(GB) == 2
    assert np.all(lam[:, 0] == 1) and np.all(lam[:, 1:] == 0)
