"""Pins for oracle/su.py (simple update, Trotter sequences).

* D = 1: the simple update reduces to propagating a product state; an independent product-state
  script (kron, gate, rank-1 SVD) must give the same local densities.
* One bond update from the CDW at D = 4 is exact: the new bond weights are the Schmidt values of
  the exact two-site state and nothing is discarded, for every bond orientation.
* J = 0: the CDW is an eigenstate; every bond spectrum stays (1, 0, ...).
* J -> -J (sublattice gauge) and h -> -h (auxiliary flip) leave every bond spectrum unchanged.
"""
import numpy as np
import pytest

from oracle import model, su


def _product_state_reference(J, V, h, dt, order, n_steps):
    """Independent D = 1 propagation: psi_A, psi_B d-vectors; per bond theta = U (psi_A x psi_B)
    reshaped d x d, keep the top singular pair.  Returns n_A, n_B per step."""
    b, n, tau, I = model.local_ops(2)
    pA = np.array([0, 0, 1, 1], dtype=complex) / np.sqrt(2)
    pB = np.array([1, 1, 0, 0], dtype=complex) / np.sqrt(2)
    if order == 1:
        deltas = [dt] * 4
    else:
        deltas = [dt / 2] * 3 + [dt] + [dt / 2] * 3
    gates = {x: model.gate(J, V, h, x) for x in set(deltas)}
    out = []
    for _ in range(n_steps):
        for x in deltas:
            th = (gates[x] @ np.kron(pA, pB)).reshape(4, 4)
            u, s, vh = np.linalg.svd(th)
            pA, pB = u[:, 0], vh[0]
        out.append((np.vdot(pA, n @ pA).real / np.vdot(pA, pA).real,
                    np.vdot(pB, n @ pB).real / np.vdot(pB, pB).real))
    return out


@pytest.mark.parametrize("order", [1, 2])
def test_d1_equals_product_state_propagation(order):
    J, V, h, dt = 1.0, 1.0, 5.0, 0.05
    ref = _product_state_reference(J, V, h, dt, order, 12)
    GA, GB, lam = model.initial_tensors(1)
    seq = su.trotter_sequence(order, dt)
    gates = {x: model.gate(J, V, h, x) for _, x in seq}
    b, n, tau, I = model.local_ops(2)
    for step in range(12):
        GA, GB, lam, _ = su.trotter_step(GA, GB, lam, gates, order, dt)
        A, B = su.physical_tensors(GA, GB, lam)
        a, c = A[:, 0, 0, 0, 0], B[:, 0, 0, 0, 0]
        nA = np.vdot(a, n @ a).real / np.vdot(a, a).real
        nB = np.vdot(c, n @ c).real / np.vdot(c, c).real
        assert abs(nA - ref[step][0]) < 1e-13
        assert abs(nB - ref[step][1]) < 1e-13


@pytest.mark.parametrize("leg", [0, 1, 2, 3])
def test_single_gate_from_cdw_is_exact_dimer(leg):
    J, V, h, delta = 1.0, 1.0, 5.0, 0.3
    U = model.gate(J, V, h, delta)
    GA, GB, lam = model.initial_tensors(4)
    GA2, GB2, lam2, eps = su.bond_update(GA, GB, lam, leg, U)
    psi = (U @ np.kron(GA[:, 0, 0, 0, 0], GB[:, 0, 0, 0, 0])).reshape(4, 4)
    sv = np.linalg.svd(psi, compute_uv=False)
    ref = np.zeros(4)
    ref[:len(sv)] = sv / np.linalg.norm(sv)
    assert eps < 1e-28
    assert np.max(np.abs(lam2[leg] - ref)) < 1e-14
    for g in range(4):
        if g != leg:
            assert np.array_equal(lam2[g], lam[g])


def test_zero_hopping_keeps_product_state():
    p = dict(J=0.0, V=1.0, h=5.0)
    for order in (1, 2):
        GA, GB, lam = model.initial_tensors(3)
        seq = su.trotter_sequence(order, 0.05)
        gates = {x: model.gate(p['J'], p['V'], p['h'], x) for _, x in seq}
        for _ in range(10):
            GA, GB, lam, eps = su.trotter_step(GA, GB, lam, gates, order, 0.05)
            assert eps < 1e-28
            assert np.allclose(lam[:, 0], 1.0, atol=1e-15) and np.max(np.abs(lam[:, 1:])) < 1e-15


def _evolve_lam(J, V, h, D=3, order=2, dt=0.05, steps=8):
    GA, GB, lam = model.initial_tensors(D)
    seq = su.trotter_sequence(order, dt)
    gates = {x: model.gate(J, V, h, x) for _, x in seq}
    for _ in range(steps):
        GA, GB, lam, _ = su.trotter_step(GA, GB, lam, gates, order, dt)
    return lam


def test_gauge_and_field_flip_symmetry():
    base = _evolve_lam(1.0, 1.0, 5.0)
    assert np.max(np.abs(_evolve_lam(-1.0, 1.0, 5.0) - base)) < 1e-12
    assert np.max(np.abs(_evolve_lam(1.0, 1.0, -5.0) - base)) < 1e-12


def test_trotter_sequences():
    assert su.trotter_sequence(1, 0.1) == [(3, 0.1), (0, 0.1), (1, 0.1), (2, 0.1)]
    s2 = su.trotter_sequence(2, 0.1)
    assert [g for g, _ in s2] == [3, 0, 1, 2, 1, 0, 3]
    assert abs(sum(x for g, x in s2 if g == 3) - 0.1) < 1e-15
    assert all(abs(sum(x for g2, x in s2 if g2 == g) - 0.1) < 1e-15 for g in range(4))


def test_truncation_rank_multiplets():
    s = np.array([1.0, 0.5, 0.5, 0.5, 0.1])
    assert su.truncation_rank(s, 2) == 1          # split triplet -> cut moves down
    assert su.truncation_rank(s, 4) == 4
    assert su.truncation_rank(np.array([1.0, 0.0, 0.0]), 2) == 2   # zeros are not a multiplet
    assert su.truncation_rank(np.array([1.0, 0.3, 0.2]), 2) == 2
