"""Pins for oracle/ctmrg.py and oracle/measure.py (engine checks use a projector cutoff of 1e-10
so that the truncation bias stays below the closed-form tolerances).

* Ising PEPS (norm network = 2D Ising partition function): one-site <sigma^z> equals Yang's
  spontaneous magnetisation, nearest-neighbour <sigma^z sigma^z> equals Onsager's -u/2 on both
  bond orientations, and the CTM norm per site equals exp(-beta f) from Onsager's integral.
* Dimer states (one bond layer of gates on the CDW): CTMRG observables equal the exact two-site
  values for every bond orientation.
* Small random PEPS: one- and two-site expectation values approach the exact contraction of
  periodic L x L tori, with the gap shrinking from L = 2 to L = 4.
* Product state at chi = 1 is exact; rotating the lattice by 90 degrees maps horizontal bond
  RDMs onto vertical ones.
"""
import numpy as np
import pytest

from inputs import random_site_tensors
from oracle import ctmrg, measure, model, su
from tests.pins import ising, torus

SZ = np.diag([1.0, -1.0]).astype(complex)


def _converge(A, B, chi, D, tol=1e-10, init_from=None, max_sweeps=300, cut_rel=1e-10):
    a = ctmrg.checkerboard(ctmrg.double_layer(A), ctmrg.double_layer(B))
    a0 = a if init_from is None else ctmrg.checkerboard(ctmrg.double_layer(init_from[0]),
                                                         ctmrg.double_layer(init_from[1]))
    env = ctmrg.init_env(a0, 2, 2, chi, D)
    env, n, delta = ctmrg.ctmrg(a, env, chi, tol=tol, max_sweeps=max_sweeps, cut_rel=cut_rel)
    return env, n, delta


@pytest.mark.parametrize("beta", [0.5, 0.35])
def test_ising_onsager_yang(beta):
    A = ising.peps_tensor(beta)
    bias = None
    if beta > ising.BETA_C:                 # seed the + phase through the initial environment
        Ab = A.copy()
        Ab[1] = 0.0
        bias = (Ab, Ab)
    env, n, delta = _converge(A, A, 16, 2, tol=1e-10, init_from=bias)
    m = measure.expect1(measure.rho1(A, env, (0, 0)), SZ).real
    assert abs(m - ising.magnetisation(beta)) < 1e-7
    ref = ising.nn_correlation(beta)
    h = measure.expect2(measure.rho2_h(A, A, env, (0, 0), (1, 0)), np.kron(SZ, SZ)).real
    v = measure.expect2(measure.rho2_v(A, A, env, (0, 0), (0, 1)), np.kron(SZ, SZ)).real
    assert abs(h - ref) < 1e-7 and abs(v - ref) < 1e-7
    kappa = measure.norm_site(A, env, (0, 0)).real
    assert abs(kappa / ising.z_per_site(beta) - 1) < 1e-9


def _dimer_exact(U, leg):
    """Exact observables of the dimer state made by one gate on bond ``leg`` of the CDW."""
    b, n, tau, I = model.local_ops(2)
    pA = np.array([0, 0, 1, 1], dtype=complex) / np.sqrt(2)
    pB = np.array([1, 1, 0, 0], dtype=complex) / np.sqrt(2)
    psi = U @ np.kron(pA, pB)
    rho = np.outer(psi, psi.conj()).reshape(4, 4, 4, 4)     # [sA, sB, sA', sB']
    rA = np.einsum('abcb->ac', rho)
    rB = np.einsum('abad->bd', rho)
    hb = model.bond_hamiltonian(1.0, 1.0, 0.0)
    e_dimer = np.vdot(psi, hb @ psi).real
    e_prod = np.trace(np.kron(rA, rB) @ hb).real                    # <h> in rho_A x rho_B
    return dict(nA=np.trace(rA @ n).real, nB=np.trace(rB @ n).real, e_dimer=e_dimer, e_prod=e_prod)


@pytest.mark.parametrize("leg,h,D", [(0, 0.0, 2), (1, 0.0, 2), (2, 0.0, 2), (3, 0.0, 2), (3, 5.0, 4)])
def test_dimer_states_exact(leg, h, D):
    U = model.gate(1.0, 1.0, h, 0.4)
    GA, GB, lam = model.initial_tensors(D)
    GA, GB, lam, eps = su.bond_update(GA, GB, lam, leg, U)
    assert eps < 1e-28
    A, B = su.physical_tensors(GA, GB, lam)
    env, n, delta = _converge(A, B, D * D, D)
    ex = _dimer_exact(U, leg)
    b, nop, tau, I = model.local_ops(2)
    assert abs(measure.expect1(measure.rho1(A, env, (0, 0)), nop).real - ex['nA']) < 1e-12
    assert abs(measure.expect1(measure.rho1(B, env, (1, 0)), nop).real - ex['nB']) < 1e-12
    hb = model.bond_hamiltonian(1.0, 1.0, 0.0)
    # the four bonds of the unit cell, named by A's leg: R, L (horizontal), D, U (vertical)
    e = {3: measure.expect2(measure.rho2_h(A, B, env, (0, 0), (1, 0)), hb).real,
         1: measure.expect2(measure.rho2_h(B, A, env, (1, 0), (0, 0)), hb).real,
         2: measure.expect2(measure.rho2_v(A, B, env, (0, 0), (0, 1)), hb).real,
         0: measure.expect2(measure.rho2_v(B, A, env, (0, 1), (0, 0)), hb).real}
    for g in range(4):
        want = ex['e_dimer'] if g == leg else ex['e_prod']
        assert abs(e[g] - want) < 1e-12, (g, e[g], want)


def _rand_op(d, seed):
    rng = np.random.default_rng(seed)
    O = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    return O + O.conj().T


def test_random_peps_matches_torus():
    d, D = 2, 2
    A, B = random_site_tensors(d, D, seed=7, noise=0.05)
    env, n, delta = _converge(A, B, 8, D, tol=1e-12)
    O1, O2 = _rand_op(d, 1), _rand_op(d, 2)
    ctm = {
        'A': measure.expect1(measure.rho1(A, env, (0, 0)), O1).real,
        'B': measure.expect1(measure.rho1(B, env, (1, 0)), O1).real,
        'h': measure.expect2(measure.rho2_h(A, B, env, (0, 0), (1, 0)), np.kron(O1, O2)).real,
        'v': measure.expect2(measure.rho2_v(A, B, env, (0, 0), (0, 1)), np.kron(O1, O2)).real,
    }
    for L in (2, 4):
        ex = {
            'A': torus.one_site(A, B, L, O1, (0, 0)).real,
            'B': torus.one_site(A, B, L, O1, (1, 0)).real,
            'h': torus.two_site(A, B, L, O1, O2, (0, 0), (1, 0)).real,
            'v': torus.two_site(A, B, L, O1, O2, (0, 0), (0, 1)).real,
        }
        err = {k: abs(ctm[k] - ex[k]) for k in ctm}
        if L == 2:
            err2 = err
    for k in ctm:
        assert err[k] < 2e-3, (k, err[k])
        assert err[k] < err2[k] / 3, (k, err[k], err2[k])


def test_product_state_chi1_exact():
    GA, GB, lam = model.initial_tensors(1)
    U = model.gate(1.0, 1.0, 5.0, 0.1)
    for leg in (3, 0, 1, 2, 3, 0):
        GA, GB, lam, _ = su.bond_update(GA, GB, lam, leg, U)
    A, B = su.physical_tensors(GA, GB, lam)
    env, n, delta = _converge(A, B, 1, 1)
    b, nop, tau, I = model.local_ops(2)
    a = A[:, 0, 0, 0, 0]
    want = np.vdot(a, nop @ a).real / np.vdot(a, a).real
    assert abs(measure.expect1(measure.rho1(A, env, (0, 0)), nop).real - want) < 1e-14


def test_rotation_maps_horizontal_to_vertical():
    d, D = 2, 2
    A, B = random_site_tensors(d, D, seed=11, noise=0.05)
    rot = (0, 4, 1, 2, 3)                     # new (u, l, d, r) = old (r, u, l, d)
    Ar, Br = A.transpose(rot), B.transpose(rot)
    env, _, _ = _converge(A, B, 8, D, tol=1e-12)
    envr, _, _ = _converge(Ar, Br, 8, D, tol=1e-12)
    rv = measure.rho2_v(A, B, env, (0, 0), (0, 1))
    rh = measure.rho2_h(Ar, Br, envr, (0, 0), (1, 0))
    rv, rh = rv / np.einsum('ssvv->', rv), rh / np.einsum('ssvv->', rh)
    assert np.max(np.abs(rv - rh)) < 1e-9


def test_torus_helper_matches_state_vector():
    """The transfer-matrix torus helper equals a plain state-vector contraction at L = 2, and the
    state vector is invariant under a 90-degree rotation of the lattice."""
    from tests.pins import statevector
    d, D = 2, 2
    A, B = random_site_tensors(d, D, seed=7, noise=0.3)
    O = _rand_op(d, 5)
    T = {(x, y): (A if (x + y) % 2 == 0 else B) for x in range(2) for y in range(2)}
    sv = statevector.one_site(T, 2, O, (0, 0)).real
    assert abs(torus.one_site(A, B, 2, O, (0, 0)).real - sv) < 1e-12
    rot = (0, 4, 1, 2, 3)
    Tr = {p: t.transpose(rot) for p, t in T.items()}
    assert abs(statevector.one_site(Tr, 2, O, (0, 0)).real - sv) < 1e-12


def test_projector_multiplet_rule_and_margin():
    """The chi-cut rule of the projectors (C8): a relative gap below 1e-10 or an absolute gap below
    1e-11 s_1 is one multiplet; values under the cutoff are not examined; cut_margin measures the
    distance of the deciding test from its threshold in decades."""
    from oracle.su import truncation_rank
    abs_floor = ctmrg.PROJ_DEGEN_ABS
    # exact pair at the cut (relative test), well above the floor
    s = np.array([1.0, 0.3, 0.1, 0.1, 0.05])
    assert truncation_rank(s, 3, degen_abs=abs_floor) == 2
    # small pair whose relative gap (1e-6) passes the relative test but whose absolute gap (3e-12)
    # is below the floor: one multiplet only through the absolute test
    s = np.array([1.0, 0.5, 3.000003e-6, 3.0e-6, 1e-7])
    assert truncation_rank(s, 3) == 3
    assert truncation_rank(s, 3, degen_abs=abs_floor) == 2
    # a genuine gap is kept
    s = np.array([1.0, 0.5, 2e-6, 1e-6, 1e-7])
    assert truncation_rank(s, 3, degen_abs=abs_floor) == 3
    # margins: an exact pair is far from both thresholds; the cut then stops at the gap 0.3 / 0.1,
    # whose decision lies log10(0.2 / 1e-11) = 10.3 decades from the absolute threshold
    assert abs(ctmrg.cut_margin(np.array([1.0, 0.3, 0.1, 0.1, 0.05]), 3) - np.log10(0.2 / 1e-11)) < 1e-9
    # a gap of 1e-9 s_1 between values ~1e-3: the relative test is 4 decades from its threshold, the
    # absolute one 2 decades -- the decision (not a multiplet) is 2 decades from flipping
    m = ctmrg.cut_margin(np.array([1.0, 0.5, 1e-3 + 1e-9, 1e-3, 1e-4]), 3)
    assert abs(m - 2.0) < 1e-3
    # below the cutoff nothing is examined
    assert ctmrg.cut_margin(np.array([1.0, 1e-12, 1e-12, 1e-13]), 2, cut_rel=1e-10) == np.inf
