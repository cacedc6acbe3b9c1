"""More disorder levels (d_A > 2, d = 2 d_A) and the Renyi entropies on the GPU, against the oracle.

The paper's localised regime needs d_A = 3..5 levels per site (field values spaced uniformly in
[-h, h], Sec. "Set up for iPEPS"; d = 6, 8, 10 in the Appendix) and reads out Renyi entropies of the
physical one-site RDM (Sec. "Results for interacting case").  Checked here, through the C ABI:
the simple-update bond spectra and discarded weight (1e-12), CTMRG at a fixed number of sweeps from
the same tensors (one-site observables and Renyi entropies at 1e-10), the entropies against the
closed forms that particle-number conservation fixes from n_A, and a converged d_A = 3 trajectory
against the oracle's (tests/golden/quench_dA3_D3_oracle.json, unique readouts at 1e-10, every
readout checked at the GPU's own environment).
"""
import json
import os

import numpy as np
import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctmrg, evolve, measure, model  # noqa: E402
from tests.test_gpu_parity import GOLDEN, _compare_rows, _evolve_like, _sim  # noqa: E402

TOL = 1e-10


@pytest.mark.parametrize("d_A,D", [(3, 3), (4, 3), (5, 4)])
def test_simple_update_spectra_levels(d_A, D):
    Vs, hs = [1.0, 0.0], [5.0, 2.0]
    sim = _sim(J=[1.0, 1.0], V=Vs, h=hs, D=D, chi=D * D, order=2, dt=0.05, d_A=d_A)
    eps = sim.trotter_step(4)
    lam = sim.get_lambda()
    sim.close()
    for b, (V, h) in enumerate(zip(Vs, hs)):
        p = dict(J=1.0, V=V, h=h, D=D, order=2, dt=0.05, d_A=d_A)
        _, _, lam_ref, eps_ref = evolve.evolve_tensors(p, 4)
        assert np.max(np.abs(lam[b] - lam_ref)) < 1e-12, (d_A, b)
        assert abs(eps[b] - eps_ref) < 1e-12 + 1e-9 * eps_ref


def _one_site(A, B, env, d_A):
    n_op = model.local_ops(d_A)[1]
    rA, rB = measure.rho1(A, env, (0, 0)), measure.rho1(B, env, (1, 0))
    nA, nB = measure.expect1(rA, n_op).real, measure.expect1(rB, n_op).real
    pA = measure.physical_rdm(rA, d_A)
    return dict(nA=nA, nB=nB, imbalance=nA - nB, renyi1A=measure.renyi(pA, 1.0),
                renyi_halfA=measure.renyi(pA, 0.5), renyi2A=measure.renyi(pA, 2.0))


@pytest.mark.parametrize("d_A,D,chi", [(3, 3, 9), (5, 4, 16)])
def test_ctmrg_fixed_sweeps_levels(d_A, D, chi):
    """From the same tensors (the oracle's, after 3 Trotter steps) and the same traced start, 3 CTMRG
    sweeps: one-site observables and entropies agree to 1e-10; the entropies equal the binary
    entropies of n_A (the physical RDM is diag(1 - n_A, n_A) by particle-number conservation)."""
    p = dict(J=1.0, V=1.0, h=5.0, D=D, order=2, dt=0.05, d_A=d_A)
    GA, GB, lam, _ = evolve.evolve_tensors(p, 3)
    sim = _sim(D=D, chi=chi, order=2, dt=0.05, d_A=d_A)
    sim.set_tensors(GA[None], GB[None], lam[None])
    sim.ctmrg_converge(tol=0.0, max_sweeps=3)
    obs = sim.measure()[0]
    sim.close()
    A, B, a = evolve.ctm_state(GA, GB, lam)
    env = ctmrg.init_env(a, 2, 2, chi, D)
    env, _, _ = ctmrg.ctmrg(a, env, chi, tol=0.0, max_sweeps=3)
    ref = _one_site(A, B, env, d_A)
    err = max(abs(obs[k] - ref[k]) for k in ref)
    print("d_A = %d: one-site observables and entropies within %.1e of the oracle" % (d_A, err))
    assert err < TOL
    q = obs["nA"]
    assert abs(obs["renyi1A"] + q * np.log(q) + (1 - q) * np.log(1 - q)) < TOL
    assert abs(obs["renyi_halfA"] - 2 * np.log(np.sqrt(q) + np.sqrt(1 - q))) < TOL
    assert abs(obs["renyi2A"] + np.log(q * q + (1 - q) ** 2)) < TOL
    assert obs["renyi1A"] > 1e-3


def test_zero_hopping_keeps_product_state_levels():
    sim = _sim(J=[0.0], V=[1.0], h=[5.0], D=3, chi=9, order=2, dt=0.05, d_A=4)
    sim.trotter_step(4)
    sim.ctmrg_converge(tol=1e-10, max_sweeps=50)
    o = sim.measure()[0]
    sim.close()
    assert abs(o["imbalance"] - 1.0) < 1e-13
    assert abs(o["renyi1A"]) < 1e-13 and abs(o["renyi_halfA"]) < 1e-13


def test_quench_dA3_matches_golden():
    path = os.path.join(GOLDEN, "quench_dA3_D3_oracle.json")
    g = json.load(open(path))
    keys = ("imbalance", "nA", "nB", "energy", "renyi1A", "renyi_halfA", "renyi2A")
    for cold in (False, True):
        out = _evolve_like(g, cold=cold)
        rows = _compare_rows(out, g, keys, g["params"]["chi"], g["params"]["D"], cold=cold)
        assert sum(1 for r in rows if r[2]) >= 3
