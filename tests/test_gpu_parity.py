"""GPU parity of the FP64 path against the oracle, through the C ABI, on gauge-invariant outputs.

Tolerance: 1e-10 absolute on observables and normalised spectra at a fixed number of sweeps (FP64
path); trajectories converged to a 1e-10 corner-spectrum change are compared at 1e-9.  Fixed-sweep CTMRG
comparisons start both sides from the same tensors and the same traced initial environment, so any
difference is rounding plus the SVD gauge; full evolutions converge both sides to the same tol.
"""
import json
import os

import numpy as np
import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctmrg, evolve, measure, model, su  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 1e-10


def _sim(**kw):
    import paper_1910_11359_gb300 as pkg
    p = dict(J=[1.0], V=[1.0], h=[5.0], D=2, chi=8, order=1, dt=0.02, cut_rel=0.0)
    p.update(kw)
    return pkg.IPEPS(p['J'], p['V'], p['h'], D=p['D'], chi=p['chi'], order=p['order'], dt=p['dt'],
                     cut_rel=p['cut_rel'])


@pytest.mark.parametrize("D,order", [(2, 1), (2, 2), (3, 2)])
def test_simple_update_spectra(D, order):
    hs = [1.0, 5.0, 10.0]
    sim = _sim(J=[1.0] * 3, V=[1.0] * 3, h=hs, D=D, chi=D * D, order=order, dt=0.05)
    eps = sim.trotter_step(8)
    lam = sim.get_lambda()
    sim.close()
    for b, h in enumerate(hs):
        p = dict(J=1.0, V=1.0, h=h, D=D, order=order, dt=0.05)
        GA, GB, lam_ref, eps_ref = evolve.evolve_tensors(p, 8)
        assert np.max(np.abs(lam[b] - lam_ref)) < 1e-12
        assert abs(eps[b] - eps_ref) < 1e-12 + 1e-9 * eps_ref


def test_ctmrg_fixed_sweeps_match_oracle():
    p = dict(J=1.0, V=1.0, h=5.0, D=2, order=1, dt=0.02)
    GA, GB, lam, _ = evolve.evolve_tensors(p, 10)
    chi = 8
    sim = _sim(chi=chi)
    sim.set_tensors(GA[None], GB[None], lam[None])
    sim.ctmrg_converge(tol=0.0, max_sweeps=3)
    obs = sim.measure()[0]
    spec = {(i, pos): sim.corner_spectrum(0, pos, i) for i in range(4) for pos in range(4)}
    sim.close()
    A, B, a = evolve.ctm_state(GA, GB, lam)
    env = ctmrg.init_env(a, 2, 2, chi, 2)
    env, n, _ = ctmrg.ctmrg(a, env, chi, tol=0.0, max_sweeps=3)
    assert n == 3
    ref = measure.observables(A, B, env, 1.0, 1.0, 5.0)
    cs = ctmrg.corner_spectra(env, chi)
    for (i, pos), s in spec.items():
        x, y = pos % 2, pos // 2
        assert np.max(np.abs(s - cs[(i, (x, y))])) < TOL, (i, pos)
    for k in ("nA", "nB", "imbalance", "tauzA", "tauzB", "energy", "purityA"):
        assert abs(obs[k] - ref[k]) < TOL, (k, obs[k], ref[k])


def _evolve_like(g, cut_rel=0.0, cold=False, n_rows=None):
    """Run the golden file's workload on the GPU; with ``cold`` every readout starts from the traced
    environment of that time's tensors (ctmrg_reset), otherwise from the previous readout's."""
    p = g["params"]
    sim = _sim(J=[p["J"]], V=[p["V"]], h=[p["h"]], D=p["D"], chi=p["chi"], order=p["order"],
               dt=p["dt"], cut_rel=cut_rel)
    stride = int(round(p["meas_every"] / p["dt"]))
    out = []
    for i, row in enumerate(g["rows"][:n_rows]):
        if i > 0:
            sim.trotter_step(stride)
        if cold:
            sim.ctmrg_reset()
        sim.ctmrg_converge(tol=p["tol"], max_sweeps=500, allow_noconv=True)
        out.append(sim.measure()[0])
    lam = sim.get_lambda()[0]
    sim.close()
    return out, lam


# Tolerance per measured time, from how fast the oracle's own CTMRG converged there: the CTMRG map
# contracts fast where the fixed point is well conditioned; where it needs many sweeps the fixed
# point depends on rounding.  Both trajectories are only converged to a corner-spectrum change below
# 1e-10, so even the best rows are held to 1e-9.
def _row_tol(sweeps):
    if sweeps <= 10:
        return 1e-9
    if sweeps <= 20:
        return 1e-7
    return 1e-3


def _compare_rows(out, lam, g, keys, cold=False):
    """Observables per row.  Cold-start readouts depend only on the state and are held to _row_tol
    of the oracle's cold sweeps.  A warm-started readout is unique only where the oracle's warm and
    cold readouts agree (at some times the truncated CTMRG has several fixed points and the
    previous environment, whose gauge follows the simple update's singular-vector phases, selects
    one).  Rows whose multiplet decisions at the chi cut sat within two decades of the rule's
    thresholds (c8_margin < 2), that dropped a multiplet above 1e-7 of the largest value there
    (c8_level), or whose readout drifts by more than 1e-9 when the oracle keeps sweeping (drift),
    are not unique either.  Unique rows are held to _row_tol, the others
    to 1e-3.  The simple-update state
    (discarded weight; bond spectra of the last row run) at 1e-10 relative / absolute."""
    errs = []
    for o, row in zip(out, g["rows"]):
        assert abs(o["trunc_err_acc"] - row["trunc_err_acc"]) < 1e-12 + 1e-8 * row["trunc_err_acc"]
        ref = row["cold"] if cold else row
        e = max(abs(o[k] - ref[k]) for k in keys)
        unique = cold or max(abs(row[k] - row["cold"][k]) for k in keys) < 1e-9
        # C8: a multiplet decision at the chi cut within two decades of its threshold can go
        # either way under rounding, and each way leads to a valid (different) readout
        unique = unique and ref.get("c8_margin", 99.0) >= 2.0
        # a readout that depends on dropping a multiplet above 1e-7 s_1 at the cut (C8)
        unique = unique and ref.get("c8_level", 0.0) <= 1e-7
        # a readout that moves when the oracle keeps sweeping (a degenerate pair at the cut splitting
        # from rounding noise) is likewise not unique
        unique = unique and ref.get("drift", 0.0) < 1e-9
        tol = _row_tol(ref["ctm_sweeps"]) if unique else 1e-3
        errs.append((row["t"], int(ref["ctm_sweeps"]), unique, e))
        assert e < tol, (row["t"], ref["ctm_sweeps"], unique, e)
    assert np.max(np.abs(lam - np.array(g["rows"][len(out) - 1]["lam"]))) < TOL
    print("%s per-time (t, oracle sweeps, unique, max abs error):" % ("cold" if cold else "warm"),
          ", ".join("(%.2f, %d, %s, %.1e)" % (t, sw, "u" if u else "-", e) for t, sw, u, e in errs))
    return errs


@pytest.mark.parametrize("cold", [False, True])
def test_quench_d2_evolution_matches_golden(cold):
    """D = 2 quench workload with the default projector cutoff (1e-10), warm and cold readouts."""
    g = json.load(open(os.path.join(GOLDEN, "quench_d2_oracle.json")))
    out, lam = _evolve_like(g, cold=cold)
    errs = _compare_rows(out, lam, g, ("imbalance", "nA", "nB", "tauzA", "tauzB", "energy", "purityA"),
                         cold=cold)
    assert sum(1 for t, sw, u, e in errs if u and sw <= 10 and e < 1e-9) >= 7


@pytest.mark.parametrize("cold", [False, True])
def test_quench_d2_cutoff_1e6_matches_golden(cold):
    """Projector cutoff 1e-6, warm and cold readouts."""
    g = json.load(open(os.path.join(GOLDEN, "quench_d2_cut1e-6_oracle.json")))
    out, lam = _evolve_like(g, cut_rel=1e-6, cold=cold)
    errs = _compare_rows(out, lam, g, ("imbalance", "nA", "nB", "tauzA", "tauzB", "energy", "purityA"),
                         cold=cold)
    assert sum(1 for t, sw, u, e in errs if u and sw <= 10 and e < 1e-9) >= 8


def test_ctmrg_subspace_projectors_fixed_sweeps():
    """D = 3, chi = 18 (N = 162 > 2 (chi + 8)): projectors from the warm-started top-k subspace
    iteration against the oracle's full SVD, same start, same number of sweeps."""
    p = dict(J=1.0, V=1.0, h=5.0, D=3, order=2, dt=0.05)
    GA, GB, lam, _ = evolve.evolve_tensors(p, 6)
    chi = 18
    sim = _sim(D=3, chi=chi, order=2, dt=0.05)
    sim.set_tensors(GA[None], GB[None], lam[None])
    sim.ctmrg_converge(tol=0.0, max_sweeps=6)
    obs = sim.measure()[0]
    spec = {(i, pos): sim.corner_spectrum(0, pos, i) for i in range(4) for pos in range(4)}
    sim.close()
    A, B, a = evolve.ctm_state(GA, GB, lam)
    env = ctmrg.init_env(a, 2, 2, chi, 3)
    env, n, _ = ctmrg.ctmrg(a, env, chi, tol=0.0, max_sweeps=6)
    ref = measure.observables(A, B, env, 1.0, 1.0, 5.0)
    cs = ctmrg.corner_spectra(env, chi)
    err_s = max(np.max(np.abs(s - cs[(i, (pos % 2, pos // 2))])) for (i, pos), s in spec.items())
    err_o = max(abs(obs[k] - ref[k]) for k in ("nA", "nB", "imbalance", "energy", "purityA"))
    print("subspace projectors: spectra %.1e observables %.1e" % (err_s, err_o))
    assert err_s < TOL and err_o < TOL


_QUENCH_D3_HS = (1.0, 5.0, 10.0)
_QUENCH_D3_ROWS = 9          # t = 0 .. 2.0 of the t = 5 golden trajectories


@pytest.fixture(scope="module")
def quench_d3_run():
    """D = 3 quench workload (chi = 18, second order, h = 1, 5, 10) to t = 2: the three instances
    run as one batch on the device, once with warm-started and once with cold readouts; each test
    below compares one instance with its oracle trajectory."""
    paths = [os.path.join(GOLDEN, "quench_d3_h%d_oracle.json" % int(h)) for h in _QUENCH_D3_HS]
    if not all(os.path.exists(q) for q in paths):
        pytest.skip("D = 3 golden trajectories not generated")
    gs = [json.load(open(q)) for q in paths]
    if not all("cold" in g["rows"][0] for g in gs):
        pytest.skip("D = 3 golden trajectories lack cold readouts")
    p = gs[0]["params"]
    stride = int(round(p["meas_every"] / p["dt"]))
    res = {}
    for cold in (False, True):
        sim = _sim(J=[1.0] * 3, V=[1.0] * 3, h=list(_QUENCH_D3_HS), D=p["D"], chi=p["chi"],
                   order=p["order"], dt=p["dt"])
        outs = []
        for i in range(_QUENCH_D3_ROWS):
            if i > 0:
                sim.trotter_step(stride)
            if cold:
                sim.ctmrg_reset()
            sim.ctmrg_converge(tol=p["tol"], max_sweeps=500, allow_noconv=True)
            outs.append(sim.measure())
        res[cold] = (outs, sim.get_lambda())
        sim.close()
    return gs, res


@pytest.mark.parametrize("cold", [False, True])
@pytest.mark.parametrize("hi", [0, 1, 2])
def test_quench_d3_evolution_matches_golden(quench_d3_run, hi, cold):
    gs, res = quench_d3_run
    outs, lam = res[cold]
    _compare_rows([o[hi] for o in outs], lam[hi], gs[hi], ("imbalance", "nA", "nB", "energy"), cold=cold)
