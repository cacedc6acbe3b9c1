"""End-to-end pins for the oracle's time evolution (simple update + CTMRG + measurement).

* J = 0: the CDW is an eigenstate, I(t) = 1 exactly (pin P1).
* Short times: I(t) = 1 - 8 J^2 t^2 + O(t^4) independent of V and h (pin P2; derivation:
  <[H,[H,n_i]]> = 2 z J^2 for the CDW, time-reversal symmetry removes odd orders).
* J -> -J and h -> -h leave I(t) unchanged (pin P3); <tau^z> stays 0 and n_A + n_B stays 1 up to
  the truncation error (pin P5).
* Short-time agreement with exact dynamics of the 8-site tilted cluster averaged over all 2^8
  disorder configurations, with an O(t^4) finite-size gap (pin P9); the same at three disorder
  levels (d_A = 3, all 3^8 configurations), with J = 0 exactness and the 1 - 8 t^2 law there too.
* Cold and warm CTMRG starts give the same observables.
"""
import numpy as np
import pytest

from oracle import ctmrg, evolve, model, su
from tests.pins import ed


def _run(**kw):
    p = dict(J=1.0, V=1.0, h=5.0, D=2, chi=8, order=2, dt=0.01, t_max=0.1, meas_every=0.05)
    p.update(kw)
    return evolve.run(p, tol=1e-11)


def test_zero_hopping_imbalance_is_one():
    out = _run(J=0.0, t_max=0.2, dt=0.02, meas_every=0.1, order=1)
    for o in out:
        assert abs(o['imbalance'] - 1.0) < 1e-13
        assert abs(o['nA'] - 1.0) < 1e-13 and abs(o['nB']) < 1e-13
        assert o['trunc_err_acc'] < 1e-28


@pytest.mark.parametrize("V,h", [(1.0, 5.0), (0.0, 10.0)])
def test_short_time_closed_form(V, h):
    """Least-squares fit I = 1 - a t^2 - b t^4 on t <= 0.04 gives a = 8 J^2 for any V, h."""
    out = _run(V=V, h=h, dt=0.001, t_max=0.04, meas_every=0.01)
    t = np.array([o['t'] for o in out[1:]])
    y = 1 - np.array([o['imbalance'] for o in out[1:]])
    coef, *_ = np.linalg.lstsq(np.stack([t ** 2, t ** 4], 1), y, rcond=None)
    assert abs(coef[0] - 8.0) < 0.02, coef


def test_gauge_and_field_flip_invariance():
    base = _run()
    for kw in (dict(J=-1.0), dict(h=-5.0)):
        other = _run(**kw)
        for o1, o2 in zip(base, other):
            assert abs(o1['imbalance'] - o2['imbalance']) < 1e-11
            assert abs(o1['energy'] - o2['energy']) < 1e-11


def test_conservation_within_truncation():
    out = _run(D=2, chi=8, order=1, dt=0.02, t_max=0.3, meas_every=0.1)
    for o in out:
        bound = 4 * np.sqrt(o['trunc_err_acc']) + 1e-12
        assert abs(o['nA'] + o['nB'] - 1) <= bound
        assert abs(o['tauzA']) <= bound and abs(o['tauzB']) <= bound


def test_tracks_exact_dynamics_of_8_site_cluster():
    times = [0.05, 0.1]
    ex = ed.imbalance(1.0, 1.0, 5.0, times)
    out = _run(D=2, chi=8, order=2, dt=0.01, t_max=0.1, meas_every=0.05)
    diff = [abs(o['imbalance'] - e) for o, e in zip(out[1:], ex)]
    assert diff[0] < 1e-4 and diff[1] < 1.5e-3
    assert 8 < diff[1] / diff[0] < 24          # the gap grows like t^4


def test_cluster_short_time_expansion():
    """The ED pin itself obeys the closed form 1 - 8 t^2 + O(t^4)."""
    t = np.array([0.01, 0.02])
    ex = ed.imbalance(1.0, 1.0, 5.0, t)
    assert np.all(np.abs(ex - (1 - 8 * t * t)) < 60 * t ** 4)


def test_warm_and_cold_start_agree():
    p = dict(J=1.0, V=1.0, h=5.0, D=2, chi=8, order=1, dt=0.02)
    GA, GB, lam, _ = evolve.evolve_tensors(p, 10)
    A, B, a = evolve.ctm_state(GA, GB, lam)
    GA0, GB0, lam0, _ = evolve.evolve_tensors(p, 7)
    _, _, a0 = evolve.ctm_state(GA0, GB0, lam0)
    env_old, _, _ = ctmrg.ctmrg(a0, ctmrg.init_env(a0, 2, 2, 8, 2), 8, tol=1e-12)
    env_cold, _, _ = ctmrg.ctmrg(a, ctmrg.init_env(a, 2, 2, 8, 2), 8, tol=1e-12)
    env_warm, _, _ = ctmrg.ctmrg(a, env_old, 8, tol=1e-12)
    from oracle import measure
    o1 = measure.observables(A, B, env_cold, 1.0, 1.0, 5.0)
    o2 = measure.observables(A, B, env_warm, 1.0, 1.0, 5.0)
    for k in ('nA', 'nB', 'energy', 'purityA'):
        assert abs(o1[k] - o2[k]) < 1e-10, k


def test_convergence_in_chi_and_d():
    """P11, the paper's own criterion (Appendix: results are trusted where D vs D+1 and chi vs 2 chi
    agree).  At D = 2 the readout is converged in chi: chi = 8 and chi = 16 give the same imbalance
    to 3e-7 up to t = 0.5 (observed 2.2e-7).  In D the simple-update truncation dominates: D = 2
    and D = 3 agree to 1e-4 at t = 0.1 (observed 4.1e-5) and drift apart afterwards, as the
    discarded weight of D = 2 (1.7e-2 at t = 0.5 vs 1.1e-4 at D = 3 by t = 0.2) says they should."""
    base = dict(J=1.0, V=1.0, h=5.0, order=2, dt=0.05, meas_every=0.1)
    a = evolve.run(dict(base, D=2, chi=8, t_max=0.5))
    b = evolve.run(dict(base, D=2, chi=16, t_max=0.5))
    assert max(abs(x["imbalance"] - y["imbalance"]) for x, y in zip(a, b)) < 3e-7
    c = evolve.run(dict(base, D=3, chi=9, t_max=0.1))
    assert abs(a[1]["imbalance"] - c[1]["imbalance"]) < 1e-4
    assert c[-1]["trunc_err_acc"] < a[1]["trunc_err_acc"]


def test_three_levels_zero_hopping_and_short_time():
    """d_A = 3 (fields h, 0, -h per site): J = 0 keeps the CDW (I = 1); the short-time law
    I = 1 - 8 J^2 t^2 + O(t^4) holds whatever the levels."""
    out = _run(J=0.0, d_A=3, t_max=0.2, dt=0.02, meas_every=0.1, order=1)
    for o in out:
        assert abs(o['imbalance'] - 1.0) < 1e-13
    out = _run(d_A=3, dt=0.001, t_max=0.04, meas_every=0.01)
    t = np.array([o['t'] for o in out[1:]])
    y = 1 - np.array([o['imbalance'] for o in out[1:]])
    coef, *_ = np.linalg.lstsq(np.stack([t ** 2, t ** 4], 1), y, rcond=None)
    assert abs(coef[0] - 8.0) < 0.02, coef


def test_three_levels_track_exact_dynamics_of_8_site_cluster():
    """d_A = 3 against the 8-site cluster averaged over all 3^8 = 6561 disorder configurations:
    the O(t^4) finite-size gap of the two-level pin (observed 5e-5 at t = 0.05, 7.7e-4 at 0.1)."""
    times = [0.05, 0.1]
    ex = ed.imbalance(1.0, 1.0, 5.0, times, d_A=3)
    out = _run(D=2, chi=8, order=2, dt=0.01, t_max=0.1, meas_every=0.05, d_A=3)
    diff = [abs(o['imbalance'] - e) for o, e in zip(out[1:], ex)]
    assert diff[0] < 1e-4 and diff[1] < 1.5e-3
    assert 8 < diff[1] / diff[0] < 24          # the gap grows like t^4
    t = np.array([0.01, 0.02])
    ex = ed.imbalance(1.0, 1.0, 5.0, t, d_A=3)
    assert np.all(np.abs(ex - (1 - 8 * t * t)) < 60 * t ** 4)
