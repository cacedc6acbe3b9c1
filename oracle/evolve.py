"""Time-evolution driver: Trotter steps interleaved with CTMRG convergence and measurement.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Paper: Sec. "Set up for iPEPS" -- initialise |Psi_0> (CDW x |+>), quench with the simple update,
read out local expectation values with CTMRG.  The environment at each measurement time starts from
the previous measurement's converged environment (warm start); the first one starts from the traced
double layer (see ``ctmrg.init_env``).

Parity: pinned end to end by tests/test_oracle_evolve.py.
"""
import numpy as np

from . import ctmrg, measure, model, su


def ctm_state(GA, GB, lam):
    """Double layers of the 2x2 unit cell and the physical tensors (sqrt(lam) on every leg)."""
    A, B = su.physical_tensors(GA, GB, lam)
    a = ctmrg.checkerboard(ctmrg.double_layer(A), ctmrg.double_layer(B))
    return A, B, a


PROBE_NOISE = 1e-6      # stability probe: relative kick of the converged environment
SPLIT_NOISE = 1e-4      # robustness probe at the split-precision path's noise scale
ROUNDING_KICK = 1e-13   # conditioning probe: relative kick of the site tensors
PROBE_SEED = 12345


def converge_and_measure(GA, GB, lam, env, p, tol, max_sweeps, probe_sweeps=0):
    """Converge the environment (warm from ``env``, or from the traced start when it is None) and
    measure.  ``c8_margin`` in the result is the smallest ctmrg.cut_margin() over the 16 projector
    computations of the last sweep: how far (in decades) the multiplet decisions at the chi cut
    were from their thresholds when the readout was taken; ``c8_level`` is the largest s_K / s_1
    the multiplet rule moved out of the kept set there (0 when it moved nothing): a readout that
    depends on keeping or dropping a multiplet of that size is one of several correct ones (C8).
    ``ctm_stop`` says how the CTMRG ended: "tol" (delta < tol), "stall" (delta at its rounding
    floor) or "cap" (max_sweeps reached).

    With ``probe_sweeps`` > 0 the readout is probed for stability: a copy of the converged
    environment is perturbed by a seeded relative 1e-6 and converged again by the same rules
    (at most ``probe_sweeps`` sweeps); ``drift`` is the largest change of the one-site observables
    (occupations, imbalance, purity of rho_A) between the two readouts.  At an attracting fixed
    point the perturbation dies out and drift stays at the convergence level; at a fixed point
    the CTMRG map departs from (an unstable one) or where several attractors lie close together,
    the perturbed run ends elsewhere and drift is large: such a readout is not a unique result of
    the method.  ``drift_split`` repeats the probe with a relative 1e-4 kick (the noise scale of the
    split-precision contractions).  ``sensitivity`` measures how well FP64 arithmetic determines the
    readout: the site tensors are kicked by a relative 1e-13 (the size of rounding differences between
    two correct implementations) and the environment re-converged; where the fixed point is
    ill-conditioned (slow contraction, a small gap at the chi cut) the readout moves by far more than
    1e-13."""
    A, B, a = ctm_state(GA, GB, lam)
    if env is None:
        env = ctmrg.init_env(a, 2, 2, p['chi'], p['D'])
    log = []
    cut_rel = p.get('cut_rel', ctmrg.PROJ_CUT_REL)
    env, sweeps, delta = ctmrg.ctmrg(a, env, p['chi'], tol=tol, max_sweeps=max_sweeps,
                                     cut_rel=cut_rel, log=log)
    obs = measure.observables(A, B, env, p['J'], p['V'], p['h'], p.get('d_A', 2))
    last = log[-16:]
    stop = "tol" if delta < tol else ("cap" if sweeps >= max_sweeps else "stall")
    obs.update(ctm_sweeps=sweeps, ctm_delta=delta, ctm_stop=stop,
               c8_margin=float(min(m for m, _ in last)), c8_level=float(max(v for _, v in last)))
    if probe_sweeps > 0:
        before = _site_obs(A, B, env, p)

        def reconverge(e_start, a_used):
            e2, n2, _ = ctmrg.ctmrg(a_used, e_start, p['chi'], tol=tol, max_sweeps=probe_sweeps, cut_rel=cut_rel)
            return e2, n2

        # stability: the environment kicked by a relative PROBE_NOISE
        e2, n2 = reconverge(_kick_env(env, PROBE_NOISE, PROBE_SEED), a)
        after = _site_obs(A, B, e2, p)
        obs['drift'] = float(max(abs(after[k] - before[k]) for k in before))
        obs['probe_sweeps'] = n2
        # robustness at the split path's noise scale: a relative 1e-4 kick of the environment
        e3, _ = reconverge(_kick_env(env, SPLIT_NOISE, PROBE_SEED + 1), a)
        after = _site_obs(A, B, e3, p)
        obs['drift_split'] = float(max(abs(after[k] - before[k]) for k in before))
        # conditioning: the site tensors kicked by a relative ROUNDING_KICK (the size of rounding
        # differences between two correct implementations), re-converged from the converged
        # environment; the readout moves by ~ROUNDING_KICK directly plus whatever the fixed point's
        # sensitivity adds
        rng = np.random.default_rng(PROBE_SEED + 2)
        Ak, Bk = [X * (1.0 + ROUNDING_KICK * (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)))
                  for X in (A, B)]
        ak = ctmrg.checkerboard(ctmrg.double_layer(Ak), ctmrg.double_layer(Bk))
        e4, _ = reconverge(env.copy(), ak)
        after = _site_obs(Ak, Bk, e4, p)
        obs['sensitivity'] = float(max(abs(after[k] - before[k]) for k in before))
    return env, obs


def _kick_env(env, rel, seed):
    """A copy of the environment with every tensor perturbed by a seeded relative kick."""
    rng = np.random.default_rng(seed)
    e2 = env.copy()
    for group in (e2.C, e2.T):
        for tens in group:
            for key in sorted(tens):
                t = tens[key]
                noise = rng.standard_normal(t.shape) + 1j * rng.standard_normal(t.shape)
                tens[key] = t + rel * np.abs(t).max() * noise
    return e2


def _site_obs(A, B, env, p):
    """The one-site part of the readout (occupations, imbalance, purity of rho_A), cheap enough to
    evaluate after the probe."""
    n = model.local_ops(p.get('d_A', 2))[1]
    rA, rB = measure.rho1(A, env, (0, 0)), measure.rho1(B, env, (1, 0))
    nA, nB = measure.expect1(rA, n).real, measure.expect1(rB, n).real
    purA = (np.einsum('st,ts->', rA, rA) / np.trace(rA) ** 2).real
    return dict(nA=nA, nB=nB, imbalance=nA - nB, purityA=purA)


def run(p, tol=1e-10, max_sweeps=500, callback=None, cold=False, probe_sweeps=0):
    """Evolve with parameters p (J, V, h, D, chi, order, dt, t_max, meas_every[, d_A, cut_rel]).

    Returns a list of observation dicts at t = 0, meas_every, 2 meas_every, ... t_max
    (``probe_sweeps``: see converge_and_measure).  With
    ``cold`` each dict also holds, under 'cold', the readout converged from the traced start of
    that time's tensors instead of the previous environment.  The cold readout depends only on the
    state; the warm one can also depend on the simple update's gauge (the phases of its singular
    vectors), because at some times the truncated CTMRG has several fixed points and the previous
    environment selects one of them.
    """
    d_A = p.get('d_A', 2)
    GA, GB, lam = model.initial_tensors(p['D'], d_A)
    seq = su.trotter_sequence(p['order'], p['dt'])
    gates = {delta: model.gate(p['J'], p['V'], p['h'], delta, d_A) for _, delta in seq}
    n_steps = int(round(p['t_max'] / p['dt']))
    stride = int(round(p['meas_every'] / p['dt']))
    env = None
    eps_acc = 0.0
    out = []
    for step in range(n_steps + 1):
        if step % stride == 0:
            env, obs = converge_and_measure(GA, GB, lam, env, p, tol, max_sweeps, probe_sweeps)
            obs.update(t=step * p['dt'], trunc_err_acc=eps_acc, lam=lam.copy())
            if cold:
                obs['cold'] = converge_and_measure(GA, GB, lam, None, p, tol, max_sweeps,
                                                   probe_sweeps)[1]
            out.append(obs)
            if callback is not None:
                callback(obs)
        if step < n_steps:
            GA, GB, lam, e = su.trotter_step(GA, GB, lam, gates, p['order'], p['dt'])
            eps_acc += e
    return out


def evolve_tensors(p, n_steps):
    """Only the simple-update part: returns (GA, GB, lam, eps_acc) after n_steps Trotter steps."""
    d_A = p.get('d_A', 2)
    GA, GB, lam = model.initial_tensors(p['D'], d_A)
    seq = su.trotter_sequence(p['order'], p['dt'])
    gates = {delta: model.gate(p['J'], p['V'], p['h'], delta, d_A) for _, delta in seq}
    eps = 0.0
    for _ in range(n_steps):
        GA, GB, lam, e = su.trotter_step(GA, GB, lam, gates, p['order'], p['dt'])
        eps += e
    return GA, GB, lam, eps
