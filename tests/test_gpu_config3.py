"""The standalone CTMRG contraction workload (random iPEPS tensors, chi = 2 D^2) against the
oracle's CTMRG with full SVD projectors, at a fixed number of sweeps from the same traced start.

These sizes reach the code paths the smaller workloads never touch: subspace blocks of N = 512 and
1250 rows with k = chi + 8 = 40 and 58 columns (Cholesky-QR orthonormalisation, k x k Jacobi),
split workspaces of the tcgen05 GEMM, and tall Jacobi fall-backs.  FP64 path: normalised corner
spectra and one-site observables within 1e-10.  Split path (BF16x3 contractions, FP64 projectors):
one-site observables within 1e-4 (its bar), leading corner-spectrum values within 5e-2.  Corner
spectra after a few unconverged sweeps amplify rounding: the FP64 path holds them to 1e-10 or to ten
times the oracle's own spread under a rounding-level kick of its inputs, whichever is larger.
"""
import functools

import numpy as np
import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import random_ctmrg_tensors  # noqa: E402
from oracle import ctmrg, measure, model  # noqa: E402

TOL = 1e-10


def _one_site(A, B, env):
    n_op = model.local_ops(2)[1]
    rA, rB = measure.rho1(A, env, (0, 0)), measure.rho1(B, env, (1, 0))
    nA, nB = measure.expect1(rA, n_op).real, measure.expect1(rB, n_op).real
    pur = (np.einsum('st,ts->', rA, rA) / np.trace(rA) ** 2).real
    return dict(nA=nA, nB=nB, imbalance=nA - nB, purityA=pur)


@functools.lru_cache(maxsize=None)
def _oracle(D, sweeps, kick=0.0):
    """The oracle's readout and corner spectra; kick > 0 perturbs the site tensors by a seeded
    relative kick first (the size of rounding differences between two correct implementations)."""
    A, B = random_ctmrg_tensors(D)
    if kick > 0:
        rng = np.random.default_rng(3)
        A, B = [X * (1.0 + kick * (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape))) for X in (A, B)]
    chi = 2 * D * D
    a = ctmrg.checkerboard(ctmrg.double_layer(A), ctmrg.double_layer(B))
    env = ctmrg.init_env(a, 2, 2, chi, D)
    env, _, _ = ctmrg.ctmrg(a, env, chi, tol=0.0, max_sweeps=sweeps)
    return _one_site(A, B, env), ctmrg.corner_spectra(env, chi)


def _oracle_spread(D, sweeps):
    """How far the oracle's own corner spectra move when the inputs are kicked at the rounding
    level (1e-13 relative): unconverged CTMRG sweeps amplify rounding, so spectra are determined by
    FP64 arithmetic only to about this level."""
    _, cs = _oracle(D, sweeps)
    _, ck = _oracle(D, sweeps, kick=1e-13)
    return max(np.max(np.abs(cs[key] - ck[key])) for key in cs)


def _gpu(D, sweeps, precision):
    import paper_1910_11359_gb300 as pkg
    A, B = random_ctmrg_tensors(D)
    chi = 2 * D * D
    sim = pkg.IPEPS([1.0], [1.0], [5.0], D=D, chi=chi, order=2, dt=0.05, precision=precision)
    sim.set_tensors(A[None], B[None], None)
    sim.ctmrg_converge(tol=0.0, max_sweeps=sweeps)
    obs = sim.measure()[0]
    spec = {(i, (pos % 2, pos // 2)): sim.corner_spectrum(0, pos, i) for i in range(4) for pos in range(4)}
    sim.close()
    return obs, spec


@pytest.mark.parametrize("D,sweeps", [(4, 3), (5, 2)])
def test_random_ctmrg_fp64_matches_oracle(D, sweeps):
    ref, cs = _oracle(D, sweeps)
    obs, spec = _gpu(D, sweeps, 0)
    err_o = max(abs(obs[k] - ref[k]) for k in ref)
    err_s = max(np.max(np.abs(s - cs[key])) for key, s in spec.items())
    spread = _oracle_spread(D, sweeps)
    print("D = %d FP64: observables %.1e, corner spectra %.1e (the oracle's own spread under a "
          "rounding-level kick: %.1e)" % (D, err_o, err_s, spread))
    assert err_o < TOL
    assert err_s < max(TOL, 10 * spread)


@pytest.mark.parametrize("D,sweeps", [(4, 3), (5, 2)])
def test_random_ctmrg_split_matches_oracle(D, sweeps):
    ref, cs = _oracle(D, sweeps)
    obs, spec = _gpu(D, sweeps, 1)
    err_o = max(abs(obs[k] - ref[k]) for k in ref)
    lead = max(np.max(np.abs(s - cs[key])[cs[key] > 1e-2]) for key, s in spec.items())
    print("D = %d split: observables %.1e, leading corner spectra %.1e" % (D, err_o, lead))
    assert err_o < 1e-4 and lead < 5e-2
    assert err_o > 1e-13                  # the contractions really ran in reduced precision
