"""Workload parameters and seeded random tensors (NumPy PCG64 generators).

Workloads (shapes and parameters of the paper's runs, restated for the hard-core boson form):

* QUENCH_D2 -- d = 4 (boson x aux spin-1/2), D = 2, chi = 8, J = V = 1, h = 5, first-order Trotter,
  dt = 0.02 to t = 1, CTMRG to 1e-10, measured every 0.1.
* QUENCH_D3 -- D = 3, chi = 18, J = V = 1, h in {1, 5, 10}, second-order Trotter, dt = 0.05 to t = 5,
  measured every 0.25.
* RANDOM_CTMRG -- standalone CTMRG contraction on random iPEPS tensors (4, D, D, D, D) with i.i.d.
  N(0,1) + i N(0,1) entries scaled to unit largest singular value of the 4 x D^4 matricisation;
  D in {4, 5, 6}, chi = 2 D^2, 20 sweeps.  A uses seed 0, B seed 1.
* DISORDER_SWEEP -- batched disorder sweep of 64 instances of mixed D (disorder_sweep_points).
* QUENCH_DA3 -- d_A = 3 disorder levels (d = 6), D = 3, chi = 9, J = V = 1, h = 5, second-order
  Trotter, dt = 0.05 to t = 0.5, measured every 0.1.
"""
import numpy as np

QUENCH_D2 = dict(J=1.0, V=1.0, h=5.0, D=2, chi=8, order=1, dt=0.02, t_max=1.0, meas_every=0.1,
               tol=1e-10)
QUENCH_D3 = dict(J=1.0, V=1.0, hs=(1.0, 5.0, 10.0), D=3, chi=18, order=2, dt=0.05, t_max=5.0,
               meas_every=0.25, tol=1e-10)
RANDOM_CTMRG = dict(Ds=(4, 5, 6), sweeps=20, seeds=(0, 1))
# three disorder levels (field values h, 0, -h per site, d = 6), the paper's next step up in d_A
QUENCH_DA3 = dict(J=1.0, V=1.0, h=5.0, D=3, chi=9, order=2, dt=0.05, t_max=0.5, meas_every=0.1,
                  tol=1e-10, d_A=3)


def disorder_sweep_points(n=64, seed=4):
    """Batched disorder sweep: n independent instances, h = linspace(0.5, 16, n), V drawn from
    {0, 1} and D from {2, 3, 4} (default_rng(seed)), chi = 2 D^2, J = 1; second-order Trotter,
    dt = 0.05 to t = 4, measured every 0.5."""
    rng = np.random.default_rng(seed)
    hs = np.linspace(0.5, 16.0, n)
    Vs = rng.choice([0.0, 1.0], size=n)
    Ds = rng.choice([2, 3, 4], size=n)
    return [dict(J=1.0, V=float(V), h=float(h), D=int(D), chi=2 * int(D) ** 2)
            for h, V, D in zip(hs, Vs, Ds)]


DISORDER_SWEEP = dict(n=64, order=2, dt=0.05, t_max=4.0, meas_every=0.5, tol=1e-10)


def gaussian_complex(shape, seed):
    """i.i.d. N(0,1) + i N(0,1) entries from numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_ctmrg_tensors(D, d=4, seeds=(0, 1)):
    """Random site tensors A, B of shape (d, D, D, D, D), each with unit largest singular value
    of its d x D^4 matricisation."""
    out = []
    for seed in seeds:
        t = gaussian_complex((d, D, D, D, D), seed)
        t = t / np.linalg.norm(t.reshape(d, -1), 2)
        out.append(t.astype(np.complex128))
    return out[0], out[1]


def random_site_tensors(d, D, seed, product_weight=1.0, noise=0.3):
    """Short-correlated random site tensors: a product-state part on bond index 0 plus seeded noise.

    Returns A, B of shape (d, D, D, D, D).  Used to build small test networks whose correlation
    length is short enough for finite tori to approach the infinite lattice quickly."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        t = noise * (rng.standard_normal((d, D, D, D, D)) + 1j * rng.standard_normal((d, D, D, D, D)))
        v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        t[:, 0, 0, 0, 0] += product_weight * v / np.linalg.norm(v)
        out.append(t)
    return out[0], out[1]


# Free-fermion exact-diagonalisation workload (paper Sec. "Set up for non-interacting fermions";
# Fig. 2-4): L x L lattices, 100 disorder realisations, h in {4, 10, 100}, continuous disorder or a
# three-level (spin-1) discrete one, Neel start, particle numbers on even / odd sites for t in
# [0, 5] (a few tunnelling times), inverse participation ratios binned over the rescaled spectrum.
ED = dict(Ls=(10, 20, 40), R=100, hs=(4.0, 10.0, 100.0), levels=3, J=1.0,
          times=tuple(0.1 * k for k in range(51)), bin_width=0.05)


def ed_fields(L, R, h, levels, seed):
    """On-site fields [R][L*L] of R disorder realisations (numpy default_rng(seed)): continuous
    (levels = 0) uniform in [-h, h]; discrete, `levels` values -h + 2 h k / (levels - 1) drawn with
    equal probability."""
    rng = np.random.default_rng(seed)
    if levels == 0:
        return rng.uniform(-h, h, size=(R, L * L))
    k = rng.integers(0, levels, size=(R, L * L))
    return -h + 2.0 * h * k / (levels - 1)
