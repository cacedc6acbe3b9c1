"""Free-fermion ED workload on the device (include/ipeps_ed.h) against the oracle (oracle/ed.py):
spectra, even / odd occupations along the Neel evolution, IPRs and their interval sums.  Spectra
and occupations do not depend on the eigenvector basis and are compared everywhere; the IPR of an
eigenvector is compared where its eigenvalue is separated from its neighbours (a degenerate
eigenspace has no unique basis)."""
import numpy as np
import pytest

from inputs import ED, ed_fields
from oracle import ed

pytestmark = pytest.mark.gpu


def _compare(Lx, Ly, J, f, times, gap_min=1e-6):
    import paper_1910_11359_gb300 as pkg
    g = pkg.ed_run(Lx, Ly, J, f, times)
    o = ed.run(Lx, Ly, J, f, times)
    scale = 4 * abs(J) + np.max(np.abs(f)) + 1.0
    e_spec = np.max(np.abs(g["spectra"] - o["spectra"])) / scale
    e_occ = max(np.max(np.abs(g["n_even"] - o["n_even"])), np.max(np.abs(g["n_odd"] - o["n_odd"])))
    # IPR on separated eigenvalues; cumulative IPR where every state of the realisation is separated
    sep = np.ones_like(o["spectra"], dtype=bool)
    d = np.diff(o["spectra"], axis=1)
    sep[:, 1:] &= d > gap_min * scale
    sep[:, :-1] &= d > gap_min * scale
    e_ipr = np.max(np.abs(g["ipr"] - o["ipr"])[sep]) if sep.any() else 0.0
    e_cum = np.max(np.abs(g["cum_ipr"] - o["cum_ipr"])) if sep.all() else None
    print("ED %dx%d R=%d: spectra %.1e occupations %.1e ipr %.1e cum %s sweeps %s"
          % (Lx, Ly, len(f), e_spec, e_occ, e_ipr, "-" if e_cum is None else "%.1e" % e_cum,
             g["sweeps"].tolist()[:4]))
    return e_spec, e_occ, e_ipr, e_cum, g, o


@pytest.mark.parametrize("Lx,Ly,h,levels", [(4, 4, 4.0, 0), (6, 5, 10.0, 0), (10, 10, 4.0, 0),
                                            (5, 3, 100.0, 0), (8, 7, 10.0, 3), (10, 10, 100.0, 3)])
def test_ed_matches_oracle(Lx, Ly, h, levels):
    """Several tiles of the batched GEMMs and a ragged odd lattice (5 x 3: 8 even, 7 odd sites);
    continuous and three-level disorder; h from 4 to 100."""
    f = ed_fields(max(Lx, Ly), 3, h, levels, seed=11)[:, :Lx * Ly]
    times = [0.0, 0.05, 0.4, 1.0, 2.5, 5.0]
    e_spec, e_occ, e_ipr, e_cum, g, _ = _compare(Lx, Ly, 1.0, f, times)
    assert e_spec < 1e-13
    assert e_occ < 1e-11
    assert e_ipr < 1e-9
    if e_cum is not None:
        assert e_cum < 1e-9
    assert abs(g["n_even"][0] - 1.0) < 1e-14 and abs(g["n_odd"][0]) < 1e-14


def test_ed_edge_cases():
    """A two-site lattice; a clean chain (closed-form spectrum, IPR 3 / (2 (L + 1))); J = 0 (frozen
    occupations, IPR 1); many realisations of a small lattice (several time blocks' worth)."""
    import paper_1910_11359_gb300 as pkg
    g = pkg.ed_run(2, 1, 1.0, np.array([[0.3, -0.2]]), [0.0, 1.0])
    o = ed.run(2, 1, 1.0, np.array([[0.3, -0.2]]), [0.0, 1.0])
    assert np.allclose(g["spectra"], o["spectra"], atol=1e-14) and np.allclose(g["n_odd"], o["n_odd"], atol=1e-14)
    L = 12
    g = pkg.ed_run(L, 1, 1.0, np.zeros((1, L)), [0.0])
    a = np.arange(1, L + 1)
    assert np.allclose(g["spectra"][0], np.sort(-2 * np.cos(np.pi * a / (L + 1))), atol=1e-13)
    assert np.allclose(g["ipr"][0], 1.5 / (L + 1), atol=1e-12)
    f = ed_fields(6, 2, 4.0, 0, seed=5)
    g = pkg.ed_run(6, 6, 0.0, f, [0.0, 2.0, 7.0])
    assert np.allclose(g["ipr"], 1.0, atol=1e-13)
    assert np.allclose(g["n_even"], 1.0, atol=1e-13) and np.allclose(g["n_odd"], 0.0, atol=1e-13)
    f = ed_fields(4, 300, 10.0, 0, seed=6)
    times = np.linspace(0.0, 5.0, 11)
    _, e_occ, _, _, _, _ = _compare(4, 4, 1.0, f, times)
    assert e_occ < 1e-11


def test_ed_full_size_sample():
    """The benchmark lattice (20 x 20, the paper's L = 20; 51 times in [0, 5]) on a sample of 6 of its
    100 realisations, continuous disorder h = 10: every output against the oracle."""
    L = 20
    f = ed_fields(L, ED["R"], 10.0, 0, seed=21)[:6]
    e_spec, e_occ, e_ipr, e_cum, g, _ = _compare(L, L, 1.0, f, list(ED["times"]))
    assert e_spec < 1e-13 and e_occ < 1e-11 and e_ipr < 1e-9
    assert abs(g["n_even"][-1] + g["n_odd"][-1] - 1.0) < 1e-12      # half filling: n_e + n_o = 1
