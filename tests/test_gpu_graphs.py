"""The convergence graph (conditional WHILE nodes over sweeps and subspace rounds) against the host
loop: the same kernels in the same order, so the same environment, sweep counts and readouts, bit for
bit, along quench trajectories (warm starts, frozen instances in a batch, a fixed-sweep call, split
precision)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(prec, graphs, D=3, chi=18, intervals=4, hs=(1.0, 5.0, 10.0)):
    import paper_1910_11359_gb300 as pkg
    n = len(hs)
    sim = pkg.IPEPS([1.0] * n, [1.0] * n, list(hs), D=D, chi=chi, order=2, dt=0.05, precision=prec)
    sim.set_graphs(graphs)
    out = []
    for it in range(intervals):
        sim.trotter_step(5)
        sw, dl, _ = sim.ctmrg_converge(tol=1e-10, max_sweeps=300, allow_noconv=True)
        obs = sim.measure()
        spec = np.array([[sim.corner_spectrum(b, pos, i) for i in range(4) for pos in range(4)]
                         for b in range(n)])
        out.append((list(sw), list(dl), [(o["imbalance"], o["energy"], o["purityA"]) for o in obs], spec))
    # a fixed-sweep call (tol = 0: another graph) from the converged environment
    sw, dl, _ = sim.ctmrg_converge(tol=0.0, max_sweeps=3)
    obs = sim.measure()
    out.append((list(sw), list(dl), [(o["imbalance"], o["energy"], o["purityA"]) for o in obs], None))
    sim.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_equals_host_loop(prec):
    eager = _run(prec, False)
    graph = _run(prec, True)
    for row, ((s0, d0, o0, c0), (s1, d1, o1, c1)) in enumerate(zip(eager, graph)):
        print("row %d sweeps eager %s graph %s" % (row, s0, s1))
        assert s0 == s1
        assert d0 == d1
        assert o0 == o1
        if c0 is not None:
            assert np.array_equal(c0, c1)


def test_graph_reused_and_profile_fallback():
    """The cached graph serves repeated calls; with launch timing on, the host loop runs instead and
    gives the same result."""
    import paper_1910_11359_gb300 as pkg
    res = []
    for prof in (False, True):
        sim = pkg.IPEPS([1.0], [1.0], [5.0], D=2, chi=8, order=2, dt=0.05)
        pkg.profile_enable(prof)
        rows = []
        for it in range(5):
            sim.trotter_step(4)
            sw, dl, _ = sim.ctmrg_converge(tol=1e-10, max_sweeps=200)
            rows.append((list(sw), sim.measure()[0]["imbalance"]))
        pkg.profile_enable(False)
        sim.close()
        res.append(rows)
    assert res[0] == res[1]
