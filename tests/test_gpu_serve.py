"""Serving loop on the device: requests admitted while others run, on two worker streams, give
exactly the readouts of the same requests served alone."""
import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_served_requests_match_requests_served_alone():
    from paper_1910_11359_gb300.serve import LibraryEngine, Request, Server, percentile
    reqs = [Request(rid=i, arrival=0.05 * i, J=1.0, V=float(i % 2), h=2.0 + 3 * i, D=2,
                    chi=4 + 4 * (i % 2), t_max=1.0) for i in range(4)]
    out = Server(LibraryEngine(), budget_bytes=10 ** 10, workers=2).run(reqs)
    assert len(out) == 4
    worst = 0.0
    for r in out:
        assert len(r.readouts) == 3
        alone = Server(LibraryEngine(), budget_bytes=10 ** 10, workers=1).run(
            [Request(rid=0, arrival=0.0, J=r.J, V=r.V, h=r.h, D=r.D, chi=r.chi, t_max=r.t_max)])[0]
        worst = max(worst, max(abs(a[k] - b[k]) for a, b in zip(alone.readouts, r.readouts)
                               for k in ("imbalance", "energy", "purityA")))
    print("served vs alone: max abs difference %.1e, p50 latency %.2f s"
          % (worst, percentile([r.latency for r in out], 50)))
    assert worst < 1e-12
    assert abs(out[0].readouts[-1]["imbalance"] - 1.0) > 1e-2


def test_split_mixed_d_served_match_alone():
    """Split precision with requests of different D and chi in the mix (so different contraction
    shapes share the device and the tile-width tuner): each request's readouts equal those of the
    request served alone."""
    import paper_1910_11359_gb300 as pkg
    from paper_1910_11359_gb300.serve import LibraryEngine, Request, Server
    shapes = [(2, 4), (3, 9), (2, 8), (3, 18)]
    reqs = [Request(rid=i, arrival=0.02 * i, J=1.0, V=0.5 * (i % 3), h=3.0 + 2 * i, D=D, chi=chi, t_max=1.0,
                    precision=pkg.SPLIT_BF16X3) for i, (D, chi) in enumerate(shapes)]
    eng = LibraryEngine(tol=1e-7)
    out = Server(eng, budget_bytes=10 ** 11, workers=3).run(reqs)
    assert len(out) == len(reqs)
    worst = 0.0
    for r in out:
        alone = Server(eng, budget_bytes=10 ** 11, workers=1).run(
            [Request(rid=0, arrival=0.0, J=r.J, V=r.V, h=r.h, D=r.D, chi=r.chi, t_max=r.t_max,
                     precision=r.precision)])[0]
        worst = max(worst, max(abs(a[k] - b[k]) for a, b in zip(alone.readouts, r.readouts)
                               for k in ("imbalance", "energy", "purityA")))
    print("split, mixed D: served vs alone max abs difference %.1e" % worst)
    assert worst < 1e-12
