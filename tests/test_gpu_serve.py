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
