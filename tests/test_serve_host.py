"""Host logic of the serving loop with a host-only engine (no device): admission by footprint in
arrival order, the memory budget, continuous admission as memory frees up, and results that do
not depend on the other requests in the mix."""
import threading
import time

import numpy as np
import pytest

from paper_1910_11359_gb300.serve import Request, Server, percentile, poisson_requests


class FakeEngine:
    """Deterministic stand-in: a request's readouts depend only on its own parameters."""

    def __init__(self, unit=0.002):
        self.unit = unit
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0

    def footprint(self, r):
        return 100 * r.D * r.D

    def new_stream(self):
        return None

    def start(self, r, stream):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
        time.sleep(self.unit)
        return {"t": 0.0}, {"t": 0.0, "imbalance": 1.0}

    def interval(self, r, state):
        time.sleep(self.unit * r.D)
        state["t"] += r.meas_every
        t = state["t"]
        return {"t": t, "imbalance": float(np.exp(-t / r.h) * np.cos(r.V * t))}

    def finish(self, r, state):
        with self.lock:
            self.active -= 1


def _requests():
    return poisson_requests(24, rate=200.0, seed=5, d_choices=(2, 3, 4), t_max_choices=(1.0, 2.0),
                            precision=0)


def test_all_requests_served_and_results_independent_of_the_mix():
    eng = FakeEngine()
    out = Server(eng, budget_bytes=100 * 16 * 4, workers=3).run(_requests())
    assert [r.rid for r in out] == list(range(24))
    for r in out:
        assert len(r.readouts) == r.n_intervals + 1
        assert r.admitted >= r.arrival - 1e-9 and r.finished >= r.admitted
        alone = Server(FakeEngine(unit=0.0), budget_bytes=10 ** 9, workers=1).run(
            [Request(rid=0, arrival=0.0, J=r.J, V=r.V, h=r.h, D=r.D, chi=r.chi, t_max=r.t_max)])[0]
        assert alone.readouts == r.readouts


def test_budget_limits_what_runs_at_once():
    eng = FakeEngine()
    budget = 100 * 16 * 2                 # two D = 4 requests, or more smaller ones
    srv = Server(eng, budget_bytes=budget, workers=4)
    srv.run(_requests())
    assert srv.peak_used <= budget
    assert srv.free == budget
    assert eng.max_active >= 2            # requests did overlap


def test_admission_is_in_arrival_order():
    out = Server(FakeEngine(), budget_bytes=100 * 16 * 2, workers=2).run(_requests())
    order = sorted(out, key=lambda r: (r.arrival, r.rid))
    adm = [r.admitted for r in order]
    assert all(a <= b + 1e-9 for a, b in zip(adm, adm[1:]))


def test_request_larger_than_budget_is_refused():
    r = Request(rid=0, arrival=0.0, J=1.0, V=0.0, h=2.0, D=6, chi=36, t_max=1.0)
    with pytest.raises(ValueError):
        Server(FakeEngine(), budget_bytes=100, workers=1).run([r])


def test_engine_errors_reach_the_caller():
    class Broken(FakeEngine):
        def interval(self, r, state):
            raise RuntimeError("device error")
    with pytest.raises(RuntimeError):
        Server(Broken(), budget_bytes=10 ** 9, workers=2).run(_requests()[:3])


def test_percentile_and_request_stream():
    v = list(np.random.default_rng(0).exponential(size=101))
    for q in (50, 99):
        assert abs(percentile(v, q) - np.percentile(v, q)) < 1e-12
    rs = poisson_requests(400, rate=4.0, seed=5)
    gaps = np.diff([0.0] + [r.arrival for r in rs])
    assert abs(np.mean(gaps) - 0.25) < 0.05
    assert all(r.D * r.D <= r.chi <= 3 * r.D * r.D for r in rs)


def test_deadline_returns_finished_and_unfinished():
    """With a deadline the server stops admitting, stops after the current intervals, returns the
    requests finished by then and lists the rest (with the intervals they completed) as
    unfinished; every admitted request's memory is returned."""
    reqs = poisson_requests(40, rate=100.0, seed=7, d_choices=(2, 3, 4), t_max_choices=(1.0, 8.0),
                            precision=0)
    eng = FakeEngine(unit=0.01)
    srv = Server(eng, budget_bytes=10 ** 6, workers=2)
    out = srv.run(reqs, deadline=0.5)
    assert out and srv.unfinished
    assert len(out) + len(srv.unfinished) <= len(reqs)
    assert all(len(r.readouts) == r.n_intervals + 1 for r in out)
    assert all(len(r.readouts) <= r.n_intervals for r in srv.unfinished)
    assert srv.free == srv.budget
    assert eng.active == 0
