"""Serving loop for quench requests: admission by device-memory footprint, overlapping work.

Each request asks for one quench (J, V, h, D, chi, t_max; second-order Trotter steps of dt,
readouts every meas_every).  The server keeps every admitted request's tensors and CTM
environment resident in its own library handle, and runs the requests on a pool of worker
threads, each with its own CUDA stream, so that the work of different requests overlaps on the
device.  A request is admitted, in arrival order, once its footprint (ipeps_footprint_bytes)
fits in the memory still free under the server's budget; its memory is returned when it
finishes.  Requests that arrive while others run are admitted as memory frees up (continuous
admission); a worker interleaves its requests readout interval by readout interval, so a long
request does not hold back short ones queued on the same worker.

The engine is pluggable: LibraryEngine drives libipeps; the tests use a host-only engine.
Every request's results are those of the same request run alone: each has its own handle.

A run may be given a deadline (seconds after the start): admission stops there, the workers stop
after the readout interval they are in, and requests not finished by then are returned in
`unfinished` with the intervals they completed (a bounded window over a stream whose requests
would take hours, e.g. D = 6 at chi = 108).  A worker still inside a long library call at the
deadline is given `grace` seconds; after that run() returns without it (its request is listed as
unfinished) and the caller should end the process rather than wait for it.
"""
import threading
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    arrival: float                      # seconds after the server starts
    J: float
    V: float
    h: float
    D: int
    chi: int
    t_max: float
    dt: float = 0.05
    meas_every: float = 0.5
    precision: int = 0
    # filled in by the server
    admitted: float = None
    finished: float = None
    readouts: list = field(default_factory=list)

    @property
    def n_intervals(self):
        return int(round(self.t_max / self.meas_every))

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class LibraryEngine:
    """One libipeps handle per request, on the calling worker's stream."""

    def __init__(self, tol=1e-10, max_sweeps=500):
        self.tol, self.max_sweeps = tol, max_sweeps

    def footprint(self, r):
        from ._lib import footprint_bytes
        return footprint_bytes([r.J], [r.V], [r.h], D=r.D, chi=r.chi, order=2, dt=r.dt,
                               precision=r.precision)

    def new_stream(self):
        import torch
        return torch.cuda.Stream()

    def start(self, r, stream):
        from ._lib import IPEPS
        sim = IPEPS([r.J], [r.V], [r.h], D=r.D, chi=r.chi, order=2, dt=r.dt, precision=r.precision,
                    stream=stream.cuda_stream if stream is not None else None)
        sim.ctmrg_converge(tol=self.tol, max_sweeps=self.max_sweeps, allow_noconv=True)
        return sim, sim.measure()[0]

    def interval(self, r, sim):
        sim.trotter_step(int(round(r.meas_every / r.dt)), sync=False)
        sim.ctmrg_converge(tol=self.tol, max_sweeps=self.max_sweeps, allow_noconv=True)
        return sim.measure()[0]

    def finish(self, r, sim):
        sim.close()


class Server:
    """Admit requests by footprint under `budget_bytes` and run them on `workers` threads."""

    def __init__(self, engine, budget_bytes, workers=4):
        self.engine, self.budget, self.nworkers = engine, budget_bytes, workers
        self.lock = threading.Condition()
        self.free = budget_bytes
        self.peak_used = 0
        self.queues = [[] for _ in range(workers)]       # per worker: active (request, state)
        self.done = []
        self.unfinished = []
        self.errors = []
        self.t0 = None
        self.deadline = None
        self.grace = 5.0

    def _now(self):
        return time.perf_counter() - self.t0

    def _expired(self):
        return self.deadline is not None and self._now() >= self.deadline

    def run(self, requests, deadline=None):
        """Serve `requests` (their arrival times relative to the start); returns them finished.
        With a deadline, returns the requests finished by then (the others are in
        self.unfinished)."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if self.engine.footprint(r) > self.budget:
                raise ValueError("request %d needs more memory than the whole budget" % r.rid)
        self.deadline = deadline
        self.t0 = time.perf_counter()
        stop = threading.Event()
        threads = [threading.Thread(target=self._worker, args=(w, stop), daemon=True)
                   for w in range(self.nworkers)]
        for t in threads:
            t.start()
        try:
            self._admit_loop(pending)
            with self.lock:
                while len(self.done) < len(requests) and not self.errors and not self._expired():
                    self.lock.wait(0.05)
        finally:
            stop.set()
            with self.lock:
                self.lock.notify_all()
            for t in threads:
                t.join(None if deadline is None else self.grace)
            with self.lock:
                # requests of workers still busy past the grace period
                for w in range(self.nworkers):
                    for r, state, need in self.queues[w]:
                        if r not in self.unfinished:
                            self.unfinished.append(r)
        if self.errors:
            raise self.errors[0]
        return sorted(self.done, key=lambda r: r.rid)

    def _admit_loop(self, pending):
        nxt = 0
        for r in pending:
            need = self.engine.footprint(r)
            while not self.errors:
                if self._expired():
                    return
                wait = r.arrival - self._now()
                if wait > 0:
                    time.sleep(min(wait, 0.05))
                    continue
                with self.lock:
                    if self.free >= need:
                        self.free -= need
                        self.peak_used = max(self.peak_used, self.budget - self.free)
                        r.admitted = self._now()
                        # least-loaded worker takes it
                        w = min(range(self.nworkers), key=lambda i: (len(self.queues[i]), (i - nxt) % self.nworkers))
                        nxt = (w + 1) % self.nworkers
                        self.queues[w].append([r, None, need])
                        self.lock.notify_all()
                        break
                    self.lock.wait(0.05)

    def _worker(self, w, stop):
        try:
            self._serve(w, stop)
        except Exception as e:            # reported by run() on the calling thread
            with self.lock:
                self.errors.append(e)
                self.lock.notify_all()

    def _serve(self, w, stop):
        stream = self.engine.new_stream()
        while True:
            with self.lock:
                while not self.queues[w] and not stop.is_set():
                    self.lock.wait(0.05)
                if stop.is_set() and (not self.queues[w] or self._expired()):
                    self._drop_unfinished(w)
                    return
                batch = list(self.queues[w])
            for item in batch:
                if self._expired():
                    break
                r, state, need = item
                if state is None:
                    state, obs = self.engine.start(r, stream)
                    item[1] = state
                    r.readouts.append(obs)
                else:
                    r.readouts.append(self.engine.interval(r, state))
                if len(r.readouts) == r.n_intervals + 1:
                    self.engine.finish(r, state)
                    with self.lock:
                        self.queues[w].remove(item)
                        self.free += need
                        r.finished = self._now()
                        self.done.append(r)
                        self.lock.notify_all()


    def _drop_unfinished(self, w):
        """(lock held) after the deadline: release the worker's unfinished requests."""
        for r, state, need in self.queues[w]:
            if state is not None:
                self.engine.finish(r, state)
            self.free += need
            self.unfinished.append(r)
        self.queues[w] = []


def percentile(values, q):
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    v = sorted(values)
    if not v:
        return None
    pos = (len(v) - 1) * q / 100.0
    lo = int(pos)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (pos - lo)


def poisson_requests(n, rate, seed, d_choices=(2, 3, 4, 5, 6), t_max_choices=(2.0, 4.0, 8.0),
                     v_choices=(0.0, 0.5, 1.0), precision=1):
    """Seeded request stream: exponential gaps of mean 1/rate, D uniform in d_choices, chi uniform
    in [D^2, 3 D^2], h uniform in [0.5, 16], V and t_max uniform over their choices."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        D = int(rng.choice(d_choices))
        out.append(Request(rid=i, arrival=t, J=1.0, V=float(rng.choice(v_choices)),
                           h=float(rng.uniform(0.5, 16.0)), D=D,
                           chi=int(rng.integers(D * D, 3 * D * D + 1)),
                           t_max=float(rng.choice(t_max_choices)), precision=precision))
    return out
