"""Batched disorder sweep: many independent instances of the quench, grouped by shape.

Every kernel of the library takes a batch of instances with one bond dimension D and one chi.
A sweep over disorder strength, interaction and D is therefore run as one handle per (D, chi)
group, whose instances share every launch, and the groups run concurrently: each on its own CUDA
stream, driven by its own host thread (the library's calls release the GIL through ctypes and only
synchronise their own stream).  This module only schedules; all arithmetic runs in libipeps.
"""
import threading

from ._lib import IPEPS, SPLIT_BF16X3


def group_points(points):
    """{(D, chi): [indices into points]} in first-seen order."""
    groups = {}
    for i, p in enumerate(points):
        groups.setdefault((int(p["D"]), int(p["chi"])), []).append(i)
    return groups


def _run_group(points, idx, D, chi, n_readouts, stride, order, dt, precision, tol, max_sweeps,
               out, errors, stream):
    try:
        import torch
        st = torch.cuda.Stream() if stream else None
        with torch.cuda.stream(st) if st is not None else _nullcontext():
            sim = IPEPS([points[i]["J"] for i in idx], [points[i]["V"] for i in idx],
                        [points[i]["h"] for i in idx], D=D, chi=chi, order=order, dt=dt,
                        precision=precision, stream=st.cuda_stream if st is not None else None)
            rows = []
            for r in range(n_readouts):
                if r > 0:
                    sim.trotter_step(stride, sync=False)
                sim.ctmrg_converge(tol=tol, max_sweeps=max_sweeps, allow_noconv=True)
                rows.append(sim.measure())
            sim.close()
        for k, i in enumerate(idx):
            out[i] = [row[k] for row in rows]
    except Exception as e:          # reported by disorder_sweep on the calling thread
        errors.append(e)


class _nullcontext:
    def __enter__(self):
        return None

    def __exit__(self, *a):
        return False


def disorder_sweep(points, t_max, meas_every, dt=0.05, order=2, precision=SPLIT_BF16X3, tol=1e-10,
                   max_sweeps=500, concurrent=True):
    """Evolve every point (dict with J, V, h, D, chi) from the CDW state to t_max, reading the
    observables out every meas_every.  Returns a list (one entry per point, input order) of lists
    of observation dicts at t = 0, meas_every, ..., t_max.  With concurrent=False the groups run one
    after the other on the default stream."""
    stride = int(round(meas_every / dt))
    n_readouts = int(round(t_max / meas_every)) + 1
    out = [None] * len(points)
    errors = []
    threads = []
    for (D, chi), idx in group_points(points).items():
        args = (points, idx, D, chi, n_readouts, stride, order, dt, precision, tol, max_sweeps,
                out, errors, concurrent)
        if concurrent:
            t = threading.Thread(target=_run_group, args=args)
            t.start()
            threads.append(t)
        else:
            _run_group(*args)
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return out
