"""Write the oracle's reference trajectories for the parity tests (calls only oracle/ and inputs/).

    python tests/golden/make_golden.py quench_d2      -> tests/golden/quench_d2_oracle.json
    python tests/golden/make_golden.py quench_d2_cut   -> tests/golden/quench_d2_cut1e-6_oracle.json
    python tests/golden/make_golden.py quench_d3      -> tests/golden/quench_d3_h{1,5,10}_oracle.json
    python tests/golden/make_golden.py quench_d3@5    -> tests/golden/quench_d3_h5_oracle.json only
    python tests/golden/make_golden.py quench_d3:2@5  -> the same, stopped at t = 2
    python tests/golden/make_golden.py quench_da3     -> tests/golden/quench_dA3_D3_oracle.json

Workloads: inputs.QUENCH_D2 (D=2, chi=8, first order dt=0.02 to t=1, measured every 0.1),
inputs.QUENCH_D3 (D=3, chi=18, second order dt=0.05 to t=5, measured every 0.25, h in {1,5,10}) and
inputs.QUENCH_DA3 (d_A=3 disorder levels, D=3, chi=9, second order dt=0.05 to t=0.5, every 0.1).
Every stored value is the oracle's; nothing here touches the CUDA path.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from inputs import QUENCH_D2, QUENCH_D3, QUENCH_DA3  # noqa: E402
from oracle import evolve  # noqa: E402

# at most this many sweeps for the stability probe of every readout (evolve.converge_and_measure)
PROBE = 100

KEYS = ("t", "nA", "nB", "imbalance", "tauzA", "tauzB", "energy", "purityA", "trunc_err_acc",
        "ctm_sweeps", "ctm_delta", "ctm_stop", "c8_margin", "c8_level", "drift", "probe_sweeps",
        "drift_split", "sensitivity", "renyi1A", "renyi_halfA", "renyi2A")


def _val(v):
    if isinstance(v, str):
        return v
    if isinstance(v, (int, np.integer)):
        return int(v)
    return min(float(v), 99.0)          # c8_margin is inf when no multiplet decision was taken


def _dump(path, params, out, seconds):
    rows = []
    for o in out:
        r = {k: _val(o[k]) for k in KEYS if k in o}
        r["lam"] = [[float(x) for x in row] for row in o["lam"]]
        # the same readout converged from the traced start (gauge independent, see evolve.run)
        r["cold"] = {k: _val(o["cold"][k]) for k in KEYS if k in o["cold"]}
        rows.append(r)
    with open(path, "w") as f:
        json.dump(dict(params=params, oracle_seconds=seconds, rows=rows), f, indent=1)


def run(name):
    if name == "quench_d2":
        p = dict(QUENCH_D2)
        t0 = time.time()
        out = evolve.run(p, tol=p["tol"], cold=True, probe_sweeps=PROBE)
        _dump(os.path.join(HERE, "quench_d2_oracle.json"), p, out, time.time() - t0)
    elif name == "quench_d2_cut":
        p = dict(QUENCH_D2, cut_rel=1e-6)
        t0 = time.time()
        out = evolve.run(p, tol=p["tol"], cold=True, probe_sweeps=PROBE)
        _dump(os.path.join(HERE, "quench_d2_cut1e-6_oracle.json"), p, out, time.time() - t0)
    elif name == "quench_da3":
        p = dict(QUENCH_DA3)
        t0 = time.time()
        out = evolve.run(p, tol=p["tol"], cold=True, probe_sweeps=PROBE)
        _dump(os.path.join(HERE, "quench_dA3_D3_oracle.json"), p, out, time.time() - t0)
    elif name.startswith("quench_d3"):
        # "quench_d3" = the full workload; "quench_d3:T" stops at t = T (same trajectory, fewer points);
        # "quench_d3@H" writes only the instance with h = H (the instances are independent)
        base, _, only = name.partition("@")
        t_max = float(base.split(":")[1]) if ":" in base else QUENCH_D3["t_max"]
        hs = [float(only)] if only else QUENCH_D3["hs"]
        for h in hs:
            p = {k: v for k, v in QUENCH_D3.items() if k != "hs"}
            p["h"] = h
            p["t_max"] = t_max
            t0 = time.time()
            out = evolve.run(p, tol=p["tol"], cold=True, probe_sweeps=PROBE,
                             callback=lambda o: print(name, h, o["t"], o["imbalance"],
                                                      o["cold"]["imbalance"], flush=True))
            _dump(os.path.join(HERE, "quench_d3_h%d_oracle.json" % int(h)), p, out, time.time() - t0)
    else:
        raise SystemExit("unknown workload " + name)


if __name__ == "__main__":
    for n in sys.argv[1:]:
        run(n)
