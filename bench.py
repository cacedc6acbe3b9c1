#!/usr/bin/env python
"""Benchmark of the iPEPS real-time-evolution hot path: Trotter + CTMRG steps per second.

Workload (one GPU): three instances of the dilated hard-core boson lattice (J = V = 1,
h = 1, 5, 10), PEPS bond dimension D = 3, environment chi = 18, second-order Trotter steps of
dt = 0.05 with the CTMRG environment converged to 1e-10 and the observables read out every 0.25
(every 5 Trotter steps), from t = 0 to t = 5.  One bench step is one such readout interval for all
three instances: 5 Trotter steps (7 bond updates each), CTMRG to convergence, measurement.  The
steps walk the trajectory in order and start again from the CDW state after t = 5.

metric  Trotter steps per second, summed over instances (and ranks), CTMRG and readout included
value   device-resident state, timed with CUDA events on the library's stream, per-launch events off
e2e     the same K steps through the public API with the state copied in from pinned host memory
        (ipeps_set_tensors) and the tensors, bond weights and observables copied back every step
roofline  from a separate profiled pass (per-launch CUDA events): the kernel class with the largest
          share, algorithmic flops per launch over its average duration, against GB300's FP64 rate
contraction  the standalone CTMRG contraction workload (random tensors, D = 6, chi = 72, split
          precision, 20 sweeps): algorithmic contraction TFLOP/s and the tcgen05 GEMM's own
          executed / algorithmic TFLOP/s against the measured BF16 peak
cpu_baseline  the FP64 oracle on the host: one whole readout interval of one instance

--impl reference times the oracle (this workload's reference implementation) instead.
Multi-GPU (torchrun): independent replicas, one per rank, no collectives on the data path.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

J, V, HS = 1.0, 1.0, (1.0, 5.0, 10.0)
D, CHI, ORDER, DT = 3, 18, 2, 0.05
STEPS_PER_READOUT = 5          # 0.25 / 0.05
TOL, MAX_SWEEPS = 1e-10, 500
METRIC = "Trotter+CTMRG steps/s"
UNIT = "Trotter steps/s"
WORKLOAD = ("iPEPS MBL quench, D=3 chi=18, 3 instances (J=V=1, h=1,5,10), 2nd-order dt=0.05, "
            "CTMRG to 1e-10 + readout every 0.25")
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--contraction-D", type=int, default=6,
                    help="bond dimension of the contraction sub-benchmark in the default line (0: skip)")
    ap.add_argument("--requests", type=int, default=400, help="serve workload: requests in the stream")
    ap.add_argument("--serve-seconds", type=float, default=240.0,
                    help="serve workload: window served per precision (seconds)")
    ap.add_argument("--serve-one", action="store_true",
                    help="serve workload: serve one window at --precision in this process and print its "
                         "summary (the parent runs one such process per precision)")
    ap.add_argument("--workload", choices=("quench", "ctmrg", "sweep", "serve", "ed"), default="quench",
                    help="quench: the Trotter+CTMRG readout workload (default); ctmrg: the standalone "
                         "CTMRG contraction benchmark on random tensors; sweep: the batched "
                         "64-instance disorder sweep; serve: the request stream; ed: the free-fermion "
                         "exact-diagonalisation workload")
    ap.add_argument("--sequential", action="store_true",
                    help="sweep workload: run the (D, chi) groups one after the other")
    ap.add_argument("--D", type=int, default=4, help="ctmrg workload: bond dimension (chi = 2 D^2)")
    ap.add_argument("--precision", choices=("fp64", "split"), default="fp64")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks sampler
class Clocks:
    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self._proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                          text=True)
        except OSError:
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()
        time.sleep(0.1)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.samples)}


# ----------------------------------------------------------------------------- oracle sample
ORACLE_STATE_T = 0.75          # the sampled readout interval is t = 0.75 -> 1.0 of the h = 5 instance
ORACLE_CODE = r"""
import json, sys, time
sys.path.insert(0, %r)
from oracle import ctmrg, evolve, measure, model, su
p = dict(J=1.0, V=1.0, h=5.0, D=3, chi=18, order=2, dt=0.05)
mode = sys.argv[1]
# state at t = 0.75 and its converged environment (preparation, not timed)
GA, GB, lam, _ = evolve.evolve_tensors(p, int(round(%r / p['dt'])))
A, B, a = evolve.ctm_state(GA, GB, lam)
env0, _, _ = ctmrg.ctmrg(a, ctmrg.init_env(a, 2, 2, 18, 3), 18, tol=1e-10, max_sweeps=500)
seq = su.trotter_sequence(2, 0.05)
gates = {d: model.gate(1.0, 1.0, 5.0, d) for _, d in seq}
def interval(full):
    t0 = time.perf_counter()
    g = (GA, GB, lam)
    for _ in range(5):
        g = su.trotter_step(g[0], g[1], g[2], gates, 2, 0.05)[:3]
    t1 = time.perf_counter()
    A2, B2, a2 = evolve.ctm_state(*g)
    if full:
        env, n, _ = ctmrg.ctmrg(a2, env0.copy(), 18, tol=1e-10, max_sweeps=500)
    else:
        env, n = ctmrg.sweep(a2, env0.copy(), 18), 1
    t2 = time.perf_counter()
    measure.observables(A2, B2, env, 1.0, 1.0, 5.0)
    t3 = time.perf_counter()
    return dict(su=t1 - t0, ctmrg=t2 - t1, sweeps=n, readout=t3 - t2, total=t3 - t0)
warm, count = int(sys.argv[2]), int(sys.argv[3])
for _ in range(warm):
    for _ in range(5):
        su.trotter_step(GA, GB, lam, gates, 2, 0.05)
print(json.dumps([interval(mode == "full") for _ in range(count)]))
"""


def oracle_run(mode, count=1, warmup=0, threads=1):
    """Run the oracle in one subprocess with ``threads`` BLAS/OpenMP threads and return ``count``
    timed samples (after ``warmup`` untimed repetitions of the 5 Trotter steps).  mode "full": one
    whole readout interval of one instance (t = 0.75 -> 1.0, h = 5: 5 second-order Trotter steps,
    CTMRG warm-started from the t = 0.75 environment and converged to 1e-10, full readout), timed
    end to end; mode "parts": the same 5 Trotter steps, ONE CTMRG sweep and the full readout, each
    timed.  The state at t = 0.75 and its converged environment are prepared once, untimed."""
    n = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n)
    out = subprocess.run([sys.executable, "-c", ORACLE_CODE % (ROOT, ORACLE_STATE_T), mode, str(warmup),
                          str(count)], capture_output=True, text=True, env=env, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


ORACLE_SAMPLE = ("one whole readout interval of one instance, timed end to end: t = 0.75 -> 1.0 of "
                 "the h = 5 instance (5 second-order Trotter steps, CTMRG warm-started from the "
                 "t = 0.75 environment and converged to 1e-10, full readout); the state and its "
                 "t = 0.75 environment are prepared untimed")


def oracle_sweeps_per_readout():
    """The oracle's own mean number of CTMRG sweeps per warm-started readout on this workload
    (t in (0, 5], h = 1, 5, 10), as recorded in its stored trajectories."""
    counts = []
    for h in HS:
        g = json.load(open(os.path.join(ROOT, "tests", "golden", "quench_d3_h%d_oracle.json" % int(h))))
        counts += [r["ctm_sweeps"] for r in g["rows"][1:]]
    return float(np.mean(counts)), len(counts)


def reference_main(args):
    """The oracle as the reference arm.  A whole readout interval of the oracle takes ~20 s, so a
    step times its three parts separately -- 5 Trotter steps, one CTMRG sweep and the full readout
    of the interval t = 0.75 -> 1.0 (h = 5) -- and the line composes them into a readout interval
    with the oracle's own mean sweeps per readout on this workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    t0 = time.perf_counter()
    parts = oracle_run("parts", count=args.steps, warmup=args.warmup)
    wall = time.perf_counter() - t0
    mean_sweeps, nrows = oracle_sweeps_per_readout()
    t_su = float(np.mean([q["su"] for q in parts]))
    t_sweep = float(np.mean([q["ctmrg"] for q in parts]))
    t_read = float(np.mean([q["readout"] for q in parts]))
    t_interval = t_su + mean_sweeps * t_sweep + t_read          # one instance, one readout interval
    value = STEPS_PER_READOUT / t_interval
    sample = ("per step, timed separately on one core: the 5 Trotter steps, one CTMRG sweep and the "
              "full readout of the interval t = 0.75 -> 1.0 (h = 5); composed into a readout interval "
              "as su + %.1f sweeps + readout, %.1f being the oracle's own mean sweeps per warm "
              "readout over its %d stored readouts of this workload (t in (0, 5], h = 1, 5, 10)"
              % (mean_sweeps, mean_sweeps, nrows))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_interval * len(HS), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "host run"},
            "composed": {"su_s": t_su, "sweep_s": t_sweep, "readout_s": t_read,
                         "sweeps_per_readout": mean_sweeps,
                         "run_seconds": wall, "timed_seconds": sum(q["total"] for q in parts)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def latency_summary(step_ms, sweep_ms):
    """p50 / p99 of the per-step (readout interval) times and of the per-sweep times (a step's time
    over the CTMRG sweeps it ran: the batch sweeps until its slowest instance converges), at the
    workload's stated error (FP64, CTMRG to 1e-10)."""
    return {"step_p50": float(np.percentile(step_ms, 50)), "step_p99": float(np.percentile(step_ms, 99)),
            "sweep_p50": float(np.percentile(sweep_ms, 50)), "sweep_p99": float(np.percentile(sweep_ms, 99))}


# ----------------------------------------------------------------------------- replicas
def reduce_max_ms(total_ms, dist, device):
    """Max over ranks of a replica's timed region (every rank receives it); no data-path collective
    exists: each rank runs its own independent instances."""
    if dist is None:
        return total_ms
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, max_ms):
    """Whole-job throughput of `world` replicas: all units processed over the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


# ----------------------------------------------------------------------------- native arm
CYCLE = 20                     # readout intervals from t = 0 to t = 5 (the workload's trajectory)
PROFILED_STEPS = 10            # steps of the separate profiled pass (kernel shares, roofline)
FP64_PEAK_TFLOPS = 1.25        # GB300 FP64 (no FP64 tensor path): 152 SMs x 2 DFMA/clk x 2.07 GHz x 2


class Quench:
    """The quench workload on one handle: a step is one readout interval (5 Trotter steps, CTMRG to
    convergence, readout) of the three instances; the trajectory runs t = 0 -> 5 and starts again
    from the CDW state after 20 intervals."""

    def __init__(self, pkg, stream):
        B = len(HS)
        self.sim = pkg.IPEPS([J] * B, [V] * B, list(HS), D=D, chi=CHI, order=ORDER, dt=DT,
                             stream=stream.cuda_stream)
        GA, GB = self.sim.get_tensors()
        self.initial = (GA, GB, self.sim.get_lambda())

    def restart(self, state=None):
        """Back to t = 0 (from host buffers: the CDW tensors), traced start, t = 0 readout."""
        GA, GB, lam = state if state is not None else self.initial
        self.sim.set_tensors(GA, GB, lam)
        self.sim.ctmrg_reset()
        self.sim.ctmrg_converge(tol=TOL, max_sweeps=MAX_SWEEPS, allow_noconv=True)
        self.sim.measure()

    def interval(self):
        self.sim.trotter_step(STEPS_PER_READOUT, sync=False)
        sw, dl, rc = self.sim.ctmrg_converge(tol=TOL, max_sweeps=MAX_SWEEPS, allow_noconv=True)
        return self.sim.measure(), sw

    def step(self, i):
        if i % CYCLE == 0:
            self.restart()
        return self.interval()


def timed_pass(q, steps, stream, flush, torch):
    """K steps from t = 0, each bracketed by CUDA events on the library's stream (L2 flushed before
    each step, outside the events).  Returns (total ms, per-step ms, per-step sweeps)."""
    total, step_ms, sweeps = 0.0, [], []
    for i in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, sw = q.step(i)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        total += ms
        step_ms.append(ms)
        sweeps.append([int(x) for x in sw])
    return total, step_ms, sweeps


def native_main(args):
    import torch
    import paper_1910_11359_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    B = len(HS)
    with torch.cuda.stream(stream):
        q = Quench(pkg, stream)
        for i in range(args.warmup):
            q.step(i)
        torch.cuda.synchronize()

        # ---- value: device-resident state, profiling off
        clocks = Clocks(local)
        clocks.start()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = pkg.launch_count()
        total_ms, step_ms, sweeps = timed_pass(q, args.steps, stream, flush, torch)
        torch.cuda.synchronize()
        launches = pkg.launch_count() - launches0
        total_ms = reduce_max_ms(total_ms, dist, "cuda")
        if dist is not None:
            dist.barrier()
        clk = clocks.stop()
        value = replica_throughput(B * STEPS_PER_READOUT * args.steps, world, total_ms)
        sweep_ms = [ms / max(1, max(sw)) for ms, sw in zip(step_ms, sweeps)]

        # ---- e2e: the same K steps through the public API with the state in pinned host memory:
        # every step copies the tensors in (ipeps_set_tensors), runs the interval and copies the
        # tensors, bond weights and observables back
        GA0, GB0, lam0 = q.initial
        hGA = torch.empty(GA0.shape + (2,), dtype=torch.float64).pin_memory().numpy().view(np.complex128)[..., 0]
        hGB = torch.empty(GB0.shape + (2,), dtype=torch.float64).pin_memory().numpy().view(np.complex128)[..., 0]
        hlam = torch.empty(lam0.shape, dtype=torch.float64).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(1.0)                     # the same L2 flush as the device-timed steps
            if i % CYCLE == 0:
                hGA[...], hGB[...], hlam[...] = GA0, GB0, lam0
                q.restart((hGA, hGB, hlam))
            q.sim.set_tensors(hGA, hGB, hlam)
            obs, _ = q.interval()
            gA, gB = q.sim.get_tensors()
            hGA[...], hGB[...] = gA, gB
            hlam[...] = q.sim.get_lambda()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_value = B * STEPS_PER_READOUT * args.steps * world / e2e_s
        h2d = 2 * GA0.nbytes + lam0.nbytes
        d2h = 2 * GA0.nbytes + lam0.nbytes + B * 88

        # ---- profiled pass (not timed for value): per-class CUDA-event times on the library's
        # stream, for the kernel shares and the roofline of the dominant kernel
        nprof = min(args.steps, PROFILED_STEPS)
        torch.cuda.synchronize()
        pkg.profile_enable(True)
        prof_ms, _, _ = timed_pass(q, nprof, stream, flush, torch)
        prof = pkg.profile_read()
        pkg.profile_enable(False)
        q.sim.close()

        contraction = None
        if rank == 0 and args.contraction_D > 0:
            contraction = contraction_bench(pkg, torch, args.contraction_D, stream)

    dom = max(prof.items(), key=lambda kv: kv[1][0])
    name, (ms, flops, n) = dom
    probe = pkg.fp64_peak_tflops()
    achieved = flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        tj = json.load(open(tfile))
        if tj.get("kernel") == name and tj.get("workload") == WORKLOAD and tj.get("source_sha") == _kernel_sha(name):
            traffic = tj.get("dram_bytes_per_launch")
    shares = {k: round(v[0] / prof_ms, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])
              if v[0] > 0}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    flat = [x for sw in sweeps for x in sw]
    full = oracle_run("full")[0]
    ncores = os.cpu_count() or 1
    full_all = oracle_run("full", threads=ncores)[0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": B, "D": D, "chi": CHI,
                   "parallelism": "replicas" if world > 1 else "single",
                   "trajectory": "steps cycle through the readout intervals of t = 0 -> 5 "
                                 "(interval i covers t = 0.25 (i mod 20) -> 0.25 (i mod 20 + 1); "
                                 "every 20 steps the state restarts from the CDW)",
                   "l2": "flushed (256 MiB write) between timed steps",
                   "mean_ctm_sweeps_per_readout": float(np.mean(flat)),
                   "physics": "past t ~ 0.5 the D = 3 state's accumulated discarded weight exceeds "
                              "the ~1e-3 the paper accepts (0.1 by t = 2): the numbers past that "
                              "time are outputs of the method, not converged physics"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": args.steps,
                "timing": "wall clock over the same K steps, L2 flushed before each step"},
        "roofline": {"bound": "alu", "kernel": name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "launches": n, "avg_launch_us": 1e3 * ms / max(n, 1),
                     "peak_source": "GB300 FP64 rate from the recipe's unit counts and clock "
                                    "(1.25 TFLOP/s; no FP64 tensor path); the FP64 FMA probe "
                                    "measured %.3f TFLOP/s in this run" % probe,
                     "timing": "CUDA events per launch in a separate profiled pass of %d steps "
                               "(value itself is timed with the per-launch events off)" % nprof},
        "kernel_time_share": shares,
        "latency_ms": latency_summary(step_ms, sweep_ms),
        # the timed pass runs each convergence as one CUDA graph, whose kernels the host does not
        # launch one by one: count kernel executions from the host-loop (profiled) pass instead
        "gpu_launches": int(round(sum(v[2] for v in prof.values()) * args.steps / max(1, nprof))),
        "gpu_launches_note": "kernel executions, counted per launch in the host-loop profiled pass and "
                             "scaled to the timed steps (the timed pass itself issued %d host launches "
                             "and graph launches)" % int(launches),
        "clocks": clk,
        "cpu_baseline": {"value": STEPS_PER_READOUT / full["total"], "unit": UNIT, "cores": 1,
                         "kind": "oracle", "sample": ORACLE_SAMPLE,
                         "sample_seconds": round(full["total"], 2), "sweeps": full["sweeps"],
                         "parts_s": {k: round(full[k], 3) for k in ("su", "ctmrg", "readout")},
                         "all_cores": {"value": STEPS_PER_READOUT / full_all["total"], "cores": ncores,
                                       "sample_seconds": round(full_all["total"], 2)},
                         "note": "the sampled interval needs %d CTMRG sweeps; the GPU run averaged "
                                 "%.1f sweeps per readout over its steps" % (full["sweeps"], float(np.mean(flat)))},
    }
    if contraction is not None:
        line["contraction"] = contraction
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# source files that define each kernel class the roofline may name (the kernel and what it includes)
KERNEL_SOURCES = {"jacobi_svd": ("linalg.cu", "linalg.cuh", "common.cuh", "prof.cuh"),
                  "zgemm_f64": ("linalg.cu", "linalg.cuh", "common.cuh", "prof.cuh")}


def _kernel_sha(kernel="jacobi_svd"):
    """Hash of the sources of one kernel class (all CUDA sources for a class not listed), to tell
    whether a stored ncu traffic figure still describes that kernel."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_11359_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or tuple(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    for f in sorted(files):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def contraction_bench(pkg, torch, D, stream, sweeps=20):
    """The standalone CTMRG contraction workload (random (4, D, D, D, D) tensors, chi = 2 D^2,
    split-precision contractions, 20 sweeps from the traced start): sweeps/s and algorithmic
    contraction TFLOP/s timed with the per-launch events off, then the tcgen05 GEMM's own
    executed and algorithmic TFLOP/s from a profiled pass of 4 sweeps."""
    from inputs import random_ctmrg_tensors
    chi = 2 * D * D
    A, B = random_ctmrg_tensors(D)
    sim = pkg.IPEPS([1.0], [1.0], [5.0], D=D, chi=chi, order=2, dt=0.05, precision=pkg.SPLIT_BF16X3,
                    stream=stream.cuda_stream)
    sim.set_tensors(A[None], B[None], None)
    sim.ctmrg_converge(tol=0.0, max_sweeps=2)
    sim.ctmrg_reset()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.ctmrg_converge(tol=0.0, max_sweeps=sweeps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    sim.ctmrg_reset()
    pkg.profile_enable(True)
    sim.ctmrg_converge(tol=0.0, max_sweeps=4)
    prof = pkg.profile_read()
    executed = pkg.profile_tc_executed()
    pkg.profile_enable(False)
    sim.close()
    peaks_file = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_file)) if os.path.exists(peaks_file) else {}
    bf16 = peaks.get("bf16_tflops", 1900.0)
    tms, tfl, tn = prof.get("tc_gemm_bf16", (0.0, 0.0, 0))
    tot = sum(v[0] for v in prof.values())
    algo = contraction_flops_per_sweep(D, chi) * sweeps
    return {"workload": "CTMRG contraction, random (4,D,D,D,D) N(0,1)+iN(0,1), D=%d chi=%d, %d sweeps "
                        "from the traced start, BF16x3 split contractions, FP64 projectors" % (D, chi, sweeps),
            "sweeps_per_s": sweeps / (ms * 1e-3),
            "contraction_tflops": algo / (ms * 1e-3) / 1e12,
            "contraction_frac_of_bf16_peak": algo / (ms * 1e-3) / 1e12 / bf16,
            "tc_gemm": None if not tn else {
                "launches": tn, "avg_launch_us": 1e3 * tms / tn,
                "algorithmic_tflops": tfl / (tms * 1e-3) / 1e12,
                "executed_tflops": executed / (tms * 1e-3) / 1e12,
                "peak": bf16, "frac_algorithmic": tfl / (tms * 1e-3) / 1e12 / bf16,
                "frac_executed": executed / (tms * 1e-3) / 1e12 / bf16,
                "share_of_sweep": tms / tot if tot else None,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)" if peaks else "fallback 1900"},
            "kernel_time_share": {k: round(v[0] / tot, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])
                                  if v[0] > 0 and tot > 0}}


def contraction_flops_per_sweep(D, chi):
    """Algorithmic real flops of one sweep's contractions (16 projector computations, explicit
    double layer; SVDs excluded): per projector 4 enlarged corners (C T: chi^2 D2 chi, T X1:
    chi D2 chi D2 chi, X2 a: chi^2 D2^4), 3 N^3 products, the projector products (2 N^2 chi) and the
    absorption (C1: chi N chi; T4: chi D2 chi chi + chi^2 D2^4 + chi N D2 chi; C4: chi D2 chi chi +
    chi N chi) -- counted for the two cuts a move computes, complex multiply-add = 8 flops."""
    D2 = D * D
    N = chi * D2
    corner = chi * chi * D2 * chi + chi * D2 * chi * D2 * chi + chi * chi * D2 ** 4
    per_cut = 4 * corner + 3 * N ** 3 + 2 * N * N * chi
    absorb = chi * N * chi + (chi * D2 * chi * chi + chi * chi * D2 ** 4 + chi * N * D2 * chi) \
        + (chi * D2 * chi * chi + chi * N * chi)
    return 8.0 * 8 * 2 * (per_cut + absorb)          # 8 moves x 2 cuts


def ctmrg_main(args):
    """Standalone CTMRG contraction benchmark: random (4, D, D, D, D) tensors, chi = 2 D^2, 20 sweeps
    per step from the traced start."""
    import torch
    import paper_1910_11359_gb300 as pkg
    from inputs import random_ctmrg_tensors

    D = args.D
    chi = 2 * D * D
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    prec = pkg.SPLIT_BF16X3 if args.precision == "split" else pkg.FP64
    A, B = random_ctmrg_tensors(D)
    sim = pkg.IPEPS([1.0], [1.0], [5.0], D=D, chi=chi, order=2, dt=0.05, precision=prec,
                    stream=stream.cuda_stream)
    sim.set_tensors(A[None], B[None], None)
    sweeps = 20
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sim.ctmrg_reset()
            sim.ctmrg_converge(tol=0.0, max_sweeps=sweeps)
        torch.cuda.synchronize()
        # timed with the per-launch events off (each convergence after its first sweep is one graph)
        total = 0.0
        for _ in range(args.steps):
            sim.ctmrg_reset()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.ctmrg_converge(tol=0.0, max_sweeps=sweeps)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        obs = sim.measure()[0]
        # profiled pass of one step (host loop, per-launch events): kernel shares, roofline, launches
        sim.ctmrg_reset()
        pkg.profile_enable(True)
        launches0 = pkg.launch_count()
        sim.ctmrg_converge(tol=0.0, max_sweeps=sweeps)
        prof = pkg.profile_read()
        pkg.profile_enable(False)
        launches = (pkg.launch_count() - launches0) * args.steps
        prof_total = sum(v[0] for v in prof.values())
    sim.close()
    flops = contraction_flops_per_sweep(D, chi) * sweeps * args.steps
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    name, (ms, fl, n) = dom
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    if name == "tc_gemm_bf16":
        peak, bound, unit = bf16_peak, "tensor", "TFLOP/s"
    else:
        peak, bound, unit = pkg.fp64_peak_tflops(), "alu", "TFLOP/s"
    tc_ms, tc_fl, tc_n = prof.get("tc_gemm_bf16", (0.0, 0.0, 0))
    line = {"metric": "CTMRG sweeps/s", "value": sweeps * args.steps / (total * 1e-3),
            "unit": "sweeps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3" if prec else "f64", "data": "synthetic",
            "config": {"workload": "CTMRG contraction, random (4,D,D,D,D), D=%d chi=%d, 20 sweeps" % (D, chi),
                       "precision": args.precision},
            "contraction_tflops": flops / (total * 1e-3) / 1e12,
            "roofline": {"bound": bound, "kernel": name, "achieved": fl / (ms * 1e-3) / 1e12 if ms else 0,
                         "peak": peak, "unit": unit, "frac": (fl / (ms * 1e-3) / 1e12) / peak if ms else 0,
                         "launches": n, "avg_launch_us": 1e3 * ms / max(n, 1)},
            "tensor_core_gemm": None if not tc_n else {
                "kernel": "tc_gemm_bf16", "launches": tc_n, "avg_launch_us": 1e3 * tc_ms / tc_n,
                "executed_tflops": tc_fl / (tc_ms * 1e-3) / 1e12, "peak": bf16_peak,
                "frac": tc_fl / (tc_ms * 1e-3) / 1e12 / bf16_peak,
                "peak_source": "MEASURED_PEAKS.json bf16 burst" if peaks else "fallback"},
            "kernel_time_share": {k: round(v[0] / prof_total, 4) for k, v in
                                  sorted(prof.items(), key=lambda kv: -kv[1][0]) if v[0] > 0},
            "gpu_launches": int(launches),
            "gpu_launches_note": "kernel executions of one step counted in a host-loop pass, times steps",
            "imbalance_after": obs["imbalance"]}
    print(json.dumps(line))
    return 0


def _sweep_run(prec, args, pts, conc):
    import torch
    from inputs import DISORDER_SWEEP
    from paper_1910_11359_gb300.sweep import disorder_sweep
    import paper_1910_11359_gb300 as pkg
    kw = dict(dt=DISORDER_SWEEP["dt"], order=DISORDER_SWEEP["order"], precision=prec, concurrent=conc)
    for _ in range(args.warmup):                      # handles, t = 0 readout
        disorder_sweep(pts, 0.0, DISORDER_SWEEP["meas_every"], **kw)
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    t_max = DISORDER_SWEEP["meas_every"] * args.steps
    t0 = time.perf_counter()
    out = disorder_sweep(pts, t_max, DISORDER_SWEEP["meas_every"], **kw)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return out, sec, t_max, pkg.launch_count() - launches0


def sweep_main(args):
    """Batched disorder sweep (64 instances of mixed D, one handle per (D, chi) group, groups on
    concurrent streams): `steps` readout intervals of 0.5 from t = 0, wall-clock timed, at the
    requested precision and then at the other one (split BF16x3 / FP64), with the largest imbalance
    difference between the two over every instance and readout."""
    from inputs import DISORDER_SWEEP, disorder_sweep_points
    from paper_1910_11359_gb300.sweep import group_points
    import paper_1910_11359_gb300 as pkg
    prec = pkg.SPLIT_BF16X3 if args.precision == "split" else pkg.FP64
    other = pkg.FP64 if prec != pkg.FP64 else pkg.SPLIT_BF16X3
    pts = disorder_sweep_points(DISORDER_SWEEP["n"])
    conc = not args.sequential
    out, sec, t_max, launches = _sweep_run(prec, args, pts, conc)
    out2, sec2, _, _ = _sweep_run(other, args, pts, conc)
    diff = max(abs(a["imbalance"] - b["imbalance"]) for o1, o2 in zip(out, out2) for a, b in zip(o1, o2))
    steps_total = len(pts) * round(t_max / DISORDER_SWEEP["dt"])
    pph = lambda s: len(pts) * 3600.0 / (s * DISORDER_SWEEP["t_max"] / t_max)
    name = lambda p: "split_bf16x3" if p else "fp64"
    line = {"metric": "instance Trotter steps/s", "value": steps_total / sec, "unit": "Trotter steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if prec else "f64", "data": "synthetic",
            "config": {"workload": "batched disorder sweep, 64 instances, h = linspace(0.5, 16, 64), "
                                   "V in {0, 1}, D in {2, 3, 4}, chi = 2 D^2, 2nd-order dt = 0.05, "
                                   "readout every 0.5 (timed from t = 0 to t = %.1f)" % t_max,
                       "groups": {"D=%d chi=%d" % k: len(v) for k, v in group_points(pts).items()},
                       "concurrent_groups": conc, "timing": "wall clock around the whole sweep"},
            "sweep_points_per_hour": {name(prec): pph(sec), name(other): pph(sec2)},
            "seconds": {name(prec): sec, name(other): sec2},
            "max_imbalance_difference_split_vs_fp64": diff,
            "gpu_launches": int(launches),
            "imbalance_last": [round(o[-1]["imbalance"], 6) for o in out[:4]]}
    print(json.dumps(line))
    return 0


def _serve_run(prec, args):
    """One bounded window of the request stream at the given precision (run in a process of its
    own: a worker may still be inside a long library call when the window ends)."""
    import torch
    from paper_1910_11359_gb300.serve import LibraryEngine, Server, percentile, poisson_requests
    import paper_1910_11359_gb300 as pkg
    reqs = poisson_requests(args.requests, rate=4.0, seed=5, d_choices=(2, 3, 4, 5, 6),
                            t_max_choices=(2.0, 4.0, 8.0), precision=prec)
    free, _ = torch.cuda.mem_get_info()
    srv = Server(LibraryEngine(tol=1e-10 if prec == pkg.FP64 else 1e-7), budget_bytes=free // 2,
                 workers=4)
    launches0 = pkg.launch_count()
    t0 = time.perf_counter()
    out = srv.run(reqs, deadline=args.serve_seconds)
    sec = time.perf_counter() - t0
    per = lambda r: int(round(r.meas_every / r.dt))
    steps = sum(per(r) * max(0, len(r.readouts) - 1) for r in out + srv.unfinished)
    lat = [r.latency for r in out]
    arrived = sum(1 for r in reqs if r.arrival <= sec)
    by_d = {}
    for r in out:
        by_d.setdefault(r.D, []).append(r.latency)
    return {"steps_per_s": steps / sec, "seconds": sec, "trotter_steps": steps, "arrived": arrived,
            "admitted": len(out) + len(srv.unfinished), "finished": len(out),
            "unfinished": len(srv.unfinished),
            "latency_s": {"p50": percentile(lat, 50), "p99": percentile(lat, 99),
                          "p50_by_D": {str(k): percentile(v, 50) for k, v in sorted(by_d.items())}},
            "budget_bytes": srv.budget, "peak_admitted_bytes": srv.peak_used,
            "gpu_launches": int(pkg.launch_count() - launches0)}


def serve_main(args):
    """Serving loop on the request stream: seeded Poisson requests (mean 4 per second), D in 2..6,
    chi in [D^2, 3 D^2], h in [0.5, 16], V in {0, 0.5, 1}, t_max in {2, 4, 8}, readouts every 0.5,
    admitted by footprint under half of the free device memory and run on 4 worker streams, split
    precision; then the same stream on the FP64 path.  A D = 6, chi = 108 request alone runs for
    hours on one GPU, so each precision is served for a bounded window (--serve-seconds), each in a
    process of its own: the line reports the Trotter steps completed in it (finished and unfinished
    requests alike), the latency of the requests that finished, and how many arrived, were
    admitted, finished."""
    import paper_1910_11359_gb300 as pkg
    if args.serve_one:
        prec = pkg.SPLIT_BF16X3 if args.precision == "split" else pkg.FP64
        print("SERVE " + json.dumps(_serve_run(prec, args)), flush=True)
        os._exit(0)                      # leave any worker still inside a library call behind
    runs = {}
    for prec in (args.precision, "fp64" if args.precision == "split" else "split"):
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", "serve", "--serve-one", "--precision", prec,
               "--requests", str(args.requests), "--serve-seconds", str(args.serve_seconds)]
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=args.serve_seconds + 900)
        lines = [l for l in out.stdout.splitlines() if l.startswith("SERVE ")]
        if not lines:
            raise RuntimeError("serve window at %s failed: %s" % (prec, out.stderr[-2000:]))
        runs[prec] = json.loads(lines[-1][6:])
    main = runs[args.precision]
    other_name = "fp64" if args.precision == "split" else "split"
    line = {"metric": "served Trotter steps/s", "value": main["steps_per_s"], "unit": "Trotter steps/s",
            "n_gpus": 1, "steps": main["trotter_steps"], "warmup": 0,
            "ms_per_step": 1e3 * main["seconds"] / max(1, main["trotter_steps"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if args.precision == "split" else "f64", "data": "synthetic",
            "config": {"workload": "serving loop, seeded Poisson stream of %d requests (mean 4/s), D in 2..6, "
                                   "chi in [D^2, 3 D^2], h in [0.5, 16], V in {0, 0.5, 1}, t_max in {2, 4, 8}, "
                                   "dt = 0.05, readouts every 0.5; served for a %.0f s window per precision"
                                   % (args.requests, args.serve_seconds),
                       "workers": 4, "timing": "wall clock over the window"},
            "served": main, other_name: runs[other_name],
            "gpu_launches": main["gpu_launches"],
            "gpu_launches_note": "host launch calls; convergences after their first sweep run as CUDA graphs"}
    print(json.dumps(line))
    return 0


def ed_main(args):
    """Free-fermion ED workload: 20 x 20 lattices (the paper's L = 20; its L = 40 exceeds the device
    eigensolver), 100 realisations, h = 10, continuous disorder and the three-level one, 51 times in
    [0, 5]; each step is one full ipeps_ed_run (host fields in, host readouts out) per disorder kind.
    The oracle is timed on a sample of the same workload."""
    import torch
    from inputs import ED, ed_fields
    import paper_1910_11359_gb300 as pkg
    L, R, h = 20, ED["R"], 10.0
    times = list(ED["times"])
    fields = {kind: ed_fields(L, R, h, lv, seed=31 + lv) for kind, lv in (("continuous", 0), ("discrete3", 3))}
    st = torch.cuda.Stream()
    for _ in range(args.warmup):
        for f in fields.values():
            pkg.ed_run(L, L, 1.0, f, times, stream=st.cuda_stream)
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for f in fields.values():
            out = pkg.ed_run(L, L, 1.0, f, times, stream=st.cuda_stream)
    sec = time.perf_counter() - t0
    launches = pkg.launch_count() - launches0
    pkg.profile_enable(True)
    for f in fields.values():
        pkg.ed_run(L, L, 1.0, f, times, stream=st.cuda_stream)
    prof = pkg.profile_read()
    pkg.profile_enable(False)
    total = sum(v[0] for v in prof.values())
    reals = 2 * R * args.steps
    dom_name, (dom_ms, dom_flops, dom_n) = max(prof.items(), key=lambda kv: kv[1][0])
    dom_tf = dom_flops / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
    # the oracle on 4 realisations of the continuous case, one thread (BLAS / LAPACK pinned to 1)
    code = ("import sys, time; sys.path.insert(0, %r); from inputs import ED, ed_fields; from oracle import ed; "
            "f = ed_fields(20, 100, 10.0, 0, seed=31)[:4]; t = time.perf_counter(); "
            "ed.run(20, 20, 1.0, f, list(ED['times'])); print(time.perf_counter() - t)" % ROOT)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    osec = float(subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                                timeout=900).stdout.strip().split()[-1])
    line = {"metric": "ED realisations/s", "value": reals / sec, "unit": "realisations/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "free-fermion ED, 20x20 open lattice, 100 realisations x {continuous, 3-level} "
                                   "disorder, h = 10, Neel evolution at 51 times in [0, 5], IPR + cumulative IPR",
                       "timing": "wall clock around ipeps_ed_run (host buffers in and out, workspace allocated "
                                 "per call)"},
            "kernel_time_share": {k: round(v[0] / total, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])
                                  if v[0] > 0},
            "roofline": {"bound": "alu", "kernel": dom_name, "achieved": dom_tf, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": dom_tf / FP64_PEAK_TFLOPS, "traffic": None,
                         "launches": dom_n, "avg_launch_us": 1e3 * dom_ms / max(dom_n, 1),
                         "timing": "CUDA events per launch in a separate profiled call (both disorder kinds)"},
            "jacobi_sweeps_mean": float(np.mean(out["sweeps"])),
            "gpu_launches": int(launches),
            "cpu_baseline": {"value": 4 / osec, "unit": "realisations/s", "cores": 1, "kind": "oracle",
                             "sample": "4 realisations of the continuous case (numpy eigh + occupations)"},
            "n_even_last": float(out["n_even"][-1]), "n_odd_last": float(out["n_odd"][-1])}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_main(args)
    if args.workload == "ctmrg":
        return ctmrg_main(args)
    if args.workload == "sweep":
        return sweep_main(args)
    if args.workload == "serve":
        return serve_main(args)
    if args.workload == "ed":
        return ed_main(args)
    return native_main(args)


if __name__ == "__main__":
    sys.exit(main())
