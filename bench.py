#!/usr/bin/env python
"""Benchmark of the iPEPS real-time-evolution hot path: Trotter + CTMRG steps per second.

Workload (one GPU): three instances of the dilated hard-core boson lattice (J = V = 1,
h = 1, 5, 10), PEPS bond dimension D = 3, environment chi = 18, second-order Trotter steps of
dt = 0.05 with the CTMRG environment converged to 1e-10 and the observables read out every 0.25
(every 5 Trotter steps).  One bench step is one such readout interval for all three instances:
5 Trotter steps (7 bond updates each), CTMRG to convergence, measurement.

metric  Trotter steps per second, summed over instances (and ranks), CTMRG and readout included
value   device-resident state, timed with CUDA events on the library's stream
e2e     the same steps through the public API with the state copied in from pinned host memory
        (ipeps_set_tensors) and the tensors and observables copied back every step
roofline  the kernel class with the largest share of the timed region, algorithmic flops per
          launch over its event-timed average duration, against the FP64 rate measured in this run
cpu_baseline  the FP64 oracle on the host, one instance, a bounded sample of the same workload

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
REFERENCE_SWEEPS_PER_READOUT = 87.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--requests", type=int, default=32, help="serve workload: requests in the stream")
    ap.add_argument("--workload", choices=("quench", "ctmrg", "sweep", "serve"), default="quench",
                    help="quench: the Trotter+CTMRG readout workload (default); ctmrg: the standalone "
                         "CTMRG contraction benchmark on random tensors; sweep: the batched "
                         "64-instance disorder sweep")
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
ORACLE_SAMPLE = ("one instance (h=5), 5 second-order Trotter steps from t=0, 2 CTMRG sweeps from "
                 "the traced start and one readout; scaled to a full step with the GPU run's mean "
                 "sweeps per readout")


def oracle_sample(sweeps_per_readout, threads=1):
    """Time the oracle on a bounded sample with `threads` BLAS/OpenMP threads; returns (steps/s,
    sample seconds, parts)."""
    code = r"""
import json, sys, time
sys.path.insert(0, %r)
from oracle import ctmrg, evolve, measure
p = dict(J=1.0, V=1.0, h=5.0, D=3, chi=18, order=2, dt=0.05)
t0 = time.perf_counter(); GA, GB, lam, _ = evolve.evolve_tensors(p, 5); t1 = time.perf_counter()
A, B, a = evolve.ctm_state(GA, GB, lam)
env = ctmrg.init_env(a, 2, 2, 18, 3)
t2 = time.perf_counter()
for _ in range(2):
    env = ctmrg.sweep(a, env, 18)
t3 = time.perf_counter()
measure.observables(A, B, env, 1.0, 1.0, 5.0)
t4 = time.perf_counter()
print(json.dumps(dict(su=t1 - t0, sweep=(t3 - t2) / 2, measure=t4 - t3, total=t4 - t0)))
""" % ROOT
    n = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=600)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    per_instance = r["su"] + sweeps_per_readout * r["sweep"] + r["measure"]
    rate = STEPS_PER_READOUT / per_instance          # Trotter steps/s for one instance
    return rate, r["total"], r


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # CTMRG sweeps per readout of this workload (same tolerance and stall rule as the oracle's),
    # mean over instances measured on the GPU path: the oracle needs as many
    mean_sweeps = REFERENCE_SWEEPS_PER_READOUT
    times = []
    samples = []
    for i in range(args.warmup + args.steps):
        rate, sec, r = oracle_sample(mean_sweeps)
        if i >= args.warmup:
            times.append(STEPS_PER_READOUT / rate * len(HS))
            samples.append(rate)
    value = len(HS) * STEPS_PER_READOUT * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": ORACLE_SAMPLE + "; %.0f sweeps per readout assumed" % mean_sweeps},
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
    sim = pkg.IPEPS([J] * B, [V] * B, list(HS), D=D, chi=CHI, order=ORDER, dt=DT,
                    stream=stream.cuda_stream)

    def step():
        sim.trotter_step(STEPS_PER_READOUT, sync=False)
        sw, dl, rc = sim.ctmrg_converge(tol=TOL, max_sweeps=MAX_SWEEPS, allow_noconv=True)
        return sim.measure(), sw

    with torch.cuda.stream(stream):
        sim.ctmrg_converge(tol=TOL, max_sweeps=MAX_SWEEPS, allow_noconv=True)
        sim.measure()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks = Clocks(local)
        clocks.start()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = pkg.launch_count()
        pkg.profile_enable(True)
        total_ms = 0.0
        sweeps = []
        step_ms = []
        sweep_ms = []                                         # per step: time / sweeps run
        last = None
        for _ in range(args.steps):
            flush.fill_(1.0)                                  # L2 flush between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last, sw = step()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            total_ms += ms
            step_ms.append(ms)
            sweep_ms.append(ms / max(1, max(int(s) for s in sw)))
            sweeps.extend(int(s) for s in sw)
        torch.cuda.synchronize()
        prof = pkg.profile_read()
        pkg.profile_enable(False)
        launches = pkg.launch_count() - launches0
        total_ms = reduce_max_ms(total_ms, dist, "cuda")
        if dist is not None:
            dist.barrier()
        clk = clocks.stop()
        value = replica_throughput(B * STEPS_PER_READOUT * args.steps, world, total_ms)

        # end to end through the public API with host buffers (pinned), copies inside the timing
        GA, GB = sim.get_tensors()
        lam = sim.get_lambda()
        hGA = torch.from_numpy(GA.view(np.float64)).pin_memory().numpy().view(np.complex128)
        hGB = torch.from_numpy(GB.view(np.float64)).pin_memory().numpy().view(np.complex128)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sim.set_tensors(hGA, hGB, lam)
            obs, _ = step()
            gA, gB = sim.get_tensors()
            hGA[...] = gA
            hGB[...] = gB
            lam = sim.get_lambda()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_value = B * STEPS_PER_READOUT * args.e2e_steps * world / e2e_s
        h2d = 2 * GA.nbytes + lam.nbytes
        d2h = 2 * GA.nbytes + lam.nbytes + B * 88
    sim.close()

    # roofline of the dominant kernel class
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    name, (ms, flops, n) = dom
    peak = pkg.fp64_peak_tflops()
    achieved = flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        tj = json.load(open(tfile))
        if tj.get("kernel") == name and tj.get("workload") == WORKLOAD:
            traffic = tj.get("dram_bytes_per_launch")
    shares = {k: round(v[0] / total_ms, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])
              if v[0] > 0}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    mean_sweeps = float(np.mean(sweeps)) if sweeps else 10.0
    cpu_rate, cpu_sec, cpu_parts = oracle_sample(mean_sweeps)
    ncores = os.cpu_count() or 1
    all_rate, all_sec, _ = oracle_sample(mean_sweeps, threads=ncores)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": B, "D": D, "chi": CHI,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed (256 MiB write) between timed steps",
                   "mean_ctm_sweeps_per_readout": mean_sweeps},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                     "traffic": traffic, "launches": n, "avg_launch_us": 1e3 * ms / max(n, 1),
                     "peak_source": "FP64 FMA rate measured in this run (no FP64 tensor path)"},
        "kernel_time_share": shares,
        "latency_ms": latency_summary(step_ms, sweep_ms),
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": ORACLE_SAMPLE, "sample_seconds": round(cpu_sec, 2),
                         "parts_s": {k: round(v, 3) for k, v in cpu_parts.items()},
                         "all_cores": {"value": all_rate, "cores": ncores,
                                       "sample_seconds": round(all_sec, 2)}},
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


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
        pkg.profile_enable(True)
        launches0 = pkg.launch_count()
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
        prof = pkg.profile_read()
        pkg.profile_enable(False)
        launches = pkg.launch_count() - launches0
        obs = sim.measure()[0]
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
            "kernel_time_share": {k: round(v[0] / total, 4) for k, v in
                                  sorted(prof.items(), key=lambda kv: -kv[1][0]) if v[0] > 0},
            "gpu_launches": int(launches), "imbalance_after": obs["imbalance"]}
    print(json.dumps(line))
    return 0


def sweep_main(args):
    """Batched disorder sweep (64 instances of mixed D, one handle per (D, chi) group, groups on
    concurrent streams): `steps` readout intervals of 0.5 from t = 0, wall-clock timed."""
    import torch
    from inputs import DISORDER_SWEEP, disorder_sweep_points
    from paper_1910_11359_gb300.sweep import disorder_sweep, group_points
    import paper_1910_11359_gb300 as pkg
    prec = pkg.SPLIT_BF16X3 if args.precision == "split" else pkg.FP64
    pts = disorder_sweep_points(DISORDER_SWEEP["n"])
    conc = not args.sequential
    for _ in range(args.warmup):                      # handles, t = 0 readout
        disorder_sweep(pts, 0.0, DISORDER_SWEEP["meas_every"], dt=DISORDER_SWEEP["dt"], order=DISORDER_SWEEP["order"],
                       precision=prec, concurrent=conc)
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    t_max = DISORDER_SWEEP["meas_every"] * args.steps
    t0 = time.perf_counter()
    out = disorder_sweep(pts, t_max, DISORDER_SWEEP["meas_every"], dt=DISORDER_SWEEP["dt"], order=DISORDER_SWEEP["order"],
                         precision=prec, concurrent=conc)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    launches = pkg.launch_count() - launches0
    steps_total = len(pts) * round(t_max / DISORDER_SWEEP["dt"])
    line = {"metric": "instance Trotter steps/s", "value": steps_total / sec, "unit": "Trotter steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if prec else "f64", "data": "synthetic",
            "config": {"workload": "batched disorder sweep, 64 instances, h = linspace(0.5, 16, 64), "
                                   "V in {0, 1}, D in {2, 3, 4}, chi = 2 D^2, 2nd-order dt = 0.05, "
                                   "readout every 0.5 (timed from t = 0 to t = %.1f)" % t_max,
                       "groups": {"D=%d chi=%d" % k: len(v) for k, v in group_points(pts).items()},
                       "concurrent_groups": conc, "timing": "wall clock around the whole sweep"},
            "sweep_points_per_hour": len(pts) * 3600.0 / (sec * DISORDER_SWEEP["t_max"] / t_max),
            "gpu_launches": int(launches),
            "imbalance_last": [round(o[-1]["imbalance"], 6) for o in out[:4]]}
    print(json.dumps(line))
    return 0


def serve_main(args):
    """Serving loop: a seeded Poisson stream of quench requests (mean 4 per second, D in 2..4,
    chi in [D^2, 3 D^2], h in [0.5, 16], V in {0, 0.5, 1}, t_max in {1, 2}, readouts every 0.5),
    admitted by footprint under half of the free device memory, run on 4 worker streams."""
    import torch
    from paper_1910_11359_gb300.serve import LibraryEngine, Server, percentile, poisson_requests
    import paper_1910_11359_gb300 as pkg
    prec = pkg.SPLIT_BF16X3 if args.precision == "split" else pkg.FP64
    reqs = poisson_requests(args.requests, rate=4.0, seed=5, d_choices=(2, 3, 4),
                            t_max_choices=(1.0, 2.0), precision=prec)
    free, _ = torch.cuda.mem_get_info()
    srv = Server(LibraryEngine(tol=1e-10 if prec == pkg.FP64 else 1e-7), budget_bytes=free // 2,
                 workers=4)
    launches0 = pkg.launch_count()
    t0 = time.perf_counter()
    out = srv.run(reqs)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    lat = [r.latency for r in out]
    steps = sum(int(round(r.t_max / r.dt)) for r in out)
    line = {"metric": "served Trotter steps/s", "value": steps / sec, "unit": "Trotter steps/s",
            "n_gpus": 1, "steps": len(out), "warmup": 0, "ms_per_step": 1e3 * sec / len(out),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if prec else "f64", "data": "synthetic",
            "config": {"workload": "serving loop, %d Poisson requests (mean 4/s), D in 2..4, "
                                   "chi in [D^2, 3 D^2], t_max in {1, 2}" % len(out),
                       "budget_bytes": srv.budget, "peak_admitted_bytes": srv.peak_used,
                       "workers": srv.nworkers, "timing": "wall clock over the whole stream"},
            "latency_s": {"p50": percentile(lat, 50), "p99": percentile(lat, 99)},
            "gpu_launches": int(pkg.launch_count() - launches0)}
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
    return native_main(args)


if __name__ == "__main__":
    sys.exit(main())
