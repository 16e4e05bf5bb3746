"""Benchmark: grid-point stage updates per second of the TVD-RK3 step on the
256^3 decaying isotropic-turbulence workload (hybrid UD7/WENO7/WENO5 scheme,
viscous, periodic box), through the C ABI of the CUDA library.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--precision fp64] [--n 256]

Prints one JSON line on rank 0.  The path does not exchange data between
ranks (each rank advances its own independent box), so N > 1 runs replicas
(weak scaling) with a barrier and max-over-ranks timing.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SEED = 20220930
MT = 0.5
GAMMA = 1.4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="one stage profile, for ncu runs")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n):
    from paper_2209_15333_gb300 import cases
    U, Re = cases.isotropic_turbulence(n, SEED, Mt=MT, gamma=GAMMA)
    met = cases.uniform_metrics(n, n, n)
    params = dict(gamma=GAMMA, Re=Re, Ma=MT, Pr=0.72, visc_law=1, visc_omega=0.76, scheme=3, theta1=0.02,
                  theta2=0.1, visc_order=8)
    return U, met, params, Re


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# algorithmic FP64 flops per node of each kernel of the UD7 path, counted from
# the kernel source (FMA = 2 flops; division and square root = 1 flop each)
ALGO_FLOPS = {
    "sweep": None,  # filled from flop_counts()
}


def flop_counts():
    """Per-node flop counts of the UD7 / viscous path."""
    sw = 53               # split fluxes of one node, one direction (both signs)
    recon = 5 * 2 * 13 + 5  # UD7 +/- for 5 components (7 coefficients: 6 FMA + 1 MUL) and the sum
    diff = 5
    visc_div = 4 * (2 * 4 + 1 + 3)  # 8th-order central of 4 rows
    per_sweep = sw + recon + diff + visc_div
    visc_flux = 12 * 12 + 9 * 3 * 2 + 60 + 40
    return {"sweep": per_sweep, "visc_flux": visc_flux}


def time_oracle(n, steps_of_three=1, threads=None):
    """The oracle, as it stands, on host cores: one RK3 step of an n^3 box of
    the same workload recipe.  Returns (point-stage/s, seconds, threads)."""
    import oracle
    from paper_2209_15333_gb300 import cases
    U, met, params, Re = workload(n)
    M = cases.expand_metrics(met, (n, n, n))
    th = threads or (os.cpu_count() or 1)
    c = oracle.Case(n, n, n, gamma=GAMMA, Re=Re, Ma=MT, Pr=0.72, visc_law=1, visc_omega=0.76, scheme=3,
                    theta1=0.02, theta2=0.1, visc_order=8, nthreads=th)
    dt = oracle.cfl_dt(c, M, U, 0.5)
    t0 = time.perf_counter()
    oracle.step(c, M, U, dt, steps_of_three)
    el = time.perf_counter() - t0
    return n ** 3 * 3 * steps_of_three / el, el, th


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the machine's host cores (rank 0 only)."""
    if rank != 0:
        return
    n = min(args.n, 128)
    for _ in range(args.warmup):
        time_oracle(n)
    tot, pts = 0.0, 0
    th = os.cpu_count() or 1
    for _ in range(args.steps):
        v, el, th = time_oracle(n)
        tot += el
        pts += n ** 3 * 3
    value = pts / tot
    line = {
        "impl": "reference", "metric": "grid-point stage updates/s", "value": value,
        "unit": "point-stage/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "isotropic turbulence %d^3 sample of the %d^3 case, hybrid, FP64" % (n, args.n)},
        "cpu_baseline": {"value": value, "unit": "point-stage/s", "cores": th, "kind": "oracle",
                         "sample": "one RK3 step per timed step of a %d^3 box of the same recipe" % n},
        "e2e": {"value": value, "unit": "point-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    torch.cuda.set_device(local)
    from paper_2209_15333_gb300 import build
    build.build()
    from paper_2209_15333_gb300.solver import Solver

    n = args.n
    U, met, params, Re = workload(n)
    N = n ** 3
    stream = torch.cuda.Stream()
    s = Solver((n, n, n), met, stream=stream, **params)
    Ud = torch.tensor(U, device="cuda")
    s.set_state(Ud)
    dt = s.cfl_dt(0.5)
    if args.profile_only:
        s.profile_stage(1)
        torch.cuda.synchronize()
        return

    for _ in range(args.warmup):
        s.step(dt, 1)
    s.sync(600.0)

    clocks = ClockSampler(local)
    clocks.start()
    l0 = s.launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(dt, args.steps)
    e1.record(stream)
    s.sync(600.0)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = s.launches() - l0
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    cls = s.flags()
    frac = np.bincount(cls.ravel(), minlength=3) / cls.size
    value = world * N * 3 * args.steps / (ms * 1e-3)

    # end to end through the public API with host buffers: H2D of the state,
    # one step, D2H of the result, every step
    host_in = torch.from_numpy(s.get_state()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_state(host_in)
        s.step(dt, 1)
        s.get_state(out=host_out)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * N * 3 * args.steps / e2e_s

    # per-kernel times (CUDA events on the context stream, no graph)
    prof = s.profile_stage(3)
    dom = max(prof, key=prof.get)
    fc = flop_counts()
    fp64_peak = None
    try:
        import ctypes as C
        from paper_2209_15333_gb300 import _lib
        v = C.c_double()
        _lib.check(_lib.lib().cfd_fma_peak(0, C.byref(v)))
        fp64_peak = v.value
        v32 = C.c_double()
        _lib.check(_lib.lib().cfd_fma_peak(1, C.byref(v32)))
        fp32_peak = v32.value
    except Exception:
        fp32_peak = None
    peaks, peak_kind = measured_peaks()
    kind = "sweep" if dom.startswith("sweep") else dom
    flops = fc.get(kind, fc["sweep"]) * N
    achieved = flops / (prof[dom] * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": (achieved / fp64_peak) if fp64_peak else None, "traffic": None,
            "peak_source": "cfd_fma_peak FP64 FMA probe (measured in this run)",
            "kernel_ms": prof}
    alg_bytes = (40 + 26.7 + 40) * N * 3 * args.steps
    hbm_frac = alg_bytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, el, th = time_oracle(n)
        cpu = {"value": v, "unit": "point-stage/s", "cores": th, "kind": "oracle",
               "sample": "one RK3 step (3 stages) of the full %d^3 field, %.1f s" % (n, el)}

    if rank == 0:
        line = {
            "metric": "grid-point stage updates/s", "value": value, "unit": "point-stage/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "decaying isotropic turbulence %d^3 periodic, hybrid UD7/WENO7/WENO5, "
                                   "8th-order viscous, FP64" % n, "grid": [n, n, n], "Re": Re, "Mt": MT,
                       "seed": SEED, "l2": "inputs larger than L2 (state %d MB)" % (40 * N // 2 ** 20),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "class_fraction": [float(x) for x in frac]},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "point-stage/s", "h2d_bytes_per_step": 40 * N,
                    "d2h_bytes_per_step": 40 * N},
            "gpu_launches": launches,
            "roofline": roof,
            "hbm_algorithmic": {"bytes_per_point_stage": 106.7, "frac": hbm_frac, "peak_gbs": peaks["hbm_gbs"],
                                "peak_source": peak_kind},
            "fp32_fma_peak_tflops": fp32_peak,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
