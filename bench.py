"""Benchmark: grid-point stage updates per second of the TVD-RK3 step on the
256^3 decaying isotropic-turbulence workload (hybrid UD7/WENO7/WENO5 scheme,
8th-order viscous terms, periodic box), through the C ABI of the CUDA library.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--precision both|mixed|fp64] [--n 256]

Rank 0 prints one JSON line.  The headline `value` is the FP32-bulk/FP64-state
form; the plain FP64 form is reported beside it under "fp64", each with its
error against the FP64 oracle after one RK3 step of the full field.  The path
exchanges no data between ranks (independent boxes), so N > 1 runs replicas
with a barrier and max-over-ranks timing (weak scaling).
"""
import argparse
import hashlib
import json
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
KERNEL_NAMES = ["prim", "sensor", "visc_flux", "sweep_xi", "sweep_eta", "sweep_zeta"]

# Algorithmic work per node of each kernel:
# FP64 form: counted flops (FMA = 2; division, sqrt, pow = 1);
# mixed form: compulsory bytes (inputs read once, outputs written once).
FP64_FLOPS = {"prim": 25, "sensor": 20, "visc_flux": 305, "sweep_xi": 247, "sweep_eta": 252, "sweep_zeta": 277}
MIXED_BYTES = {"prim": 69, "sensor": 5, "visc_flux": 64, "sweep_xi": 57, "sweep_eta": 77, "sweep_zeta": 164}
# DRAM bytes per node measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# on a 160^3 stage (the profiles directory), valid for the kernel sources with this
# hash prefix and the variant each kernel ran in; scaled to the full launch by the
# node count (traffic grows with it: the arrays exceed L2).
NCU_TRAFFIC = {
    "fp64": {"src": "90a3a246dda5", "per_node": {"visc_flux": 116.9, "sweep_xi": 106.4, "sweep_eta": 151.5,
                                                 "sweep_zeta": 160.3},
             "variant": {"visc_flux": [3, 0], "sweep_xi": None, "sweep_eta": [1, 16], "sweep_zeta": [1, 16]}},
    "mixed": {"src": "90a3a246dda5", "per_node": {"visc_flux": 51.9, "sweep_xi": 50.2, "sweep_eta": 72.6,
                                                  "sweep_zeta": 91.0},
              "variant": {"visc_flux": [3, 0], "sweep_xi": None, "sweep_eta": [1, 16], "sweep_zeta": [1, 16]}},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="one profiled stage per precision (ncu runs)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 48-block ensemble measurement")
    ap.add_argument("--variants", default="", help="pin kernel variants, e.g. 0:2,1:1:16,2:1:16 (dir:kind[:param])")
    return ap.parse_args()


def max_over_ranks(x, world, device="cuda"):
    """The largest x over all ranks (x itself on one rank): the job's time
    is its slowest replica's."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, nodes, steps, seconds):
    """Whole-job point-stage updates per second: every rank advances its own
    replica of `nodes` nodes by `steps` RK3 steps of 3 stages."""
    return world * nodes * 3 * steps / seconds


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def workload(n):
    from paper_2209_15333_gb300 import cases
    U, Re = cases.isotropic_turbulence(n, SEED, Mt=MT, gamma=GAMMA)
    met = cases.uniform_metrics(n, n, n)
    params = dict(gamma=GAMMA, Re=Re, Ma=MT, Pr=0.72, visc_law=1, visc_omega=0.76, scheme=3, theta1=0.02,
                  theta2=0.1, visc_order=8)
    return U, met, params, Re


def kernel_src_hash():
    h = hashlib.sha256()
    for f in ("cfd_kernels.cuh", "weno_coeffs.cuh"):
        with open(os.path.join(ROOT, "paper_2209_15333_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def field_rel_err(a, b):
    e = 0.0
    for q in range(a.shape[0]):
        den = float(np.abs(b[q]).max())
        num = float(np.abs(a[q] - b[q]).max())
        e = max(e, num / den if den > 0 else num)
    return e


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
            threading.Thread(target=self._read, daemon=True).start()
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


def fma_peaks():
    import ctypes as C
    from paper_2209_15333_gb300 import _lib
    out = {}
    for name, prec in (("fp64", 0), ("fp32", 1)):
        v = C.c_double()
        _lib.check(_lib.lib().cfd_fma_peak(prec, C.byref(v)))
        out[name] = v.value
    return out


def oracle_step(n, U, dt, threads=None):
    """The oracle, as it stands: one RK3 step of the n^3 field on host cores."""
    import oracle
    from paper_2209_15333_gb300 import cases
    _, met, params, Re = workload_params(n)
    M = cases.expand_metrics(met, (n, n, n))
    th = threads or (os.cpu_count() or 1)
    c = oracle.Case(n, n, n, gamma=GAMMA, Re=Re, Ma=MT, Pr=0.72, visc_law=1, visc_omega=0.76, scheme=3,
                    theta1=0.02, theta2=0.1, visc_order=8, nthreads=th)
    t0 = time.perf_counter()
    U1 = oracle.step(c, M, U, dt, 1)
    return U1, time.perf_counter() - t0, th


_WL = {}


def workload_params(n):
    if n not in _WL:
        _WL[n] = workload(n)
    return _WL[n]


def arm_config(n, Re, world, precision):
    """The workload both arms report (the reference arm times a bounded
    sample of it, stated in its cpu_baseline)."""
    N = n ** 3
    return {"workload": "decaying isotropic turbulence %d^3 periodic, hybrid UD7/WENO7/WENO5, 8th-order "
                        "viscous" % n,
            "grid": [n, n, n], "Re": Re, "Mt": MT, "seed": SEED,
            "l2": "inputs larger than L2 (state %d MB)" % (40 * N // 2 ** 20),
            "parallelism": "replicas" if world > 1 else "single GPU", "precision": precision}


def run_reference(args, rank):
    """Reference arm: the CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    n = min(args.n, 128)
    U, met, params, Re = workload_params(n)
    import oracle
    from paper_2209_15333_gb300 import cases
    M = cases.expand_metrics(met, (n, n, n))
    dt = oracle.cfl_dt(oracle.Case(n, n, n, Ma=MT), M, U, 0.5)
    for _ in range(args.warmup):
        oracle_step(n, U, dt)
    tot, th = 0.0, 1
    for _ in range(args.steps):
        _, el, th = oracle_step(n, U, dt)
        tot += el
    value = n ** 3 * 3 * args.steps / tot
    line = {
        "impl": "reference", "metric": "grid-point stage updates/s", "value": value, "unit": "point-stage/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(args.n, workload_params(args.n)[3], args.gpus, "FP64 CPU oracle"),
        "cpu_baseline": {"value": value, "unit": "point-stage/s", "cores": th, "kind": "oracle",
                         "sample": "one RK3 step of a %d^3 box of the same recipe per timed step (the %d^3 "
                                   "case's throughput is measured on a bounded sample)" % (n, args.n)},
        "e2e": {"value": value, "unit": "point-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_precision(args, prec, U, met, params, world, local, dt):
    """Time K graph-replayed steps of one precision; returns a result dict."""
    import torch
    from paper_2209_15333_gb300.solver import Solver
    n = args.n
    N = n ** 3
    stream = torch.cuda.Stream()
    s = Solver((n, n, n), met, stream=stream, precision=1 if prec == "mixed" else 0, **params)
    Ud = torch.tensor(U, device="cuda")
    s.set_state(Ud)
    for item in filter(None, args.variants.split(",")):
        f = [int(x) for x in item.split(":")]
        s.set_sweep_variant(f[0], f[1], f[2] if len(f) > 2 else 0)
    if args.profile_only:
        s.profile_stage(1)
        s.close()
        return None
    # accuracy: one RK3 step from the initial field
    s.step(dt, 1)
    U1 = s.get_state()
    s.set_state(Ud)
    s.set_time(0.0)
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
    ms = max_over_ranks(ms, world)
    cls = s.flags()
    frac = np.bincount(cls.ravel(), minlength=3)[:3] / cls.size
    value = job_throughput(world, N, args.steps, ms * 1e-3)
    # end to end through the public API with pinned host buffers
    host_in = torch.from_numpy(s.get_state()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_state(host_in)
        s.step(dt, 1)
        s.get_state(out=host_out)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    prof = s.profile_stage(3)
    variants = {"visc": s.sweep_variant(0), "eta": s.sweep_variant(1), "zeta": s.sweep_variant(2)}
    s.close()
    return dict(value=value, ms=ms, launches=launches, clocks=clk, class_fraction=[float(x) for x in frac],
                e2e=job_throughput(world, N, args.steps, e2e_s), prof=prof, U1=U1, variants=variants)


def run_ensemble(args, world):
    """Batched ensemble: 48 periodic isotropic-turbulence blocks with dims
    drawn from {32,48,64,96,128} per axis and Mt in [0.3, 0.7], FP32 bulk /
    FP64 state, one persistent launch per kernel kind per stage."""
    import torch
    from paper_2209_15333_gb300 import cases
    from paper_2209_15333_gb300.solver import BatchSolver
    blocks = cases.ensemble_blocks(48, SEED)
    nodes = sum(int(np.prod(b["shape"])) for b in blocks)
    params = [dict(gamma=GAMMA, Re=b["Re"], Ma=b["Mt"], Pr=0.72, visc_law=1, visc_omega=0.76, scheme=3,
                   theta1=0.02, theta2=0.1, visc_order=8, precision=1) for b in blocks]
    stream = torch.cuda.Stream()
    bs = BatchSolver([b["shape"] for b in blocks], [b["metrics"] for b in blocks], params, stream=stream)
    for i, b in enumerate(blocks):
        bs.set_state(b["U"], block=i)
    dt = min(bs.cfl_dt(0.5, block=i) for i in range(len(blocks)))
    for _ in range(args.warmup):
        bs.step(dt, 1)
    bs.sync(600.0)
    l0 = bs.launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bs.step(dt, args.steps)
    e1.record(stream)
    bs.sync(600.0)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    launches = bs.launches() - l0
    prof = bs.profile_stage(3)
    bs.close()
    names = {"sweep_xi": "sweep_xi", "sweep_eta": "sweep_eta", "sweep_zeta": "sweep_zeta"}
    return {"workload": "48 periodic isotropic-turbulence blocks, dims i.i.d. from {32,48,64,96,128}, "
                        "Mt in [0.3,0.7], hybrid, viscous, FP32 bulk / FP64 state",
            "nodes": nodes, "value": job_throughput(world, nodes, args.steps, ms * 1e-3), "unit": "point-stage/s",
            "ms_per_step": ms / args.steps, "gpu_launches": launches,
            "launches_per_step": launches / max(1, args.steps), "kernel_ms": prof}


def roofline(prec, r, N, peaks, fma, src_hash):
    prof = r["prof"]
    dom = max(prof, key=prof.get)
    tr = NCU_TRAFFIC[prec]
    traffic = None
    ran = {"visc_flux": r["variants"]["visc"], "sweep_eta": r["variants"]["eta"],
           "sweep_zeta": r["variants"]["zeta"]}.get(dom)
    if (tr["src"] and tr["src"] == src_hash and dom in tr["per_node"]
            and (tr["variant"][dom] is None or list(tr["variant"][dom]) == list(ran))):
        traffic = tr["per_node"][dom] * N
    if prec == "fp64":
        achieved = FP64_FLOPS[dom] * N / (prof[dom] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fma["fp64"], "unit": "TFLOP/s",
                "frac": achieved / fma["fp64"], "traffic": traffic,
                "peak_source": "FP64 FMA throughput measured in this run (cfd_fma_peak)", "kernel_ms": prof}
    achieved = MIXED_BYTES[dom] * N / (prof[dom] * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "kernel_ms": prof}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    torch.cuda.set_device(local)
    from paper_2209_15333_gb300 import build
    build.build()
    from paper_2209_15333_gb300.solver import Solver

    n = args.n
    N = n ** 3
    U, met, params, Re = workload_params(n)
    with Solver((n, n, n), met, **params) as s0:
        s0.set_state(U)
        dt = s0.cfl_dt(0.5)
    precs = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    res = {p: run_precision(args, p, U, met, params, world, local, dt) for p in precs}
    if args.profile_only:
        return
    ens = None if args.no_ensemble else run_ensemble(args, world)
    fma = fma_peaks()
    peaks, peak_kind = measured_peaks()
    src_hash = kernel_src_hash()
    cpu, U1o = None, None
    if rank == 0 and not args.no_cpu_baseline:
        U1o, el, th = oracle_step(n, U, dt)
        cpu = {"value": N * 3 / el, "unit": "point-stage/s", "cores": th, "kind": "oracle",
               "sample": "one RK3 step (3 stages) of the full %d^3 field, %.1f s" % (n, el)}
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    alg_b = (40 + 26.7 + 40)

    def summary(p):
        r = res[p]
        d = {"value": r["value"], "unit": "point-stage/s", "ms_per_step": r["ms"] / args.steps,
             "dtype": "f32+f64" if p == "mixed" else "f64",
             "roofline": roofline(p, r, N, peaks, fma, src_hash),
             "hbm_algorithmic": {"bytes_per_point_stage": alg_b,
                                 "frac": alg_b * r["value"] / world / 1e9 / peaks["hbm_gbs"]},
             "err_vs_oracle_1step": field_rel_err(r["U1"], U1o) if U1o is not None else None,
             "class_fraction": r["class_fraction"], "gpu_launches": r["launches"], "clocks": r["clocks"],
             "e2e": r["e2e"], "kernel_variants": r["variants"]}
        if p == "fp64":
            d["fp64_alu_frac_whole_step"] = sum(FP64_FLOPS.values()) * r["value"] / world / 1e12 / fma["fp64"]
        return d

    head = "mixed" if "mixed" in res else precs[0]
    h = summary(head)
    line = {
        "metric": "grid-point stage updates/s", "value": h["value"], "unit": "point-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": h["dtype"], "data": "synthetic",
        "config": arm_config(n, Re, world, "FP32 bulk / FP64 state" if head == "mixed" else "FP64"),
        "clocks": h["clocks"],
        "e2e": {"value": h["e2e"], "unit": "point-stage/s", "h2d_bytes_per_step": 40 * N, "d2h_bytes_per_step": 40 * N},
        "gpu_launches": h["gpu_launches"],
        "roofline": h["roofline"],
        "hbm_algorithmic": dict(h["hbm_algorithmic"], peak_gbs=peaks["hbm_gbs"], peak_source=peak_kind),
        "err_vs_oracle_1step": h["err_vs_oracle_1step"],
        "class_fraction": h["class_fraction"],
        "kernel_variants": h["kernel_variants"],
        "fma_peak_tflops": fma,
        "kernel_src": src_hash,
        "cpu_baseline": cpu,
    }
    if head == "mixed" and "fp64" in res:
        line["fp64"] = summary("fp64")
    if ens is not None:
        line["ensemble"] = ens
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
