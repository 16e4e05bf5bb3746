"""Benchmark: grid-point stage updates per second of the TVD-RK3 step through
the C ABI of the CUDA library, on one GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--forms fp64,mixed,mixed_learned] [--n 256] [--no-ramp] [--no-ensemble]

Workloads (seeded, synthetic):
  * headline: decaying isotropic turbulence on a 256^3 periodic box (hybrid
    UD7/WENO7/WENO5, 8th-order viscous terms).  The headline `value` is the
    plain FP64 form (the paper's arithmetic); the FP32-bulk / FP64-state form
    with the plain sensor ("mixed") and with the learned sensor
    ("mixed_learned") are reported beside it, each with its error against the
    FP64 oracle after one RK3 step of the full field.
  * "ramp": the Mach 2.9, 24 degree compression ramp on its 1024 x 256 x 128
    body-fitted grid from its initial field (corner shock present, so WENO
    classes occur), all three forms, with the class fractions, the mixed
    forms' state and wall-quantity differences from the FP64 form, and the
    learned sensor's fallback and misclassification rates.
  * "ensemble": 48 uneven periodic blocks in persistent launches.
Rank 0 prints one JSON line.  The path exchanges no data between ranks
(independent boxes), so N > 1 runs replicas with a barrier and max-over-ranks
timing (weak scaling).
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
FORMS = {"fp64": dict(precision=0, learned=False), "mixed": dict(precision=1, learned=False),
         "mixed_learned": dict(precision=1, learned=True)}
# the learned sensor's classifier (cfd_get_sweep_variant, dir 4)
CLASSIFIERS = {0: "mma.sync", 1: "tcgen05"}

# Algorithmic work per node of each kernel, counted from the method's
# operations (FMA = 2 flops; division, square root, power = 1):
FP64_FLOPS = {"prim": 25, "sensor": 20, "visc_flux": 305, "sweep_xi": 247, "sweep_eta": 252, "sweep_zeta": 277}
# compulsory bytes per node of each kernel in the FP32-bulk form (inputs read
# once, outputs written once), in the form cfd_profile_stage times them: the
# zeta sweep with the right-hand-side epilogue (P, class, Fv, R in; L out in
# FP64); the learned sensor reads p and rho and writes the class
MIXED_BYTES = {"prim": 69, "sensor": 5, "visc_flux": 64, "sweep_xi": 57, "sweep_eta": 77, "sweep_zeta": 97}
MIXED_BYTES_LEARNED_SENSOR = 9
# What one point-stage must move through HBM whatever the kernel design: read
# the stage state (40 B), read U^n in stages 2-3 (26.7 B on average), write
# the new state (40 B); metrics are constant on the uniform box.
ALG_BYTES_PER_POINT_STAGE = 40.0 + 80.0 / 3.0 + 40.0
# DRAM bytes per launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the full 256^3 workload ("nodes"), one launch of
# each kernel per variant (dir:kind:param as cfd_get_sweep_variant reports
# it; the RHS epilogue for zeta, as cfd_profile_stage runs it); valid only
# for the kernel sources with hash prefix "src".
NCU_TRAFFIC = {
    "src": "b647d8123341", "nodes": 256 ** 3,
    "fp64": {"prim": [{"variant": None, "bytes_per_launch": 1554652672}],
             "sensor": [{"variant": None, "bytes_per_launch": 145433856}],
             "visc_flux": [{"variant": [0, 0], "bytes_per_launch": 2157005056}],
             "sweep_xi": [{"variant": [1, 0], "bytes_per_launch": 1863278336}],
             "sweep_eta": [{"variant": [2, 0], "bytes_per_launch": 2574391040}],
             "sweep_zeta": [{"variant": [2, 64], "bytes_per_launch": 2696522496}]},
    # FP32 bulk, plain sensor: the node-parallel (0) and tiled (3) viscous
    # kernels also form the sensor's classes (no sensor launch of its own)
    "mixed": {"prim": [{"variant": None, "bytes_per_launch": 1111171072}],
              "visc_flux": [{"variant": [0, 0], "bytes_per_launch": 1114907392},
                            {"variant": [3, 0], "bytes_per_launch": 1122263808}],
              "sweep_xi": [{"variant": [0, 0], "bytes_per_launch": 923300864}],
              "sweep_eta": [{"variant": [1, 16], "bytes_per_launch": 1390976768}],
              "sweep_zeta": [{"variant": [1, 16], "bytes_per_launch": 1883188224}]},
    # learned sensor (tcgen05 classifier) and the viscous tiles without the
    # plain sensor; the sweeps are those of "mixed"
    "mixed_learned": {"sensor": [{"variant": None, "bytes_per_launch": 149448448}],
                      "visc_flux": [{"variant": [3, 0], "bytes_per_launch": 1029302784}]},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--forms", default="fp64,mixed,mixed_learned")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="one profiled stage and one step per form (ncu runs)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 48-block ensemble measurement")
    ap.add_argument("--no-ramp", action="store_true", help="skip the Mach 2.9 ramp workload")
    ap.add_argument("--ramp-scale", type=int, default=1, help="divide the ramp grid by this factor")
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
    """Hash of the CUDA sources with their comments removed and whitespace
    runs collapsed (a comment or layout edit does not change a kernel, so it
    leaves recorded ncu figures valid)."""
    import re
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2209_15333_gb300", "csrc"))):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(ROOT, "paper_2209_15333_gb300", "csrc", f), encoding="utf-8") as fh:
                text = fh.read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(" ".join(text.split()).encode("utf-8"))
    return h.hexdigest()[:12]


def field_rel_err(a, b):
    e = 0.0
    for q in range(a.shape[0]):
        den = float(np.abs(b[q]).max())
        num = float(np.abs(a[q] - b[q]).max())
        e = max(e, num / den if den > 0 else num)
    return e


def state_rel_err(a, b):
    """Largest difference of two states relative to the field's scale:
    density and energy against their own maxima, each momentum component
    against the largest momentum magnitude (a component that vanishes in the
    reference, like the spanwise momentum of a two-dimensional flow, is not
    its own scale)."""
    mom = float(np.sqrt(np.sum(b[1:4] ** 2, axis=0)).max())
    e = 0.0
    for q in range(5):
        den = mom if 1 <= q <= 3 else float(np.abs(b[q]).max())
        e = max(e, float(np.abs(a[q] - b[q]).max()) / den)
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
    """The workload both arms report."""
    N = n ** 3
    return {"workload": "decaying isotropic turbulence %d^3 periodic, hybrid UD7/WENO7/WENO5, 8th-order "
                        "viscous" % n,
            "grid": [n, n, n], "Re": Re, "Mt": MT, "seed": SEED,
            "l2": "inputs larger than L2 (state %d MB)" % (40 * N // 2 ** 20),
            "parallelism": "replicas" if world > 1 else "single GPU", "precision": precision}


def run_reference(args, rank):
    """Reference arm: the CPU oracle on the host cores (rank 0 only), one
    RK3 step of the full n^3 field per timed step."""
    if rank != 0:
        return
    n = args.n
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
        "config": arm_config(n, Re, args.gpus, "FP64"),
        "cpu_baseline": {"value": value, "unit": "point-stage/s", "cores": th, "kind": "oracle",
                         "sample": "one RK3 step of the full %d^3 field per timed step" % n},
        "e2e": {"value": value, "unit": "point-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def set_learned_sensor(s):
    from paper_2209_15333_gb300.train_sensor import load
    W, conf, _ = load()
    s.set_sensor_mlp(W["w1"], W["w2"], W["w3"], W["b1"], W["b2"], W["b3"], conf_min=conf)


def timed_steps(s, stream, dt, steps, world):
    """CUDA-event milliseconds of `steps` graph-replayed steps on the
    context stream (slowest rank), and the launches they issued."""
    import torch
    l0 = s.launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(dt, steps)
    e1.record(stream)
    s.sync(600.0)
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1), world), s.launches() - l0


def run_form(args, form, U, met, params, world, local, dt):
    """Time K graph-replayed steps of one form on the 256^3 box."""
    import torch
    from paper_2209_15333_gb300.solver import Solver
    n = args.n
    N = n ** 3
    stream = torch.cuda.Stream()
    s = Solver((n, n, n), met, stream=stream, precision=FORMS[form]["precision"], **params)
    if FORMS[form]["learned"]:
        set_learned_sensor(s)
    Ud = torch.tensor(U, device="cuda")
    s.set_state(Ud)
    for item in filter(None, args.variants.split(",")):
        f = [int(x) for x in item.split(":")]
        s.set_sweep_variant(f[0], f[1], f[2] if len(f) > 2 else 0)
    if args.profile_only:
        s.profile_stage(1)   # one right-hand side, kernel by kernel
        s.step(dt, 1)        # one RK3 step (the update epilogues)
        s.sync(600.0)
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
    if FORMS[form]["learned"]:
        s.sensor_fallbacks()  # reset the counter
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = timed_steps(s, stream, dt, args.steps, world)
    clk = clocks.stop()
    fallbacks = s.sensor_fallbacks() if FORMS[form]["learned"] else None
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
    variants = {"visc": s.sweep_variant(0), "xi": s.sweep_variant(3), "eta": s.sweep_variant(1),
                "zeta": s.sweep_variant(2)}
    if FORMS[form]["learned"]:
        variants["classifier"] = CLASSIFIERS[s.sweep_variant(4)[0]]
    s.close()
    r = dict(value=value, ms=ms, launches=launches, clocks=clk, class_fraction=[float(x) for x in frac],
             e2e=job_throughput(world, N, args.steps, e2e_s), prof=prof, U1=U1, variants=variants)
    if fallbacks is not None:
        r["fallback_fraction"] = fallbacks / (3.0 * args.steps * N)
    return r


def run_ramp(args, world):
    """Mach 2.9, 24 degree ramp (1024 x 256 x 128) from its initial field:
    K timed steps of each form at a fixed dt (CFL 0.3 on the initial field)."""
    import torch
    from paper_2209_15333_gb300 import ramp
    c = ramp.CASES[4]
    nx, ny, nz = ramp.case_shape(4, args.ramp_scale)
    N = nx * ny * nz
    out = {"workload": "Mach 2.9, 24 deg compression ramp %dx%dx%d, hybrid, Sutherland, Re_delta 20000, "
                       "isothermal wall with blowing strip, from the initial field" % (nx, ny, nz),
           "grid": [nx, ny, nz], "nodes": N, "unit": "point-stage/s"}
    states, flags, rc, dt = {}, {}, None, None
    for form in [f for f in ("fp64", "mixed", "mixed_learned") if f in args.forms.split(",")]:
        stream = torch.cuda.Stream()
        s, rc = ramp.run(4, FORMS[form]["precision"], FORMS[form]["learned"], 0, 1, scale=args.ramp_scale,
                         stream=stream)
        if dt is None:
            dt = s.cfl_dt(0.3)
        for _ in range(args.warmup):
            s.step(dt, 1)
        s.sync(600.0)
        if FORMS[form]["learned"]:
            s.sensor_fallbacks()
        t0 = time.perf_counter()
        ms, launches = timed_steps(s, stream, dt, args.steps, world)
        wall = time.perf_counter() - t0
        rec = {"value": job_throughput(world, N, args.steps, ms * 1e-3), "ms_per_step": ms / args.steps,
               "gpu_launches": launches, "host_wall_s": wall}
        if FORMS[form]["learned"]:
            rec["fallback_fraction"] = s.sensor_fallbacks() / (3.0 * args.steps * N)
        U = s.get_state()
        states[form] = U
        # classes of the final state's evaluation, plus (learned) the plain
        # sensor's classes of the same state for the misclassification rate
        s.rhs(np.empty_like(U))
        g = s.flags()
        flags[form] = g
        rec["class_fraction"] = (np.bincount(g.ravel(), minlength=3)[:3] / g.size).tolist()
        if FORMS[form]["learned"]:
            s.set_sensor_mlp(None, None, None, None, None, None)
            s.rhs(np.empty_like(U))
            p = s.flags()
            rec["misclassification"] = float((g != p).mean())
            rec["unsafe_rate"] = float((g < p).mean())
        pw, cf = ramp.wall_quantities(U, rc["metrics2d"], c["Ma"], c["Tw"], c["T_ref"])
        rec["_pw"], rec["_cf"] = pw, cf
        s.close()
        out[form] = rec
    if "fp64" in out:
        base = out["fp64"]
        for form in ("mixed", "mixed_learned"):
            if form not in out:
                continue
            r = out[form]
            r["speedup_vs_fp64"] = r["value"] / base["value"]
            r["state_rel_err_vs_fp64"] = state_rel_err(states[form], states["fp64"])
            r["pw_rel_l2_err_vs_fp64"] = float(np.linalg.norm(r["_pw"] - base["_pw"]) / np.linalg.norm(base["_pw"]))
            r["cf_rel_l2_err_vs_fp64"] = float(np.linalg.norm(r["_cf"] - base["_cf"]) / np.linalg.norm(base["_cf"]))
    for r in out.values():
        if isinstance(r, dict):
            r.pop("_pw", None)
            r.pop("_cf", None)
    out["dt"] = dt
    out["steps_from_initial_field"] = args.warmup + args.steps
    return out


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
    ms, launches = timed_steps(bs, stream, dt, args.steps, world)
    prof = bs.profile_stage(3)
    variants = bs.batch_variants() if hasattr(bs, "batch_variants") else None
    # the same ensemble with the learned sensor (one batched launch per stage)
    set_learned_sensor(bs)
    for _ in range(args.warmup):
        bs.step(dt, 1)
    bs.sync(600.0)
    bs.sensor_fallbacks()  # reset the counter
    ms_l, launches_l = timed_steps(bs, stream, dt, args.steps, world)
    learned = {"value": job_throughput(world, nodes, args.steps, ms_l * 1e-3), "unit": "point-stage/s",
               "ms_per_step": ms_l / args.steps, "gpu_launches": launches_l,
               "fallback_fraction": bs.sensor_fallbacks() / (3.0 * args.steps * nodes),
               "kernel_ms": bs.profile_stage(3), "classifier": CLASSIFIERS[bs.sweep_variant(4)[0]]}
    bs.close()
    return {"workload": "48 periodic isotropic-turbulence blocks, dims i.i.d. from {32,48,64,96,128}, "
                        "Mt in [0.3,0.7], hybrid, viscous, FP32 bulk / FP64 state",
            "nodes": nodes, "value": job_throughput(world, nodes, args.steps, ms * 1e-3), "unit": "point-stage/s",
            "ms_per_step": ms / args.steps, "gpu_launches": launches,
            "launches_per_step": launches / max(1, args.steps), "kernel_ms": prof, "kernel_variants": variants,
            "learned_sensor": learned}


def kernel_traffic(form, dom, variant, N, src_hash):
    """ncu DRAM bytes of one launch of kernel `dom` in the variant that ran,
    scaled from the captured workload's nodes to N; None when the capture is
    of other kernel sources or another variant."""
    tr = NCU_TRAFFIC
    if not tr["src"] or tr["src"] != src_hash:
        return None
    recs = tr.get(form, {}).get(dom) or tr.get("mixed" if form.startswith("mixed") else form, {}).get(dom, [])
    for rec in recs:
        if rec.get("variant") is None or variant is None or list(rec["variant"]) == list(variant):
            return rec["bytes_per_launch"] * N / tr["nodes"]
    return None


def rooflines(form, r, N, peaks, fma, src_hash, world):
    """Dominant-kernel roofline (CUDA-event time of one launch per stage) and
    the whole-stage algorithmic fractions."""
    prof = r["prof"]
    dom = max(prof, key=prof.get)
    ran = {"visc_flux": r["variants"]["visc"], "sweep_xi": r["variants"]["xi"], "sweep_eta": r["variants"]["eta"],
           "sweep_zeta": r["variants"]["zeta"]}.get(dom)
    traffic = kernel_traffic(form, dom, ran, N, src_hash)
    per_gpu = r["value"] / world
    stage = {"hbm_bytes_per_point_stage": ALG_BYTES_PER_POINT_STAGE,
             "hbm_achieved_gbs": ALG_BYTES_PER_POINT_STAGE * per_gpu / 1e9,
             "hbm_peak_gbs": peaks["hbm_gbs"],
             "hbm_frac": ALG_BYTES_PER_POINT_STAGE * per_gpu / 1e9 / peaks["hbm_gbs"]}
    if form == "fp64":
        flops = sum(FP64_FLOPS.values())
        stage.update(fp64_flops_per_point_stage=flops, fp64_achieved_tflops=flops * per_gpu / 1e12,
                     fp64_peak_tflops=fma["fp64"], fp64_frac=flops * per_gpu / 1e12 / fma["fp64"])
        achieved = FP64_FLOPS[dom] * N / (prof[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fma["fp64"], "unit": "TFLOP/s",
                "frac": achieved / fma["fp64"], "traffic": traffic,
                "peak_source": "FP64 FMA throughput measured in this run (cfd_fma_peak; nominal 1.25 TFLOP/s)",
                "algorithmic_per_node": FP64_FLOPS[dom], "kernel_ms": prof}
    else:
        achieved = ALG_BYTES_PER_POINT_STAGE * N / (sum(prof.values()) * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "whole stage", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "traffic_kernel": dom,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "algorithmic_per_node": ALG_BYTES_PER_POINT_STAGE, "kernel_ms": prof}
        cb = MIXED_BYTES_LEARNED_SENSOR if (form == "mixed_learned" and dom == "sensor") else MIXED_BYTES[dom]
        if form == "mixed" and dom == "visc_flux" and r["variants"]["visc"][0] in (0, 3):
            cb += MIXED_BYTES["sensor"]  # the node-flux kernels also form the plain sensor's classes
        kc = cb * N / (prof[dom] * 1e-3) / 1e9
        roof["kernel_compulsory"] = {"kernel": dom, "bytes_per_node": cb, "achieved_gbs": kc,
                                     "frac": kc / peaks["hbm_gbs"]}
    return roof, stage


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
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
    forms = [f for f in args.forms.split(",") if f]
    res = {f: run_form(args, f, U, met, params, world, local, dt) for f in forms}
    if args.profile_only:
        return
    ramp_res = None if args.no_ramp else run_ramp(args, world)
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

    def summary(f):
        r = res[f]
        roof, stage = rooflines(f, r, N, peaks, fma, src_hash, world)
        d = {"value": r["value"], "unit": "point-stage/s", "ms_per_step": r["ms"] / args.steps,
             "dtype": "f64" if f == "fp64" else "f32+f64", "roofline": roof, "stage_roofline": stage,
             "err_vs_oracle_1step": field_rel_err(r["U1"], U1o) if U1o is not None else None,
             "class_fraction": r["class_fraction"], "gpu_launches": r["launches"], "clocks": r["clocks"],
             "e2e": {"value": r["e2e"], "unit": "point-stage/s", "h2d_bytes_per_step": 40 * N,
                     "d2h_bytes_per_step": 40 * N},
             "kernel_variants": r["variants"]}
        if "fallback_fraction" in r:
            d["fallback_fraction"] = r["fallback_fraction"]
        if f != "fp64" and "fp64" in res:
            d["speedup_vs_fp64"] = r["value"] / res["fp64"]["value"]
        return d

    head = "fp64" if "fp64" in res else forms[0]
    h = summary(head)
    line = {
        "metric": "grid-point stage updates/s", "value": h["value"], "unit": "point-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": h["dtype"], "data": "synthetic",
        "config": arm_config(n, Re, world, "FP64" if head == "fp64" else "FP32 bulk / FP64 state"),
        "clocks": h["clocks"], "e2e": h["e2e"], "gpu_launches": h["gpu_launches"],
        "roofline": h["roofline"], "stage_roofline": h["stage_roofline"],
        "err_vs_oracle_1step": h["err_vs_oracle_1step"], "class_fraction": h["class_fraction"],
        "kernel_variants": h["kernel_variants"], "fma_peak_tflops": fma, "hbm_peak": {"gbs": peaks["hbm_gbs"],
                                                                                     "source": peak_kind},
        "kernel_src": src_hash, "cpu_baseline": cpu,
    }
    for f in forms:
        if f != head:
            line[f] = summary(f)
    if ramp_res is not None:
        line["ramp"] = ramp_res
    if ens is not None:
        line["ensemble"] = ens
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
