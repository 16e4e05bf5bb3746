"""Run in a process of its own by test_gpu_tune_cache.py: one single-block
context and one ensemble take two RK3 steps each; prints, as JSON, how many
kernels each step launched and the variants the contexts run."""
import json
import sys

from paper_2209_15333_gb300 import cases
from paper_2209_15333_gb300.solver import BatchSolver, Solver

from gpu_helpers import turbulence_field


def main():
    out = {}
    sh = (64, 48, 40)
    prm = dict(scheme=3, Re=200.0, Ma=0.5, theta1=0.004, theta2=0.012, precision=1)
    with Solver(sh, cases.uniform_metrics(*sh), **prm) as s:
        s.set_state(turbulence_field(sh, 91))
        l0 = s.launches()
        s.step(1e-3, 1)
        l1 = s.launches()
        s.step(1e-3, 1)
        l2 = s.launches()
        out["single"] = dict(first=l1 - l0, second=l2 - l1, variants=[s.sweep_variant(d) for d in range(4)])
    shapes = [(32, 48, 40), (48, 32, 64), (64, 32, 32)]
    with BatchSolver(shapes, [cases.uniform_metrics(*x) for x in shapes], [prm] * 3) as b:
        for i, x in enumerate(shapes):
            b.set_state(turbulence_field(x, 92 + i), block=i)
        l0 = b.launches()
        b.step(1e-3, 1)
        l1 = b.launches()
        b.step(1e-3, 1)
        l2 = b.launches()
        out["batch"] = dict(first=l1 - l0, second=l2 - l1, variants=b.batch_variants())
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())
