"""Runs a few cases through whichever CUDA library CFD_GB300_LIB names and
saves L(U) and the state after three steps (used by test_gpu_checked.py to
run the bounds-checked build in a process of its own)."""
import sys

import numpy as np

from paper_2209_15333_gb300 import cases
from paper_2209_15333_gb300.solver import Solver

from gpu_helpers import turbulence_field


def case_list():
    out = []
    sh = (37, 19, 23)
    out.append(("ragged_hybrid", sh, cases.uniform_metrics(*sh), turbulence_field(sh, 81, amp=1.5),
                dict(scheme=3, Re=200.0, Ma=0.5, theta1=0.004, theta2=0.012), {}))
    n = 20
    met, _ = cases.wavy_grid(n, amp=0.05)
    out.append(("wavy_char_mixed", (n, n, n), met, turbulence_field((n, n, n), 82, amp=1.2),
                dict(scheme=3, Re=300.0, Ma=0.5, theta1=0.004, theta2=0.012, recon_vars=1, precision=1), {}))
    rc = cases.ramp_case(40, 24, 8, 24.0, 2.9, Tw=2.8)
    out.append(("ramp_walls", (40, 24, 8), rc["metrics2d"], rc["U"],
                dict(scheme=3, Re=2000.0, Ma=2.9, T_wall=2.8, visc_law=0, T_ref=108.1, theta1=0.005, theta2=0.02),
                dict(bc_lo=(2, 1, 0), bc_hi=(3, 3, 0), inflow=rc["inflow"])))
    # walking sweeps pinned (chunks of 128 xi nodes and 8 eta/zeta positions,
    # several segments per line, one non-periodic direction)
    sh = (300, 21, 26)
    out.append(("walking_segments", sh, cases.uniform_metrics(*sh), turbulence_field(sh, 83, amp=1.5),
                dict(scheme=3, Re=200.0, Ma=0.5, theta1=0.004, theta2=0.012),
                dict(bc_lo=(3, 3, 0), bc_hi=(3, 3, 0), variants=[(3, 1, 100), (1, 2, 13), (2, 2, 0)])))
    # the FP32 walking eta/zeta sweeps staged by tensor-memory-accelerator copies
    sh = (64, 21, 26)
    out.append(("tma_walk_mixed", sh, cases.uniform_metrics(*sh), turbulence_field(sh, 84, amp=1.5),
                dict(scheme=3, Re=200.0, Ma=0.5, theta1=0.004, theta2=0.012, precision=1),
                dict(bc_lo=(0, 3, 0), bc_hi=(0, 3, 0), variants=[(1, 3, 8), (2, 3, 0)])))
    return out


def main(out_path):
    res = {}
    for name, sh, met, U, prm, extra in case_list():
        inflow = extra.pop("inflow", None)
        variants = extra.pop("variants", ())
        with Solver(sh, met, **extra, **prm) as s:
            if inflow is not None:
                s.set_inflow(inflow)
            for d, kind, param in variants:
                s.set_sweep_variant(d, kind, param)
            s.set_state(U)
            res[name + "_rhs"] = s.rhs()
            s.step(s.cfl_dt(0.4), 3)
            res[name + "_U3"] = s.get_state()
            s.sync(60.0)
    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
