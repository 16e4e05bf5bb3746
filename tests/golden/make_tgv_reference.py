"""Writes tgv32_10steps.txt: summary numbers of the oracle's state after 10
RK3 steps of the Taylor-Green case (32^3, Ma 0.5, Re 400, power law, UD7,
CFL 0.5), a regression fixture of the oracle itself.  Calls the oracle only.

    python tests/golden/make_tgv_reference.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as orc  # noqa: E402
from paper_2209_15333_gb300 import cases  # noqa: E402


def summary():
    n = 32
    U = cases.taylor_green(n, Ma=0.5)
    M = cases.expand_metrics(cases.uniform_metrics(n, n, n), (n, n, n))
    c = orc.Case(n, n, n, Re=400.0, Ma=0.5, scheme=orc.UD7, visc_law=orc.POWER, visc_omega=0.76)
    dt = orc.cfl_dt(c, M, U, 0.5)
    V = orc.step(c, M, U, dt, 10)
    rows = [("dt", dt)]
    for q in range(5):
        rows.append(("sum_%d" % q, float(V[q].sum())))
        rows.append(("max_%d" % q, float(np.abs(V[q]).max())))
        rows.append(("l2_%d" % q, float(np.sqrt((V[q] ** 2).mean()))))
    return rows


if __name__ == "__main__":
    with open(os.path.join(HERE, "tgv32_10steps.txt"), "w") as f:
        f.write("# Oracle state after 10 RK3 steps of the 32^3 Taylor-Green case (Ma 0.5, Re 400,\n"
                "# power law 0.76, UD7, CFL 0.5): written by make_tgv_reference.py (oracle only).\n")
        for k, v in summary():
            f.write("%s %.17g\n" % (k, v))
