"""Shared set-up for the GPU tests: one case description drives both the CUDA
library (through the C ABI) and the CPU oracle."""
import math

import numpy as np

from paper_2209_15333_gb300 import cases

SCHEMES = {"UD7": 0, "WENO5": 1, "WENO7": 2, "HYBRID": 3}


def field_rel_err(a, b):
    """max_q max|a_q - b_q| / max|b_q| over the 5 conserved fields (field-max
    normalisation; components that vanish identically compare absolutely)."""
    errs = []
    for q in range(a.shape[0]):
        den = np.abs(b[q]).max()
        num = np.abs(a[q] - b[q]).max()
        errs.append(num / den if den > 0 else num)
    return max(errs)


def make_pair(orc, shape, metrics, *, scheme="UD7", Re=0.0, Ma=0.5, gamma=1.4, Pr=0.72, T_wall=1.0, T_ref=288.15,
              visc_law=1, visc_omega=0.76, theta1=0.02, theta2=0.1, visc_order=8, bc_lo=(0, 0, 0),
              bc_hi=(0, 0, 0), inflow=None, blowing=None):
    """Return (solver, oracle case, full 3-D metrics for the oracle)."""
    from paper_2209_15333_gb300.solver import Solver
    nx, ny, nz = shape
    sch = SCHEMES[scheme]
    s = Solver(shape, metrics, bc_lo=bc_lo, bc_hi=bc_hi, gamma=gamma, Re=Re, Ma=Ma, Pr=Pr, T_wall=T_wall,
               T_ref=T_ref, visc_law=visc_law, visc_omega=visc_omega, scheme=sch, theta1=theta1, theta2=theta2,
               visc_order=visc_order)
    if inflow is not None:
        s.set_inflow(inflow)
    if blowing is not None:
        s.set_blowing(blowing["amp"], blowing["x0"], blowing["x1"], blowing["omega"], blowing["m"], blowing["Lz"],
                      blowing["wall_x"], blowing["wall_z"])
    c = orc.Case(nx, ny, nz, gamma=gamma, Re=Re, Ma=Ma, Pr=Pr, T_wall=T_wall, T_ref=T_ref, visc_law=visc_law,
                 visc_omega=visc_omega, scheme=sch, theta1=theta1, theta2=theta2, visc_order=visc_order,
                 bc_lo=bc_lo, bc_hi=bc_hi, inflow=inflow, blowing=blowing)
    M = cases.expand_metrics(metrics, (nz, ny, nx))
    return s, c, M


def turbulence_field(shape, seed, Mt=0.5, amp=1.0):
    """Seeded smooth random periodic field on a non-cubic box (for parity)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    X, Y, Z = cases.box_coords(nx, ny, nz)
    vel = []
    for _ in range(3):
        f = np.zeros_like(X)
        for _ in range(6):
            kx, ky, kz = rng.integers(-3, 4, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            f += rng.normal() * np.cos(kx * X + ky * Y + kz * Z + ph)
        vel.append(amp * f / 6.0)
    T = 1.0 + 0.1 * np.cos(X + 2 * Y - Z)
    p = (1.0 + 0.2 * np.sin(2 * X - Y) * np.cos(Z)) / (1.4 * Mt * Mt)
    rho = 1.4 * Mt * Mt * p / T
    return cases.conserved(rho, vel[0], vel[1], vel[2], p, 1.4)
