"""Pins of the viscous central differences and their closures (Section 2.3,
reading R11), of the TVD-RK3 update (Eq. 45), the sensor (Eqs. 42-43) and
the wall boundary condition (reading R12)."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("order", [6, 8])
def test_interior_central_polynomial_exactness(orc, order):
    n = 24
    x = np.arange(n, dtype=float) * 0.37 - 3.0
    for deg in range(order + 2):
        g = x ** deg
        dg = orc.central_deriv(order, g, periodic=False)
        exact = deg * x ** (deg - 1) if deg else np.zeros(n)
        scale = 1.0 + np.abs(g).max()
        inner = slice(4, n - 4) if order == 8 else slice(3, n - 3)
        err = np.abs(dg[inner] / 0.37 * 0.37 - exact[inner] * 0.37)
        # index-space derivative: d/di = 0.37 d/dx
        err = np.abs(dg[inner] - 0.37 * exact[inner])
        if deg <= order:
            assert err.max() <= 1e-11 * scale, deg
        else:
            assert err.max() > 1e-8 * scale


def test_closure_orders(orc):
    """Node 0: one-sided 2nd order; nodes 1, 2, 3: central 2nd, 4th, 6th."""
    n = 20
    x = np.arange(n, dtype=float)
    exact_degree = {0: 2, 1: 2, 2: 4, 3: 6}
    for node, deg_ok in exact_degree.items():
        for deg in range(deg_ok + 2):
            g = (x - 5.5) ** deg
            ex = deg * (x - 5.5) ** (deg - 1) if deg else np.zeros(n)
            for order in (6, 8):
                dg = orc.central_deriv(order, g, periodic=False)
                scale = 1.0 + np.abs(g[:10]).max()
                e_lo = abs(dg[node] - ex[node])
                e_hi = abs(dg[n - 1 - node] - ex[n - 1 - node])
                if deg <= deg_ok:
                    assert e_lo <= 1e-11 * scale and e_hi <= 1e-11 * scale, (node, deg)
                else:
                    assert e_lo > 1e-9 or e_hi > 1e-9


@pytest.mark.parametrize("order", [6, 8])
def test_periodic_central_order(orc, order):
    errs = []
    for n in (16, 32):
        h = 2 * math.pi / n
        x = np.arange(n) * h
        dg = orc.central_deriv(order, np.sin(x), periodic=True) / h
        errs.append(np.abs(dg - np.cos(x)).max())
    rate = math.log(errs[0] / errs[1], 2)
    assert rate > order - 0.3


def test_rk3_amplification(orc):
    """Eq. 45 applied to dU/dt = z U gives 1 + z + z^2/2 + z^3/6 exactly."""
    rng = np.random.default_rng(3)
    z = rng.uniform(-2.0, 0.5, size=64)
    dt = 1.0
    Un = np.ones(64)
    U1 = orc.rk3_stage(1, Un, Un, z * Un, dt)
    U2 = orc.rk3_stage(2, Un, U1, z * U1, dt)
    U3 = orc.rk3_stage(3, Un, U2, z * U2, dt)
    assert np.allclose(U3, 1 + z + z * z / 2 + z ** 3 / 6, rtol=0, atol=1e-14)


def _const_case(orc, n, **kw):
    return orc.Case(n, n, n, Ma=0.5, **kw)


def test_sensor_hand_values(orc):
    """theta on a small field with one pressure spike, by hand."""
    from paper_2209_15333_gb300 import cases
    n = 8
    g, Ma = 1.4, 0.5
    p = np.full((n, n, n), 1.0)
    p[3, 4, 5] = 1.3           # (k, j, i)
    rho = np.ones_like(p)
    z = np.zeros_like(p)
    U = cases.conserved(rho, z, z, z, p, g)
    c = orc.Case(n, n, n, Ma=Ma, gamma=g, scheme=orc.HYBRID)
    th, cls = orc.sensor(c, U)
    phi_c = abs(-1 + 2 * 1.3 - 1) / (1 + 2 * 1.3 + 1)       # at the spike, each direction
    phi_n = abs(-1 + 2 * 1 - 1.3) / (1 + 2 * 1 + 1.3)       # at a neighbour, along one direction
    assert abs(th[3, 4, 5] - 3 * phi_c) <= 1e-15
    for (k, j, i) in [(3, 4, 4), (3, 4, 6), (3, 3, 5), (3, 5, 5), (2, 4, 5), (4, 4, 5)]:
        assert abs(th[k, j, i] - phi_n) <= 1e-15
    assert th[0, 0, 0] == 0.0
    assert cls[3, 4, 5] == 2                      # 0.6 > 0.1
    assert cls[3, 4, 4] == 1                      # 0.0698 in (0.02, 0.1]
    assert cls[0, 0, 0] == 0
    # boundary nodes of non-periodic directions take phi = 0 in that direction
    c2 = orc.Case(n, n, n, Ma=Ma, gamma=g, scheme=orc.HYBRID, bc_lo=(3, 0, 0), bc_hi=(3, 0, 0))
    p2 = np.ones((n, n, n)) + 0.1 * np.arange(n)[None, None, :] ** 2
    U2 = cases.conserved(rho, z, z, z, p2, g)
    th2, _ = orc.sensor(c2, U2)
    assert np.all(th2[:, :, 0] == 0.0) and np.all(th2[:, :, -1] == 0.0)
    i = 3
    ref = abs(-p2[0, 0, i - 1] + 2 * p2[0, 0, i] - p2[0, 0, i + 1]) / (p2[0, 0, i - 1] + 2 * p2[0, 0, i] + p2[0, 0, i + 1])
    assert abs(th2[0, 0, i] - ref) <= 1e-15


def test_sensor_zero_on_linear_pressure(orc):
    from paper_2209_15333_gb300 import cases
    n = 10
    p = 1.0 + 0.05 * np.arange(n)[None, None, :] + 0.03 * np.arange(n)[None, :, None] + 0.0 * np.zeros((n, n, n))
    rho = np.ones((n, n, n))
    z = np.zeros_like(rho)
    U = cases.conserved(rho, z, z, z, p, 1.4)
    c = orc.Case(n, n, n, Ma=0.5, scheme=orc.HYBRID, bc_lo=(3, 3, 0), bc_hi=(3, 3, 0))
    th, cls = orc.sensor(c, U)
    assert np.abs(th).max() <= 1e-15
    assert np.all(cls == 0)


def test_wall_pressure_extrapolation(orc):
    """p_w = (4 p1 - p2)/3 is exact for p = a + b y^2 (zero wall gradient)."""
    from paper_2209_15333_gb300 import cases
    nx, ny, nz = 8, 10, 4
    g, Ma, Tw = 1.4, 0.8, 2.5
    y = np.arange(ny, dtype=float)
    p = (2.0 + 0.01 * y ** 2)[None, :, None] * np.ones((nz, ny, nx))
    rho = np.ones_like(p) * 1.2
    u = np.ones_like(p) * 0.3
    z = np.zeros_like(p)
    U = cases.conserved(rho, u, z, z, p, g)
    met = cases.expand_metrics(cases.uniform_metrics(nx, ny, nz, 1.0, 1.0, 1.0), (nz, ny, nx))
    c = orc.Case(nx, ny, nz, gamma=g, Ma=Ma, T_wall=Tw, bc_lo=(0, 1, 0), bc_hi=(0, 3, 0))
    Ub = orc.apply_bc(c, met, U)
    prim = orc.primitives(c, Ub)
    assert np.allclose(prim[4, :, 0, :], 2.0, rtol=1e-13)
    assert np.allclose(prim[5, :, 0, :], Tw, rtol=1e-13)
    assert np.abs(prim[1:4, :, 0, :]).max() <= 1e-15
    # extrapolation face copies the neighbour
    assert np.allclose(Ub[:, :, -1, :], U[:, :, -2, :], rtol=1e-14)
