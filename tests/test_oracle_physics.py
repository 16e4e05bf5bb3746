"""Whole-RHS pins of the oracle (Sections 2.1-2.4): free-stream preservation,
conservation, design order on the isentropic vortex, the exact Riemann
solution of the Sod shock tube, the Taylor-Green kinetic-energy dissipation
rate at t = 0, and closed-form viscous diffusion of shear and heat waves."""
import math

import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

G = 1.4


def uniform_state(shape, rho=1.1, vel=(0.6, -0.3, 0.25), p=2.0):
    o = np.ones(shape)
    return cases.conserved(rho * o, vel[0] * o, vel[1] * o, vel[2] * o, p * o, G)


def flux_scale(met, U):
    """|J| times a typical inviscid flux magnitude, for relative residuals."""
    return np.abs(met[9]).max() * np.abs(met[:9]).max() / np.abs(met[9]).max() ** 0 * (
        np.abs(U).max())


@pytest.mark.parametrize("scheme", ["UD7", "WENO5", "WENO7", "HYBRID"])
def test_free_stream_cartesian_and_affine(orc, scheme):
    n = 12
    sch = getattr(orc, scheme)
    U = uniform_state((n, n, n))
    m = cases.uniform_metrics(n, n, n, 1.0, 1.3, 0.7)
    # affine (skewed) grid: constant but non-diagonal metrics
    A = np.array([[1.0, 0.3, -0.2], [0.1, 1.2, 0.25], [-0.15, 0.05, 0.9]])
    Minv = np.linalg.inv(A)  # rows: grad xi, grad eta, grad zeta
    ma = np.zeros(10)
    ma[:9] = Minv.ravel() * 8.0
    ma[9] = abs(np.linalg.det(Minv * 8.0))
    for met in (m, ma):
        M = cases.expand_metrics(met, (n, n, n))
        c = orc.Case(n, n, n, Re=300.0, Ma=0.7, scheme=sch)
        L = orc.rhs(c, M, U)
        assert np.abs(L).max() <= 1e-13 * flux_scale(M, U)


def test_free_stream_curved_grid_fsp(orc):
    """Zero RHS to round-off on uniform flow over a curved (wavy) grid in the
    free-stream-preserving metric mode; the paper's nodal form does not
    preserve it (reading R17)."""
    n = 16
    met, _ = cases.wavy_grid(n, amp=0.06)
    U = uniform_state((n, n, n))
    res = {}
    for mode in (orc.METRIC_NODAL, orc.METRIC_FSP):
        c = orc.Case(n, n, n, Re=500.0, Ma=0.6, scheme=orc.HYBRID, metric_mode=mode)
        L = orc.rhs(c, met, U)
        res[mode] = np.abs(L).max() / flux_scale(met, U)
    assert res[orc.METRIC_FSP] <= 1e-13
    assert res[orc.METRIC_NODAL] > 1e-6


@pytest.mark.parametrize("grid", ["cartesian", "wavy"])
def test_conservation_periodic(orc, grid):
    n = 16
    if grid == "cartesian":
        met = cases.expand_metrics(cases.uniform_metrics(n, n, n), (n, n, n))
        mode = orc.METRIC_NODAL
    else:
        met, _ = cases.wavy_grid(n, amp=0.05)
        mode = orc.METRIC_FSP
    U = cases.taylor_green(n, Ma=0.5)
    rng = np.random.default_rng(0)
    U = U * (1.0 + 0.02 * rng.standard_normal(U.shape))
    c = orc.Case(n, n, n, Re=200.0, Ma=0.5, scheme=orc.HYBRID, metric_mode=mode, theta1=0.002,
                 theta2=0.01)
    L, cls = orc.rhs(c, met, U, return_cls=True)
    assert (cls > 0).any()
    Jinv = 1.0 / met[9]
    tot = (Jinv * L).reshape(5, -1).sum(1)
    mag = np.abs(Jinv * L).reshape(5, -1).sum(1)
    assert np.all(np.abs(tot) <= 1e-13 * mag.max())
    dt = orc.cfl_dt(c, met, U, 0.5)
    U2 = orc.step(c, met, U, dt, 2)
    q0 = (Jinv * U).reshape(5, -1).sum(1)
    q1 = (Jinv * U2).reshape(5, -1).sum(1)
    assert np.all(np.abs(q1 - q0) <= 1e-13 * np.abs(Jinv * U).reshape(5, -1).sum(1).max())


# Steger-Warming fluxes are only Lipschitz where a split eigenvalue changes
# sign along a grid line (sonic points, u_d = +-c, and stagnation points,
# u_d = 0), and the reconstruction then loses its order there.  The design-
# order check therefore uses a vortex (strength 2.5) and a mean flow that keep
# 0 < u_d < c along both grid directions everywhere.
VORTEX_MEAN = (0.55, 0.5)
VORTEX_BETA = 2.5


def _vortex_dudt(n, nz):
    """dU/dt of the convected vortex: 4th-order difference of the exact
    solution in time."""
    d = 1e-3
    Us = [cases.isentropic_vortex(n, nz, t=t, mean=VORTEX_MEAN, beta=VORTEX_BETA)[0] for t in (-2 * d, -d, d, 2 * d)]
    return (Us[0] - 8 * Us[1] + 8 * Us[2] - Us[3]) / (12 * d)


# The WENO weights only approach the linear weights once the smoothness
# indicators (measured on the flux per unit face area) fall well below
# eps = 1e-6, so the WENO schemes reach their order on finer grids than UD7;
# at the vortex's critical points Jiang-Shu weights converge slowly, so
# WENO7 is held to order - 1.5 on its finest pair.
@pytest.mark.parametrize("scheme,order,ns,slack", [("UD7", 7, (32, 64, 128), 1.2),
                                                  ("WENO7", 7, (128, 256, 512), 1.5),
                                                  ("WENO5", 5, (128, 256, 512), 1.2)])
def test_isentropic_vortex_order(orc, scheme, order, ns, slack):
    errs = []
    for n in ns:
        U, met, Ma, _, _ = cases.isentropic_vortex(n, nz=1, mean=VORTEX_MEAN, beta=VORTEX_BETA)
        prim = orc.primitives(orc.Case(n, n, 1, Ma=Ma), U)
        assert (prim[1:3] > 0).all() and (prim[1:3] < prim[6]).all()
        M = cases.expand_metrics(met, (1, n, n))
        c = orc.Case(n, n, 1, Re=0.0, Ma=Ma, gamma=G, scheme=getattr(orc, scheme))
        L = orc.rhs(c, M, U)
        errs.append(np.abs(L - _vortex_dudt(n, 1)).max())
    rates = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert rates[-1] > order - slack, (errs, rates)


# ---- Sod shock tube against the exact Riemann solution ----

def exact_riemann(x, t, left, right, x0=0.5, g=G):
    """Exact solution of the Riemann problem (iterative star-pressure solve)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)

    def fk(p, rk, pk, ck):
        if p > pk:
            A, B = 2 / ((g + 1) * rk), (g - 1) / (g + 1) * pk
            return (p - pk) * math.sqrt(A / (p + B))
        return 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    lo, hi = 1e-8, 10 * max(pl, pr)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if fk(mid, rl, pl, cl) + fk(mid, rr, pr, cr) + ur - ul > 0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (fk(ps, rr, pr, cr) - fk(ps, rl, pl, cl))
    out = np.zeros((3, x.size))
    for i, xi in enumerate(x):
        s = (xi - x0) / t
        if s < us:
            if ps > pl:
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                S = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[:, i] = (rl, ul, pl) if s < S else (rs, us, ps)
            else:
                rs = rl * (ps / pl) ** (1 / g)
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s < ul - cl:
                    out[:, i] = (rl, ul, pl)
                elif s > us - cs:
                    out[:, i] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    r = rl * (c / cl) ** (2 / (g - 1))
                    out[:, i] = (r, u, r * c * c / g)
        else:
            if ps > pr:
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                S = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[:, i] = (rr, ur, pr) if s > S else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1 / g)
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s > ur + cr:
                    out[:, i] = (rr, ur, pr)
                elif s < us + cs:
                    out[:, i] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    r = rr * (c / cr) ** (2 / (g - 1))
                    out[:, i] = (r, u, r * c * c / g)
    return out, ps, us


def test_exact_riemann_star_state():
    """Sanity of the test's own solver on Sod's problem (Toro, Table 4.2)."""
    _, ps, us = exact_riemann(np.array([0.5]), 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - 0.30313) < 1e-4 and abs(us - 0.92745) < 1e-4


@pytest.mark.parametrize("scheme", ["WENO5", "HYBRID"])
def test_sod_against_exact(orc, scheme):
    errs = []
    t_end = 0.2
    ns = (101, 201, 401)
    for n in ns:
        U, met, Ma, x = cases.shock_tube(n)
        M = cases.expand_metrics(met, (1, 1, n))
        c = orc.Case(n, 1, 1, Re=0.0, Ma=Ma, gamma=G, scheme=getattr(orc, scheme),
                     bc_lo=(orc.BC_OUTFLOW, 0, 0), bc_hi=(orc.BC_OUTFLOW, 0, 0))
        U = orc.apply_bc(c, M, U)
        dt0 = orc.cfl_dt(c, M, U, 0.3)
        nsteps = int(math.ceil(t_end / dt0))
        dt = t_end / nsteps
        U = orc.step(c, M, U, dt, nsteps)
        ex, _, _ = exact_riemann(x, t_end, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
        rho = U[0, 0, 0]
        errs.append(np.mean(np.abs(rho - ex[0])))
        # no overshoot beyond the initial data range by more than a few percent
        assert rho.max() <= 1.0 + 0.03 and rho.min() >= 0.125 - 0.03
    assert errs[0] > errs[1] > errs[2]
    assert math.log(errs[0] / errs[2], 4) > 0.6, errs


@pytest.mark.parametrize("scheme", ["WENO5", "WENO7", "HYBRID"])
def test_rhs_invariant_to_coordinate_scaling(orc, scheme):
    """Reading R23: the same 1-D Sod state on grids whose transverse cell
    sizes differ (J and the split fluxes scale with them) gives the same
    L(U) = J R: the shock-capturing weights do not depend on the arbitrary
    scaling of the computational coordinates."""
    n = 101
    U, met, Ma, x = cases.shock_tube(n)
    Ls = []
    for hy, hz in ((1.0, 1.0), (1e-3, 2e-2), (5e2, 1e-4)):
        m = met.copy()
        m[4], m[8] = 1.0 / hy, 1.0 / hz
        m[9] = met[9] / (hy * hz)
        M = cases.expand_metrics(m, (1, 1, n))
        c = orc.Case(n, 1, 1, Re=0.0, Ma=Ma, gamma=G, scheme=getattr(orc, scheme),
                     bc_lo=(orc.BC_OUTFLOW, 0, 0), bc_hi=(orc.BC_OUTFLOW, 0, 0))
        Ls.append(orc.rhs(c, M, orc.apply_bc(c, M, U)))
    scale = np.abs(Ls[0]).max()
    assert scale > 1.0
    for L in Ls[1:]:
        assert np.abs(L - Ls[0]).max() < 1e-12 * scale


def _kinetic_rate(U, L):
    rho = U[0]
    m = U[1:4]
    Lr, Lm = L[0], L[1:4]
    return np.mean(np.sum(m * Lm, axis=0) / rho - 0.5 * np.sum(m * m, axis=0) / rho ** 2 * Lr)


def test_taylor_green_dissipation_rate(orc):
    """dK/dt(0) = -(3/4) mu(1)/Re for the Taylor-Green vortex (div u = 0,
    T = 1 at t = 0): the viscous part of the discrete rate matches."""
    n = 32
    U = cases.taylor_green(n, Ma=0.5)
    met = cases.expand_metrics(cases.uniform_metrics(n, n, n), (n, n, n))
    Re = 400.0
    cv = orc.Case(n, n, n, Re=Re, Ma=0.5, scheme=orc.UD7, visc_law=orc.POWER, visc_omega=0.76)
    ci = orc.Case(n, n, n, Re=0.0, Ma=0.5, scheme=orc.UD7)
    kv = _kinetic_rate(U, orc.rhs(cv, met, U))
    ki = _kinetic_rate(U, orc.rhs(ci, met, U))
    assert abs((kv - ki) - (-0.75 / Re)) <= 1e-6 * 0.75 / Re
    # the inviscid scheme itself is nearly non-dissipative on this field
    assert abs(ki) < 1e-3 * 0.75 / Re


def test_shear_wave_viscous_rhs(orc):
    """u = e sin y: viscous L(rho u) = -(mu/Re) e sin y, L(E) = (mu/Re) e^2 cos 2y."""
    n = 32
    e, Re, Ma = 0.1, 50.0, 0.4
    y = np.arange(n) * 2 * math.pi / n
    shp = (1, n, 1)
    o = np.ones(shp)
    u = (e * np.sin(y)).reshape(shp)
    p = o / (G * Ma * Ma)        # T = 1 with rho = 1
    U = cases.conserved(o, u, 0 * o, 0 * o, p, G)
    met = cases.expand_metrics(cases.uniform_metrics(1, n, 1, 1.0, 2 * math.pi, 1.0), (1, n, 1))
    Lv = orc.rhs(orc.Case(1, n, 1, Re=Re, Ma=Ma, visc_law=orc.POWER, visc_omega=0.76), met, U)
    Li = orc.rhs(orc.Case(1, n, 1, Re=0.0, Ma=Ma), met, U)
    d = (Lv - Li)[:, 0, :, 0]
    assert np.allclose(d[1], -(1.0 / Re) * e * np.sin(y), atol=1e-9)
    assert np.allclose(d[4], (1.0 / Re) * e * e * np.cos(2 * y), atol=1e-9)
    assert np.abs(d[0]).max() == 0.0
    assert np.abs(d[2]).max() <= 1e-13 and np.abs(d[3]).max() <= 1e-13


@pytest.mark.parametrize("omega", [0.0, 0.76])
def test_heat_wave_viscous_rhs(orc, omega):
    """T = 1 + e sin z at rest: L(E) = d/dz(k(T) dT/dz), k = mu/((g-1) Ma^2 Pr Re)."""
    n = 32
    e, Re, Ma, Pr = 0.05, 80.0, 0.6, 0.72
    z = np.arange(n) * 2 * math.pi / n
    shp = (n, 1, 1)
    T = (1.0 + e * np.sin(z)).reshape(shp)
    p = np.ones(shp) / (G * Ma * Ma)
    rho = G * Ma * Ma * p / T
    zero = np.zeros(shp)
    U = cases.conserved(rho, zero, zero, zero, p, G)
    met = cases.expand_metrics(cases.uniform_metrics(1, 1, n, 1.0, 1.0, 2 * math.pi), shp)
    kw = dict(Ma=Ma, Pr=Pr, visc_law=orc.POWER, visc_omega=omega)
    Lv = orc.rhs(orc.Case(1, 1, n, Re=Re, **kw), met, U)
    Li = orc.rhs(orc.Case(1, 1, n, Re=0.0, **kw), met, U)
    d = (Lv - Li)[:, :, 0, 0]
    Tz = T.ravel()
    k0 = 1.0 / ((G - 1) * Ma * Ma * Pr * Re)
    dT = e * np.cos(z)
    d2T = -e * np.sin(z)
    expect = k0 * (omega * Tz ** (omega - 1) * dT * dT + Tz ** omega * d2T)
    assert np.allclose(d[4], expect, atol=1e-9)
    assert np.abs(d[:4]).max() == 0.0


def test_sutherland_law(orc):
    """mu(T)/mu(T_ref) = (T*/T_ref)^(3/2) (T_ref + S)/(T* + S), S = 110.4 K."""
    c = orc.Case(4, 4, 4, visc_law=orc.SUTHERLAND, T_ref=108.1)
    for Tstar in (60.0, 108.1, 300.0, 900.0):
        ref = (Tstar / 108.1) ** 1.5 * (108.1 + 110.4) / (Tstar + 110.4)
        assert abs(orc.viscosity(c, Tstar / 108.1) - ref) <= 1e-14 * ref
    cp = orc.Case(4, 4, 4, visc_law=orc.POWER, visc_omega=0.76)
    assert orc.viscosity(cp, 1.0) == 1.0
    assert abs(orc.viscosity(cp, 2.0) - 2.0 ** 0.76) <= 1e-15


def test_plane_shear_wave_on_affine_grid(orc):
    """Viscous RHS through non-diagonal metrics: u = a sin(s), s = q.x with
    q = (2 pi/n) grad(xi), uniform rho and T.  Closed form:
      L(rho u_i) = -(mu/Re)(a_i |q|^2 + (q_i a.q)/3) sin s,
      L(E)       =  (mu/Re)(|a|^2 |q|^2 + (a.q)^2/3) cos 2s."""
    n = 24
    Re, Ma = 60.0, 0.5
    A = np.array([[1.0, 0.3, -0.2], [0.1, 1.2, 0.25], [-0.15, 0.05, 0.9]])
    Minv = np.linalg.inv(A) * 3.0       # rows: grad xi, grad eta, grad zeta
    met = np.zeros(10)
    met[:9] = Minv.ravel()
    met[9] = abs(np.linalg.det(Minv))
    M = cases.expand_metrics(met, (n, n, n))
    q = 2 * math.pi / n * Minv[0]
    a = np.array([0.07, -0.04, 0.05])
    s = 2 * math.pi * np.arange(n) / n
    shp = (1, 1, n)
    o = np.ones((n, n, n))
    vel = [a[i] * np.broadcast_to(np.sin(s).reshape(shp), (n, n, n)) for i in range(3)]
    U = cases.conserved(o, vel[0], vel[1], vel[2], o / (G * Ma * Ma), G)
    kw = dict(Ma=Ma, visc_law=orc.POWER, visc_omega=0.76)
    Lv = orc.rhs(orc.Case(n, n, n, Re=Re, **kw), M, U)
    Li = orc.rhs(orc.Case(n, n, n, Re=0.0, **kw), M, U)
    d = Lv - Li
    q2, aq = q @ q, a @ q
    for i in range(3):
        expect = -(1.0 / Re) * (a[i] * q2 + q[i] * aq / 3.0) * np.sin(s)
        assert np.allclose(d[1 + i, 0, 0], expect, atol=1e-8 * abs(expect).max())
    expect = (1.0 / Re) * ((a @ a) * q2 + aq * aq / 3.0) * np.cos(2 * s)
    assert np.allclose(d[4, 0, 0], expect, atol=1e-8 * abs(expect).max())
    assert np.abs(d[0]).max() == 0.0
