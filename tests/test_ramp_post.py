"""Ramp post-processing on the host: the Van Driest transform."""
import numpy as np

from paper_2209_15333_gb300.ramp import van_driest


def test_van_driest_constant_density_is_plain_wall_units():
    Re, mu_w = 20000.0, 1.7
    y = np.linspace(0.0, 0.05, 60) ** 1.3
    u = np.tanh(40.0 * y)
    yp, up, ut = van_driest(y, u, np.ones_like(y), mu_w, Re)
    # u_tau from the exact wall gradient (40), to the one-sided formula's accuracy
    assert abs(ut - np.sqrt(mu_w / Re * 40.0)) < 2e-3 * ut
    assert np.allclose(up, u / ut, rtol=0, atol=1e-12)
    assert np.allclose(yp, Re * ut * y / mu_w)


def test_van_driest_integral():
    """rho/rho_w = (1 + u)^-2: u_VD = int_0^u (1 + s)^-1 ds = ln(1 + u)."""
    y = np.linspace(0.0, 1.0, 4001)
    u = 2.0 * y
    rho = 1.0 / (1.0 + u) ** 2
    _, up, ut = van_driest(y, u, rho, 1.0, 1.0)
    assert np.abs(up * ut - np.log1p(u)).max() < 1e-6


def test_wall_quantities_on_a_linear_wall_layer():
    """u_t = a d (d the distance normal to the wall, the velocity along the
    wall) on the ramp grid, upstream and on the ramp face: C_f = 2 mu_w a/Re
    from the one-sided eta derivative through the metrics, and p_w/p_inf of
    a uniform pressure."""
    import math
    from paper_2209_15333_gb300 import cases
    from paper_2209_15333_gb300.ramp import wall_quantities
    nx, ny, nz, ang, Ma, Tw, Tref, Re = 160, 64, 2, 24.0, 2.9, 2.8, 108.1, 20000.0
    met2, X, Y, z, wx = cases.ramp_grid(nx, ny, nz, ang)
    a = 3.0
    th = np.where(X[0] > 0.0, math.radians(ang), 0.0)
    d = (Y - Y[0:1, :]) * np.cos(th)[None, :]       # normal distance to the (straight) wall
    ut = a * d
    u, v = ut * np.cos(th), ut * np.sin(th)
    p = np.full_like(u, 1.3 / (1.4 * Ma * Ma))
    rho = np.ones_like(u)
    shp = (nz, ny, nx)
    U = cases.conserved(*(np.broadcast_to(q[None], shp) for q in (rho, u, v, np.zeros_like(u), p)), 1.4)
    pw, cf = wall_quantities(U, met2, Ma, Tw, Tref, Re=Re)
    s = 110.4 / Tref
    mu_w = Tw ** 1.5 * (1.0 + s) / (Tw + s)
    expect = 2.0 * mu_w * a / Re
    away = np.abs(X[0]) > 0.5                        # the corner column mixes the two faces
    assert np.allclose(pw, 1.3)
    assert np.abs(cf[away] / expect - 1.0).max() < 1e-6
