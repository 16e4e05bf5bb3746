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
