"""Input generators: the oblique-shock state used for the ramp initial field
against textbook values (weak solution, gamma = 1.4)."""
import math

import numpy as np

from paper_2209_15333_gb300 import cases


def test_oblique_shock_textbook():
    # M = 2, wedge 10 degrees: beta = 39.31 deg, p2/p1 = 1.7066, M2 = 1.6405
    Ma = 2.0
    beta, rho2, q2, p2 = cases.oblique_shock(Ma, 10.0)
    assert abs(math.degrees(beta) - 39.31) < 0.01
    assert abs(p2 * 1.4 * Ma * Ma - 1.7066) < 1e-3
    T2 = 1.4 * Ma * Ma * p2 / rho2
    M2 = q2 * Ma / math.sqrt(T2)
    assert abs(M2 - 1.6405) < 1e-3


def test_oblique_shock_detached():
    import pytest
    with pytest.raises(ValueError):
        cases.oblique_shock(2.0, 30.0)


def test_ramp_case_initial_field():
    rc = cases.ramp_case(96, 24, 8, 34.0, 6.0, Tw=5.9)
    U = rc["U"]
    assert np.isfinite(U).all() and U[0].min() > 0
    rho = U[0]
    p = 0.4 * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho)
    assert p.min() > 0
    # wall nodes at rest, T = T_wall
    assert np.abs(U[1:4, :, 0, :]).max() < 1e-12
    T = 1.4 * 36.0 * p / rho
    assert np.allclose(T[:, 0, :], 5.9)
