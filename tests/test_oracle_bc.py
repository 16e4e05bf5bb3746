"""Pins of the oracle's boundary conditions and of the Taylor-Green energy
history (CPU only).

- Blowing/suction strip on the eta-low isothermal wall (reading R12 of the
  Table 8 ramp case): values worked out by hand at chosen (x, z, t), zero net
  mass flux over the strip times the span, and the direction of the injected
  velocity along grad(eta) on a tilted wall face.
- Inflow face: the Dirichlet profile is reproduced at every eta and zeta of
  the xi-low face; the outflow face copies the first interior node's
  primitives; interior nodes are untouched.
- Taylor-Green vortex (config 1, R19): the kinetic energy over 10 RK3 steps
  follows K0 - 3 mu(1) t/(4 Re), with a tolerance set by the energy drift of
  the same run without viscosity.
"""
import math

import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

GAMMA, MA = 1.4, 0.5


def sheared_metrics(nx, ny, nz, a, b, c, e):
    """Metrics of x = a xi, y = b eta + c xi, z = e zeta: grad(xi) = (1/a, 0, 0),
    grad(eta) = (-c/(a b), 1/b, 0), grad(zeta) = (0, 0, 1/e), J = 1/(a b e)."""
    m = np.zeros(10)
    m[0] = 1.0 / a
    m[3], m[4] = -c / (a * b), 1.0 / b
    m[8] = 1.0 / e
    m[9] = 1.0 / (a * b * e)
    return cases.expand_metrics(m, (nz, ny, nx))


def uniform_state(shape, rho=1.2, vel=(0.3, -0.1, 0.05), p=None):
    nz, ny, nx = shape
    p = 1.0 / (GAMMA * MA * MA) if p is None else p
    one = np.ones(shape)
    return cases.conserved(rho * one, vel[0] * one, vel[1] * one, vel[2] * one, p * one, GAMMA)


# ----------------------------------------------------------------------------
# blowing / suction strip
# ----------------------------------------------------------------------------

NX, NY, NZ = 16, 9, 8
A_X, B_Y, C_XY, E_Z = 0.25, 0.2, 0.1, 0.5        # x = 0.25 i, y = 0.2 j + 0.1 x... see sheared_metrics
AMP, X0, X1, OMEGA, MODE = 0.03, 1.0, 3.0, 0.5, 1
LZ = NZ * E_Z                                       # span 4: z_k = 0.5 k
T_PEAK = math.pi                                    # omega t = pi/2


def blowing_case(orc, t_amp=1.0):
    wall_x = A_X * np.arange(NX)
    wall_z = E_Z * np.arange(NZ)
    blowing = dict(amp=AMP * t_amp, x0=X0, x1=X1, omega=OMEGA, m=MODE, Lz=LZ, wall_x=wall_x, wall_z=wall_z)
    c = orc.Case(NX, NY, NZ, Ma=MA, T_wall=2.0, bc_lo=(0, 1, 0), bc_hi=(0, 3, 0), blowing=blowing)
    return c, sheared_metrics(NX, NY, NZ, A_X, B_Y, C_XY, E_Z)


def wall_velocity(orc, t):
    c, met = blowing_case(orc)
    U = orc.apply_bc(c, met, uniform_state((NZ, NY, NX)), t)
    P = orc.primitives(c, U)
    return P[:, :, 0, :], P  # wall layer [7][nz][nx]


# direction of grad(eta) = (-c/(a b), 1/b, 0) = (-2, 5, 0)
N_HAT = np.array([-2.0, 5.0, 0.0]) / math.sqrt(29.0)


@pytest.mark.parametrize("i,k,expect", [
    (6, 0, 1.0),                 # x = 1.5: sin(pi/2);    z = 0:   cos(0)
    (10, 4, 1.0),                # x = 2.5: sin(3 pi/2);  z = 2:   cos(pi)       -> (-1)(-1)
    (6, 4, -1.0),                # suction half of the span
    (5, 1, 0.5),                 # x = 1.25: sin(pi/4);   z = 0.5: cos(pi/4)     -> 1/2
    (12, 0, 0.0),                # x = 3.0: strip end, sin(2 pi)
    (2, 0, 0.0),                 # x = 0.5: outside the strip
    (14, 0, 0.0),                # x = 3.5: outside the strip
])
def test_blowing_hand_values(orc, i, k, expect):
    """v_n = A sin(2 pi (x-x0)/(x1-x0)) cos(2 pi m z/Lz) sin(omega t) at
    omega t = pi/2, evaluated by hand for chosen wall nodes."""
    W, _ = wall_velocity(orc, T_PEAK)
    vel = W[1:4, k, i]
    vn = float(vel @ N_HAT)
    assert abs(vn - AMP * expect) <= 1e-15, (i, k, vn)
    # nothing along the wall: the injected velocity is normal to it
    assert np.abs(vel - vn * N_HAT).max() <= 1e-15


def test_blowing_direction_is_grad_eta_on_a_tilted_wall(orc):
    """The wall normal is grad(eta)/|grad(eta)|, pointing into the flow
    (v > 0 where v_n > 0), not a metric row of another direction."""
    W, _ = wall_velocity(orc, T_PEAK)
    u, v, w = W[1, 0, 6], W[2, 0, 6], W[3, 0, 6]
    assert v > 0 and u < 0 and w == 0.0
    assert abs(u / v - (-2.0 / 5.0)) <= 1e-14


def test_blowing_is_zero_at_rest_time_and_follows_sin_omega_t(orc):
    W0, _ = wall_velocity(orc, 0.0)
    assert np.abs(W0[1:4]).max() == 0.0
    t = math.pi / 3.0  # omega t = pi/6: half the peak
    Wh, _ = wall_velocity(orc, t)
    Wp, _ = wall_velocity(orc, T_PEAK)
    np.testing.assert_allclose(Wh[1:4], 0.5 * Wp[1:4], rtol=0, atol=1e-16)


def test_blowing_zero_net_mass_flux_over_strip_and_span(orc):
    """Sum over the wall nodes of rho_w v_n (equal face areas on this grid)
    vanishes: the strip injects as much mass as it removes."""
    W, P = wall_velocity(orc, T_PEAK)
    rho = W[0]
    vn = np.einsum("dkx,d->kx", W[1:4], N_HAT)
    flux = rho * vn
    assert np.abs(flux).max() > 0.5 * AMP * rho.max()   # the strip is active
    assert abs(flux.sum()) <= 1e-14 * np.abs(flux).sum()
    # also per spanwise row and per streamwise column
    assert np.abs(flux.sum(axis=0)).max() <= 1e-15 * NZ
    assert np.abs(flux.sum(axis=1)).max() <= 1e-15 * NX


def test_isothermal_wall_state_with_blowing(orc):
    """T = T_w and p_w = (4 p1 - p2)/3 (= p on a uniform interior) at every
    wall node, blowing or not."""
    _, P = wall_velocity(orc, T_PEAK)
    p = 1.0 / (GAMMA * MA * MA)
    np.testing.assert_allclose(P[5, :, 0, :], 2.0, rtol=1e-14)
    np.testing.assert_allclose(P[4, :, 0, :], p, rtol=1e-14)


# ----------------------------------------------------------------------------
# inflow and outflow faces
# ----------------------------------------------------------------------------

def test_inflow_profile_on_every_zeta_and_outflow_copy(orc):
    nx, ny, nz = 12, 10, 6
    rng = np.random.default_rng(5)
    yv = np.linspace(0.0, 1.0, ny)
    prof = np.stack([1.0 + 0.3 * yv, np.tanh(3.0 * yv), 0.02 * np.sin(3 * yv), -0.01 * yv,
                     (1.0 + 0.1 * yv ** 2) / (GAMMA * MA * MA)])
    c = orc.Case(nx, ny, nz, Ma=MA, T_wall=1.5, bc_lo=(2, 1, 0), bc_hi=(3, 3, 0), inflow=prof)
    met = cases.expand_metrics(cases.uniform_metrics(nx, ny, nz, 1.0, 1.0, 1.0), (nz, ny, nx))
    rho = 1.0 + 0.1 * rng.random((nz, ny, nx))
    vel = 0.2 * rng.standard_normal((3, nz, ny, nx))
    p = (1.0 + 0.1 * rng.random((nz, ny, nx))) / (GAMMA * MA * MA)
    U0 = cases.conserved(rho, vel[0], vel[1], vel[2], p, GAMMA)
    U = orc.apply_bc(c, met, U0)
    P = orc.primitives(c, U)
    # the inflow face reproduces the profile at every zeta (and every eta
    # that is not a wall node: the eta faces are applied after the xi faces)
    for k in range(nz):
        for q, row in enumerate((0, 1, 2, 3, 4)):
            np.testing.assert_allclose(P[row, k, 1:ny - 1, 0], prof[q, 1:ny - 1], rtol=1e-14, atol=1e-16)
    # zeroth-order extrapolation at the outflow: the first interior node
    np.testing.assert_allclose(P[:5, :, 1:ny - 1, nx - 1], P[:5, :, 1:ny - 1, nx - 2], rtol=1e-14, atol=1e-16)
    # interior nodes untouched, bit for bit
    assert np.array_equal(U[:, :, 1:ny - 1, 1:nx - 1], U0[:, :, 1:ny - 1, 1:nx - 1])


# ----------------------------------------------------------------------------
# Taylor-Green kinetic-energy history
# ----------------------------------------------------------------------------

def _kinetic(U):
    return float(np.mean(0.5 * np.sum(U[1:4] ** 2, axis=0) / U[0]))


def test_taylor_green_energy_history_10_steps(orc):
    """K(t) = K0 - 3 mu(1) t/(4 Re) over 10 RK3 steps at CFL 0.5 (config 1).

    For u = sin x cos y cos z, v = -cos x sin y cos z, w = 0: K0 = 1/8 and
    <|grad u|^2> = 3/4, so the viscous loss rate is 3 mu/(4 Re) while the flow
    stays near its initial state.  The same run without viscosity measures
    what else moves K over these steps (pressure-dilatation exchange and the
    scheme's own dissipation); the viscous run must follow the linear loss
    within 1.5 times that drift plus 0.1 % of the loss, and the viscous
    minus inviscid energy within 0.5 % of the linear loss at every step.
    """
    n, Re = 32, 400.0
    U0 = cases.taylor_green(n, Ma=MA)
    met = cases.expand_metrics(cases.uniform_metrics(n, n, n), (n, n, n))
    cv = orc.Case(n, n, n, Re=Re, Ma=MA, scheme=orc.HYBRID, visc_law=orc.POWER, visc_omega=0.76)
    ci = orc.Case(n, n, n, Re=0.0, Ma=MA, scheme=orc.HYBRID)
    dt = orc.cfl_dt(cv, met, U0, 0.5)
    K0 = _kinetic(U0)
    assert abs(K0 - 0.125) < 1e-15
    mu1 = orc.viscosity(cv, 1.0)
    Uv, Ui = U0, U0
    for s in range(1, 11):
        Uv = orc.step(cv, met, Uv, dt, 1)
        Ui = orc.step(ci, met, Ui, dt, 1)
        t = s * dt
        loss = 0.75 * mu1 * t / Re
        kv, ki = _kinetic(Uv), _kinetic(Ui)
        drift = abs(ki - K0)
        assert abs(kv - (K0 - loss)) <= 1.5 * drift + 1e-3 * loss, (s, kv, K0 - loss, drift)
        assert abs((kv - ki) + loss) <= 5e-3 * loss, (s, kv - ki, -loss)
    # the inviscid drift stays small next to the viscous loss it bounds
    assert drift < 0.05 * loss
