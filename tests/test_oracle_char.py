"""Pins of the oracle's characteristic-variable reconstruction (Sec. 2.2.2,
Eq. 31-40; reading R25).

  * S S^-1 = I, and S A_n S^-1 = diag(u_n, u_n, u_n, u_n - c, u_n + c) for the
    flux Jacobian A_n = d(F.n)/dU computed by complex-step differentiation
    (the definition of the left/right eigenvector matrices);
  * the normal-dependent basis of Eq. 39-40 is orthonormal on both branches;
  * with linear weights (eps -> infinity) the reconstruction is linear, so
    projecting onto characteristic fields and back changes nothing: the
    characteristic RHS equals the component-wise one;
  * a uniform stream stays uniform; Sod's problem against its exact solution.
"""
import math

import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from test_oracle_sw import G, exact_flux, jacobian_complex_step, random_state
from gpu_helpers import turbulence_field


def _normals(rng):
    out = [np.array(v, float) for v in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0.6, 0.8), (0.6, 0.8, 0), (0, 0.8, 0.6),
                                       (1, 1, 1))]
    out += [rng.normal(size=3) for _ in range(40)]
    return [n / np.linalg.norm(n) for n in out]


def test_char_matrices_are_inverse(orc):
    rng = np.random.default_rng(21)
    for n in _normals(rng):
        U = random_state(rng)
        S, Si = orc.char_matrices(G, U, n)
        assert np.abs(S @ Si - np.eye(5)).max() < 1e-12
        assert np.abs(Si @ S - np.eye(5)).max() < 1e-12


def test_char_matrices_diagonalise_flux_jacobian(orc):
    rng = np.random.default_rng(22)
    for n in _normals(rng):
        U = random_state(rng)
        A = jacobian_complex_step(U, n)
        S, Si = orc.char_matrices(G, U, n)
        D = S @ A @ Si
        rho = U[0]
        u = U[1:4] / rho
        p = (G - 1) * (U[4] - 0.5 * rho * u @ u)
        c = math.sqrt(G * p / rho)
        un = u @ n
        expect = np.diag([un, un, un, un - c, un + c])
        scale = abs(un) + c
        assert np.abs(D - expect).max() < 1e-11 * scale


def test_char_basis_orthonormal(orc):
    """Eq. 39-40: rows 2-3 of S carry l and m; with n they form an
    orthonormal right-handed basis on both branches of Eq. 39."""
    rng = np.random.default_rng(23)
    U = random_state(rng)
    for n in _normals(rng):
        S, _ = orc.char_matrices(G, U, n)
        l, m = S[1, 1:4], S[2, 1:4]
        B = np.array([n, l, m])
        assert np.abs(B @ B.T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(np.array([l, m, n])) - 1.0) < 1e-14


@pytest.mark.parametrize("scheme", ["WENO5", "WENO7", "HYBRID"])
def test_linear_weights_equal_component_wise(orc, scheme):
    """eps = 1e30 makes every WENO weight linear: characteristic and
    component-wise reconstruction then agree to round-off (on a curved
    grid, where the stencil nodes' metrics differ from the interface's)."""
    n = 18
    met, _ = cases.wavy_grid(n, amp=0.05)
    U = turbulence_field((n, n, n), 31, amp=0.6)
    M = cases.expand_metrics(met, (n, n, n))
    kw = dict(Re=0.0, Ma=0.5, scheme=getattr(orc, scheme), weno_eps=1e30)
    if scheme == "HYBRID":
        rng = np.random.default_rng(5)
        kw["forced_cls"] = rng.integers(0, 3, size=(n, n, n)).astype(np.uint8)
    Lc = orc.rhs(orc.Case(n, n, n, **kw), M, U)
    Lx = orc.rhs(orc.Case(n, n, n, recon_vars=orc.RECON_CHARACTERISTIC, **kw), M, U)
    for q in range(5):
        scale = np.abs(Lc[q]).max() + 1e-300
        assert np.abs(Lx[q] - Lc[q]).max() <= 1e-11 * max(scale, np.abs(Lc).max() * 1e-3)


def test_nonlinear_weights_differ(orc):
    """With the real eps the two forms differ where the field is not smooth
    (so the characteristic path is really taken)."""
    n = 101
    U, met, Ma, x = cases.shock_tube(n)
    M = cases.expand_metrics(met, (1, 1, n))
    kw = dict(Re=0.0, Ma=Ma, gamma=G, scheme=orc.WENO5, bc_lo=(orc.BC_OUTFLOW, 0, 0), bc_hi=(orc.BC_OUTFLOW, 0, 0))
    c0 = orc.Case(n, 1, 1, **kw)
    c1 = orc.Case(n, 1, 1, recon_vars=orc.RECON_CHARACTERISTIC, **kw)
    U = orc.apply_bc(c0, M, U)
    d = np.abs(orc.rhs(c1, M, U) - orc.rhs(c0, M, U)).max()
    assert d > 1e-3


@pytest.mark.parametrize("grid", ["cartesian", "wavy_fsp"])
def test_char_free_stream(orc, grid):
    n = 16
    if grid == "cartesian":
        met, mode = cases.uniform_metrics(n, n, n), orc.METRIC_NODAL
    else:
        met, mode = cases.wavy_grid(n, amp=0.05)[0], orc.METRIC_FSP
    shp = (n, n, n)
    U = cases.conserved(np.full(shp, 1.2), np.full(shp, 0.7), np.full(shp, -0.3), np.full(shp, 0.2),
                        np.full(shp, 1.0 / (G * 0.25)), G)
    M = cases.expand_metrics(met, shp)
    c = orc.Case(n, n, n, Re=0.0, Ma=0.5, scheme=orc.WENO5, metric_mode=mode, recon_vars=orc.RECON_CHARACTERISTIC)
    L = orc.rhs(c, M, U)
    flux_scale = np.abs(U).max() * np.abs(M[:9] / M[9]).max() * np.abs(M[9]).max()
    assert np.abs(L).max() <= 1e-12 * flux_scale


def test_char_sod(orc):
    """Sod's problem with characteristic WENO5: L1 error decreasing and
    overshoot below the component-wise form's bound."""
    from test_oracle_physics import exact_riemann
    errs, over = [], []
    for n in (101, 201, 401):
        U, met, Ma, x = cases.shock_tube(n)
        M = cases.expand_metrics(met, (1, 1, n))
        c = orc.Case(n, 1, 1, Re=0.0, Ma=Ma, gamma=G, scheme=orc.WENO5, bc_lo=(orc.BC_OUTFLOW, 0, 0),
                     bc_hi=(orc.BC_OUTFLOW, 0, 0), recon_vars=orc.RECON_CHARACTERISTIC)
        U = orc.apply_bc(c, M, U)
        dt0 = orc.cfl_dt(c, M, U, 0.3)
        nsteps = int(math.ceil(0.2 / dt0))
        U = orc.step(c, M, U, 0.2 / nsteps, nsteps)
        ex, _, _ = exact_riemann(x, 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
        rho = U[0, 0, 0]
        errs.append(np.mean(np.abs(rho - ex[0])))
        over.append(max(rho.max() - 1.0, 0.125 - rho.min()))
    assert errs[0] > errs[1] > errs[2]
    assert math.log(errs[0] / errs[2], 4) > 0.6, errs
    assert max(over) < 0.03, over


@pytest.mark.parametrize("recon", ["COMPONENT", "CHARACTERISTIC"])
def test_mirror_symmetry(orc, recon):
    """Reflecting a periodic line (x -> -x, u -> -u) reflects L(U): the
    interface state of Eq. 32 is symmetric in the two nodes, and flipping
    the normal only re-orders and re-signs the characteristic fields."""
    n = 64
    rng = np.random.default_rng(24)
    x = np.arange(n) / n
    rho = 1.0 + 0.5 * (x > 0.4) + 0.05 * rng.standard_normal(n)
    u = 0.3 * np.sin(2 * np.pi * x) + 0.05 * rng.standard_normal(n)
    p = 1.0 + 2.0 * (x > 0.6) + 0.05 * rng.standard_normal(n)
    shp = (1, 1, n)
    U = cases.conserved(rho.reshape(shp), u.reshape(shp), np.zeros(shp), np.zeros(shp), p.reshape(shp), G)
    met = np.zeros(10)
    met[0], met[4], met[8], met[9] = n, 1.0, 1.0, n
    M = cases.expand_metrics(met, shp)
    c = orc.Case(n, 1, 1, Re=0.0, Ma=1.0 / math.sqrt(G), gamma=G, scheme=orc.WENO5,
                 recon_vars=getattr(orc, "RECON_" + recon))
    L = orc.rhs(c, M, U)
    Ur = U[:, :, :, ::-1].copy()
    Ur[1] *= -1.0
    Lr = orc.rhs(c, M, Ur)
    Lback = Lr[:, :, :, ::-1].copy()
    Lback[1] *= -1.0
    assert np.abs(Lback - L).max() <= 1e-12 * np.abs(L).max()


@pytest.mark.parametrize("recon", ["COMPONENT", "CHARACTERISTIC"])
def test_mirror_symmetry_curved_grid(orc, recon):
    """The same reflection x -> -x on a curved periodic grid, whose metric
    directions vary along xi: the reflected grid has the nodes in reverse xi
    order with xi_y, xi_z, eta_x, zeta_x negated.  An interface normal or
    state that favoured one of its two nodes would break the symmetry."""
    n = 16
    met, _ = cases.wavy_grid(n, amp=0.06)
    M = cases.expand_metrics(met, (n, n, n))
    U = turbulence_field((n, n, n), 32, amp=0.5)
    Mr = M[:, :, :, ::-1].copy()
    for e in (1, 2, 3, 6):
        Mr[e] *= -1.0
    Ur = U[:, :, :, ::-1].copy()
    Ur[1] *= -1.0
    c = orc.Case(n, n, n, Re=0.0, Ma=0.5, scheme=orc.WENO5, recon_vars=getattr(orc, "RECON_" + recon))
    L = orc.rhs(c, M, U)
    Lback = orc.rhs(c, Mr, Ur)[:, :, :, ::-1].copy()
    Lback[1] *= -1.0
    assert np.abs(Lback - L).max() <= 1e-11 * np.abs(L).max()
