"""Seeded synthetic inputs: grids, metrics and initial fields.

This module holds no step of the solver.  It builds the inputs that both the
GPU library and the CPU oracle receive: grid metrics (the caller-supplied
input of Eq. 3 and Eq. 4) and initial conserved fields U = (rho, rho u,
rho v, rho w, E) with E = p/(gamma-1) + rho |u|^2/2 and p = rho T/(gamma Ma^2)
(the nondimensional gas of Eqs. 8, 16, 17).

Layouts: fields are float64 ``[5][nz][ny][nx]``; full metrics are
``[10][nz][ny][nx]`` = xi_x, xi_y, xi_z, eta_x, eta_y, eta_z, zeta_x,
zeta_y, zeta_z, J; two-dimensional (extruded) metrics are ``[10][ny][nx]``;
uniform metrics are 10 numbers.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi

# 8-point midpoint interpolation (Lagrange through offsets -3..4 at 1/2)
_MID8 = np.array([-5.0, 49.0, -245.0, 1225.0, 1225.0, -245.0, 49.0, -5.0]) / 2048.0


# ----------------------------------------------------------------------------
# conversions of initial data
# ----------------------------------------------------------------------------

def conserved(rho, u, v, w, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, E]), dtype=np.float64)


def expand_metrics(metrics, shape):
    """Expand uniform (10,) or extruded (10, ny, nx) metrics to (10, nz, ny, nx)."""
    nz, ny, nx = shape
    m = np.asarray(metrics, dtype=np.float64)
    if m.ndim == 1:
        return np.ascontiguousarray(np.broadcast_to(m[:, None, None, None], (10, nz, ny, nx)))
    if m.ndim == 3:
        return np.ascontiguousarray(np.broadcast_to(m[:, None, :, :], (10, nz, ny, nx)))
    return np.ascontiguousarray(m)


# ----------------------------------------------------------------------------
# uniform periodic boxes
# ----------------------------------------------------------------------------

def uniform_metrics(nx, ny, nz, Lx=TWO_PI, Ly=TWO_PI, Lz=TWO_PI):
    """Cartesian grid with spacings L/n (periodic, no duplicate end node)."""
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    m = np.zeros(10)
    m[0], m[4], m[8] = 1.0 / hx, 1.0 / hy, 1.0 / hz
    m[9] = 1.0 / (hx * hy * hz)
    return m


def box_coords(nx, ny, nz, Lx=TWO_PI, Ly=TWO_PI, Lz=TWO_PI, x0=0.0, y0=0.0, z0=0.0):
    x = x0 + np.arange(nx) * (Lx / nx)
    y = y0 + np.arange(ny) * (Ly / ny)
    z = z0 + np.arange(nz) * (Lz / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def taylor_green(n, Ma=0.5, gamma=1.4):
    """Compressible Taylor-Green vortex on [0, 2 pi)^3, isothermal start T = 1.

    u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = p0 + (cos 2x + cos 2y)(cos 2z + 2)/16 with rho0 = U = 1 and
    p0 = 1/(gamma Ma^2); rho = gamma Ma^2 p (T = 1).
    """
    X, Y, Z = box_coords(n, n, n)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p0 = 1.0 / (gamma * Ma * Ma)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = gamma * Ma * Ma * p
    return conserved(rho, u, v, w, p, gamma)


def isotropic_turbulence(n, seed, Mt=0.5, gamma=1.4, k0=4.0, Re_lambda=72.0, visc_mu1=1.0):
    """Decaying isotropic turbulence initial field on [0, 2 pi)^3 (n^3 nodes).

    Random-phase solenoidal velocity with E(k) ~ k^4 exp(-2 (k/k0)^2),
    scaled to <u_i u_i> = 1, uniform rho = T = 1, so the turbulent Mach
    number equals Ma = Mt.  Returns (U, Re) with Re chosen so that
    Re_lambda = u' lambda Re / mu(1), u' = 1/sqrt(3),
    lambda = u' / <(du/dx)^2>^(1/2) measured on the generated field.
    """
    return isotropic_turbulence_box(n, n, n, seed, Mt, gamma, k0, Re_lambda, visc_mu1)


def isotropic_turbulence_box(nx, ny, nz, seed, Mt=0.5, gamma=1.4, k0=4.0, Re_lambda=72.0, visc_mu1=1.0):
    """The same recipe on an nx x ny x nz box of [0, 2 pi)^3 (uneven
    resolutions per axis; integer wavenumbers, each axis up to its Nyquist)."""
    rng = np.random.default_rng(seed)
    kz1 = np.fft.fftfreq(nz, d=1.0 / nz)
    ky1 = np.fft.fftfreq(ny, d=1.0 / ny)
    kx1 = np.fft.fftfreq(nx, d=1.0 / nx)
    KZ, KY, KX = np.meshgrid(kz1, ky1, kx1, indexing="ij")
    K2 = KX * KX + KY * KY + KZ * KZ
    K = np.sqrt(K2)
    Ek = K ** 4 * np.exp(-2.0 * (K / k0) ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(K > 0, np.sqrt(Ek / (4.0 * np.pi * np.maximum(K2, 1e-300))), 0.0)
    c = [amp * np.exp(1j * rng.uniform(0.0, TWO_PI, size=K.shape)) for _ in range(3)]
    # solenoidal projection: c <- c - k (k.c)/|k|^2
    with np.errstate(divide="ignore", invalid="ignore"):
        kdotc = (KX * c[0] + KY * c[1] + KZ * c[2]) / np.where(K2 > 0, K2, 1.0)
    c[0] -= KX * kdotc
    c[1] -= KY * kdotc
    c[2] -= KZ * kdotc
    vel = np.empty((3,) + K.shape)
    for i in range(3):
        vel[i] = np.real(np.fft.ifftn(c[i]))
    del c
    # Nyquist planes make the real part slightly divergent for even n: remove the mean
    vel -= vel.mean(axis=(1, 2, 3), keepdims=True)
    scale = 1.0 / math.sqrt(float(np.mean(np.sum(vel * vel, axis=0))))
    vel *= scale
    # dudx spectrally for the Taylor microscale
    dudx = np.real(np.fft.ifftn(1j * KX * np.fft.fftn(vel[0])))
    uprime = 1.0 / math.sqrt(3.0)
    lam = uprime / math.sqrt(float(np.mean(dudx * dudx)))
    Re = Re_lambda * visc_mu1 / (uprime * lam)
    shp = (nz, ny, nx)
    rho = np.ones(shp)
    p = np.full(shp, 1.0 / (gamma * Mt * Mt))
    U = conserved(rho, vel[0], vel[1], vel[2], p, gamma)
    return U, Re


def ensemble_blocks(nblocks=48, seed=20220930, sizes=(32, 48, 64, 96, 128), mt_range=(0.3, 0.7)):
    """Batched-ensemble workload: block dims drawn i.i.d. per axis from
    `sizes`, block b seeded with seed + b and a turbulent Mach number drawn
    uniformly in mt_range.  Returns a list of dicts (shape (nx, ny, nz), U,
    Re, Mt, metrics)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nblocks):
        nx, ny, nz = (int(x) for x in rng.choice(sizes, size=3))
        mt = float(rng.uniform(*mt_range))
        U, Re = isotropic_turbulence_box(nx, ny, nz, seed + b, Mt=mt)
        out.append(dict(shape=(nx, ny, nz), U=U, Re=Re, Mt=mt, metrics=uniform_metrics(nx, ny, nz)))
    return out


def isentropic_vortex(n, nz=8, gamma=1.4, beta=5.0, L=20.0, t=0.0, mean=(1.0, 1.0)):
    """Isentropic vortex (strength beta) convected by `mean`, on [-L/2, L/2)^2.

    Uses gamma Ma^2 = 1 so that p = rho T.  Returns (U, metrics, Ma, X, Y).
    """
    Ma = 1.0 / math.sqrt(gamma)
    X, Y, Z = box_coords(n, n, nz, L, L, L * nz / n, -L / 2, -L / 2, 0.0)
    xc = X - mean[0] * t
    yc = Y - mean[1] * t
    # periodic images for t > 0
    xc = (xc + L / 2) % L - L / 2
    yc = (yc + L / 2) % L - L / 2
    r2 = xc * xc + yc * yc
    e = np.exp(0.5 * (1.0 - r2))
    u = mean[0] - beta / (2 * math.pi) * e * yc
    v = mean[1] + beta / (2 * math.pi) * e * xc
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    U = conserved(rho, u, v, np.zeros_like(u), p, gamma)
    met = uniform_metrics(n, n, nz, L, L, L * nz / n)
    return U, met, Ma, X, Y


def shock_tube(n, gamma=1.4, x0=0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Sod shock tube on [0, 1] with n nodes including both end nodes.

    Uses gamma Ma^2 = 1 (p = rho T).  Returns (U, metrics, Ma, x).
    """
    Ma = 1.0 / math.sqrt(gamma)
    x = np.linspace(0.0, 1.0, n)
    h = x[1] - x[0]
    rho = np.where(x < x0, left[0], right[0])
    u = np.where(x < x0, left[1], right[1])
    p = np.where(x < x0, left[2], right[2])
    shp = (1, 1, n)
    U = conserved(rho.reshape(shp), u.reshape(shp), np.zeros(shp), np.zeros(shp), p.reshape(shp),
                  gamma)
    met = np.zeros(10)
    met[0], met[4], met[8] = 1.0 / h, 1.0, 1.0
    met[9] = 1.0 / h
    return U, met, Ma, x


# ----------------------------------------------------------------------------
# curvilinear grids
# ----------------------------------------------------------------------------

def _mid_deriv(f, axis):
    """Composite derivative D = delta o I along `axis` of an extended array.

    I is the 8-point midpoint interpolation, delta the two-point difference;
    the result loses 4 nodes at each end of that axis.
    """
    n = f.shape[axis]
    # interface values at m+1/2 for m = 3 .. n-5 (needs m-3..m+4)
    acc = 0.0
    for l in range(8):
        sl = [slice(None)] * f.ndim
        sl[axis] = slice(l, n - 7 + l)
        acc = acc + _MID8[l] * f[tuple(sl)]
    # acc index a <-> interface (a+3)+1/2 ; D at node m = I(m+1/2) - I(m-1/2)
    sl1 = [slice(None)] * f.ndim
    sl0 = [slice(None)] * f.ndim
    sl1[axis] = slice(1, None)
    sl0[axis] = slice(0, -1)
    return acc[tuple(sl1)] - acc[tuple(sl0)]


def _trim(f, axis, k):
    sl = [slice(None)] * f.ndim
    sl[axis] = slice(k, f.shape[axis] - k)
    return f[tuple(sl)]


def wavy_grid(n, amp=0.08, L=TWO_PI, nz=None):
    """Periodic three-dimensional wavy grid with conservative metrics.

    x_a = L (xi_a/n) + amp L sin(2 pi xi_b/n) sin(2 pi xi_c/n) for the other
    two index directions b, c.  The metrics divided by J are built in the
    conservative (Thomas-Lombard) form with the composite operator
    D = delta o I (I: 8-point midpoint interpolation), evaluated on an
    index range extended past the periodic box, so that the discrete
    geometric conservation law holds to round-off.
    Returns (metrics [10][nz][n][n], coords (3, nz, n, n)).
    """
    nzz = n if nz is None else nz
    G = 12
    ii = np.arange(-G, n + G, dtype=np.float64)
    kk = np.arange(-G, nzz + G, dtype=np.float64)
    K, Jx, I = np.meshgrid(kk, ii, ii, indexing="ij")
    sx, sy, sz = I / n, Jx / n, K / nzz
    tp = TWO_PI
    x = L * sx + amp * L * np.sin(tp * sy) * np.sin(tp * sz)
    y = L * sy + amp * L * np.sin(tp * sx) * np.sin(tp * sz)
    z = (L * nzz / n) * sz + amp * L * np.sin(tp * sx) * np.sin(tp * sy)
    X = [x, y, z]
    ax = {0: 2, 1: 1, 2: 0}       # index direction -> array axis (k, j, i)

    def D(f, d):
        return _mid_deriv(f, ax[d])

    def trim_all(f, k):
        for a in range(3):
            f = _trim(f, a, k)
        return f

    # first derivatives of the coordinates, trimmed to a common shape
    dX = [[None] * 3 for _ in range(3)]   # dX[a][d] = d x_a / d xi_d
    for a in range(3):
        for d in range(3):
            g = D(X[a], d)
            # g lost 4 on axis ax[d] only: trim 4 on the other axes
            for e in range(3):
                if e != d:
                    g = _trim(g, ax[e], 4)
            dX[a][d] = g
    Xt = [trim_all(X[a], 4) for a in range(3)]
    met = np.zeros((10, nzz, n, n))
    # metric/J for coordinate a, direction d: cyclic (a, b, c), (d, e, f)
    for d in range(3):
        e, f = (d + 1) % 3, (d + 2) % 3
        for a in range(3):
            b, c = (a + 1) % 3, (a + 2) % 3
            # d_{x_a}/J = (x_b,e x_c)_f - (x_b,f x_c)_e  (conservative form)
            t1 = D(dX[b][e] * Xt[c], f)
            t2 = D(dX[b][f] * Xt[c], e)
            # trim to the common core: t1 lost 4 along f, t2 lost 4 along e
            t1 = _trim(_trim(t1, ax[d], 4), ax[e], 4)
            t2 = _trim(_trim(t2, ax[d], 4), ax[f], 4)
            core = t1 - t2
            core = trim_all(core, G - 8)
            met[3 * d + a] = core
    # J^-1 = det(dx/dxi) with the same first derivatives
    A = [[trim_all(dX[a][d], G - 4) for d in range(3)] for a in range(3)]
    detJ = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
            - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
            + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]))
    Jac = 1.0 / detJ
    for e in range(9):
        met[e] = met[e] * Jac
    met[9] = Jac
    coords = np.stack([trim_all(X[a], G) for a in range(3)])
    return np.ascontiguousarray(met), coords


def ramp_grid(nx, ny, nz, angle_deg, x_start=-20.0, x_end=15.0, H=10.0, dy_wall=3.3e-3,
              Lz=4.0):
    """Synthetic body-fitted grid over a compression ramp with a sharp corner at x = 0.

    xi along the wall (uniform in x), vertical eta lines from the wall
    y_w(x) to y_w(x) + H with tanh clustering so that the first spacing is
    dy_wall, zeta periodic over Lz.  Returns (metrics2d [10][ny][nx],
    x2d, y2d, z1d, wall_x).  Metrics use second-order central differences
    (one-sided at the edges) of the coordinates.
    """
    x = np.linspace(x_start, x_end, nx)
    tana = math.tan(math.radians(angle_deg))
    yw = np.where(x > 0.0, x * tana, 0.0)
    # tanh stretching s(t) = 1 + tanh(b (t - 1))/tanh(b), first step = dy_wall/H
    t = np.linspace(0.0, 1.0, ny)

    def first(b):
        return 1.0 + math.tanh(b * (t[1] - 1.0)) / math.tanh(b)

    lo, hi = 1e-3, 20.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if first(mid) * H > dy_wall:
            lo = mid
        else:
            hi = mid
    b = 0.5 * (lo + hi)
    s = 1.0 + np.tanh(b * (t - 1.0)) / math.tanh(b)
    X2 = np.broadcast_to(x[None, :], (ny, nx)).copy()
    Y2 = yw[None, :] + H * s[:, None]
    hz = Lz / nz
    xxi = np.gradient(X2, axis=1, edge_order=2)
    yxi = np.gradient(Y2, axis=1, edge_order=2)
    xet = np.gradient(X2, axis=0, edge_order=2)
    yet = np.gradient(Y2, axis=0, edge_order=2)
    det2 = xxi * yet - xet * yxi
    jinv = det2 * hz                      # J^-1 = z_zeta (x_xi y_eta - x_eta y_xi)
    J = 1.0 / jinv
    met = np.zeros((10, ny, nx))
    met[0] = J * yet * hz                 # xi_x
    met[1] = -J * xet * hz                # xi_y
    met[3] = -J * yxi * hz                # eta_x
    met[4] = J * xxi * hz                 # eta_y
    met[8] = J * det2                     # zeta_z
    met[9] = J
    z = np.arange(nz) * hz
    return np.ascontiguousarray(met), X2, Y2, z, x


def ramp_inflow(y_rel, Ma, gamma=1.4, Tw=2.8, Pr=0.72, delta=1.0):
    """Inflow profile on the ramp grid: u = tanh(3 y/delta), Crocco-Busemann T.

    Returns (rho, u, v, w, p) arrays over the wall distance y_rel, with
    rho_inf = T_inf = U_inf = 1 and p = 1/(gamma Ma^2).
    """
    r = Pr ** (1.0 / 3.0)
    Tr = 1.0 + r * (gamma - 1.0) / 2.0 * Ma * Ma
    ub = np.tanh(3.0 * np.asarray(y_rel) / delta)
    T = Tw + (Tr - Tw) * ub - (Tr - 1.0) * ub * ub
    p = np.full_like(ub, 1.0 / (gamma * Ma * Ma))
    rho = gamma * Ma * Ma * p / T
    return rho, ub, np.zeros_like(ub), np.zeros_like(ub), p


def oblique_shock(Ma, angle_deg, gamma=1.4):
    """Weak attached oblique shock from a wedge of the given angle in a
    uniform stream (rho = T = U = 1, p = 1/(gamma Ma^2)): the theta-beta-Mach
    relation solved by bisection for the weak shock angle beta, then the
    normal-shock jump conditions on the normal Mach number M sin(beta).
    Returns (beta, rho2, speed2, p2)."""
    theta = math.radians(angle_deg)

    def turn(b):
        return math.atan(2.0 / math.tan(b) * (Ma * Ma * math.sin(b) ** 2 - 1.0)
                         / (Ma * Ma * (gamma + math.cos(2.0 * b)) + 2.0))

    lo, hi = math.asin(1.0 / Ma), 0.5 * math.pi
    grid = np.linspace(lo, hi, 4001)[1:-1]
    bmax = grid[int(np.argmax([turn(b) for b in grid]))]
    if turn(bmax) < theta:
        raise ValueError("detached shock: no weak solution for this angle and Mach number")
    hi = bmax
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if turn(mid) < theta:
            lo = mid
        else:
            hi = mid
    beta = 0.5 * (lo + hi)
    mn2 = (Ma * math.sin(beta)) ** 2
    rho2 = (gamma + 1.0) * mn2 / ((gamma - 1.0) * mn2 + 2.0)
    p2 = (1.0 + 2.0 * gamma / (gamma + 1.0) * (mn2 - 1.0)) / (gamma * Ma * Ma)
    vt = math.cos(beta)
    vn = math.sin(beta) / rho2
    return beta, rho2, math.hypot(vt, vn), p2


def ramp_case(nx, ny, nz, angle_deg, Ma, gamma=1.4, Tw=2.8, Pr=0.72):
    """Ramp grid plus the initial condition and the inflow profile.

    Initial field: the inviscid solution of the ramp (the free stream
    upstream of the weak oblique shock from the corner, the uniform
    post-shock state parallel to the ramp face below it) with a boundary
    layer of the inflow profile's shape in the wall distance along each
    vertical grid line: u/u_e = tanh(3 d), Crocco-Busemann temperature
    between T_wall and the local edge state, uniform pressure across it.
    Starting from the inviscid solution avoids the strong starting vortex
    that an impulsive start into the ramp face produces at Mach 6."""
    met2, X2, Y2, z, wx = ramp_grid(nx, ny, nz, angle_deg)
    yw = Y2[0:1, :]
    yrel = Y2 - yw
    beta, rho2, q2, p2 = oblique_shock(Ma, angle_deg, gamma)
    pinf = 1.0 / (gamma * Ma * Ma)
    behind = (X2 > 0.0) & (Y2 < X2 * math.tan(beta))
    a = np.where(behind, math.radians(angle_deg), 0.0)
    qe = np.where(behind, q2, 1.0)
    pe = np.where(behind, p2, pinf)
    Te = np.where(behind, gamma * Ma * Ma * p2 / rho2, 1.0)
    Me2 = qe * qe * Ma * Ma / Te               # c^2 = T/Ma^2
    r = Pr ** (1.0 / 3.0)
    Tr = Te * (1.0 + r * (gamma - 1.0) / 2.0 * Me2)
    f = np.tanh(3.0 * yrel)
    T = Tw + (Tr - Tw) * f - (Tr - Te) * f * f
    rho = gamma * Ma * Ma * pe / T
    u, v = qe * f * np.cos(a), qe * f * np.sin(a)
    shp = (nz, ny, nx)
    U = conserved(*(np.broadcast_to(q[None], shp) for q in (rho, u, v, np.zeros_like(u), pe)), gamma)
    inflow = np.stack(ramp_inflow(yrel[:, 0], Ma, gamma, Tw, Pr))
    return dict(U=U, metrics2d=met2, inflow=np.ascontiguousarray(inflow), wall_x=wx, wall_z=z,
                X=X2, Y=Y2, shock_angle=beta)
