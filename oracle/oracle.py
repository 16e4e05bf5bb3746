"""ctypes binding of the C oracle (test infrastructure only).

Arrays are numpy float64, structure-of-arrays ``[var][nz][ny][nx]``.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

BC_PERIODIC, BC_WALL, BC_INFLOW, BC_OUTFLOW, BC_NONREFLECT = 0, 1, 2, 3, 5
SUTHERLAND, POWER = 0, 1
UD7, WENO5, WENO7, HYBRID = 0, 1, 2, 3
METRIC_NODAL, METRIC_FSP = 0, 1
RECON_COMPONENT, RECON_CHARACTERISTIC = 0, 1

_dp = C.POINTER(C.c_double)
_ucp = C.POINTER(C.c_ubyte)


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
        ("gamma", C.c_double), ("Re", C.c_double), ("Ma", C.c_double), ("Pr", C.c_double),
        ("T_wall", C.c_double), ("T_ref", C.c_double),
        ("visc_law", C.c_int), ("visc_omega", C.c_double),
        ("scheme", C.c_int), ("theta1", C.c_double), ("theta2", C.c_double),
        ("visc_order", C.c_int), ("metric_mode", C.c_int), ("weno_eps", C.c_double),
        ("nthreads", C.c_int),
        ("forced_cls", _ucp), ("inflow", _dp),
        ("blow_amp", C.c_double), ("blow_x0", C.c_double), ("blow_x1", C.c_double),
        ("blow_omega", C.c_double), ("blow_Lz", C.c_double), ("blow_m", C.c_int),
        ("wall_x", _dp), ("wall_z", _dp),
        ("recon_vars", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER(OrcParams)
        L.orc_primitives.argtypes = [P, _dp, _dp]
        L.orc_sensor.argtypes = [P, _dp, _dp, _ucp]
        L.orc_rhs.argtypes = [P, _dp, _dp, _dp, _ucp]
        L.orc_apply_bc.argtypes = [P, _dp, _dp, C.c_double]
        L.orc_rk3_stage.argtypes = [C.c_int, C.c_long, _dp, _dp, _dp, C.c_double, _dp]
        L.orc_step.argtypes = [P, _dp, _dp, C.c_double, C.c_int, C.c_double]
        L.orc_cfl_dt.argtypes = [P, _dp, _dp, C.c_double]
        L.orc_cfl_dt.restype = C.c_double
        L.orc_sw_split.argtypes = [C.c_double] * 9 + [_dp, _dp]
        L.orc_ud7.argtypes = [_dp]
        L.orc_ud7.restype = C.c_double
        L.orc_weno_tables.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
        L.orc_weno.argtypes = [C.c_int, _dp, C.POINTER(C.c_int), C.c_double, C.c_double, _dp]
        L.orc_weno.restype = C.c_double
        L.orc_weno_beta.argtypes = [C.c_int, C.c_int, _dp]
        L.orc_weno_beta.restype = C.c_double
        L.orc_char_matrices.argtypes = [C.c_double, _dp, _dp, _dp, _dp]
        L.orc_central_deriv.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp]
        L.orc_midpoint_weights.argtypes = [_dp]
        L.orc_viscosity.argtypes = [P, C.c_double]
        L.orc_viscosity.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Case:
    """Problem description handed to the oracle (grid, gas, scheme, BCs).

    Keeps the numpy arrays referenced by the C struct alive.
    """

    def __init__(self, nx, ny, nz, *, gamma=1.4, Re=0.0, Ma=0.5, Pr=0.72, T_wall=1.0, T_ref=288.15,
                 visc_law=POWER, visc_omega=0.76, scheme=UD7, theta1=0.02, theta2=0.1,
                 visc_order=8, metric_mode=METRIC_NODAL, weno_eps=1e-6, bc_lo=(0, 0, 0),
                 bc_hi=(0, 0, 0), nthreads=0, forced_cls=None, inflow=None, blowing=None,
                 recon_vars=RECON_COMPONENT):
        p = OrcParams()
        p.nx, p.ny, p.nz = nx, ny, nz
        for d in range(3):
            p.bc_lo[d] = bc_lo[d]
            p.bc_hi[d] = bc_hi[d]
        p.gamma, p.Re, p.Ma, p.Pr, p.T_wall, p.T_ref = gamma, Re, Ma, Pr, T_wall, T_ref
        p.visc_law, p.visc_omega = visc_law, visc_omega
        p.scheme, p.theta1, p.theta2 = scheme, theta1, theta2
        p.visc_order, p.metric_mode, p.weno_eps = visc_order, metric_mode, weno_eps
        p.nthreads = nthreads
        p.recon_vars = recon_vars
        self._keep = []
        if forced_cls is not None:
            fc = np.ascontiguousarray(forced_cls, dtype=np.uint8).ravel()
            self._keep.append(fc)
            p.forced_cls = fc.ctypes.data_as(_ucp)
        if inflow is not None:
            inf = _f64(inflow)
            assert inf.shape == (5, ny)
            self._keep.append(inf)
            p.inflow = _ptr(inf)
        if blowing is not None:
            wx = _f64(blowing["wall_x"])
            wz = _f64(blowing["wall_z"])
            self._keep += [wx, wz]
            p.blow_amp = blowing["amp"]
            p.blow_x0, p.blow_x1 = blowing["x0"], blowing["x1"]
            p.blow_omega, p.blow_Lz, p.blow_m = blowing["omega"], blowing["Lz"], blowing["m"]
            p.wall_x, p.wall_z = _ptr(wx), _ptr(wz)
        self.p = p
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz

    def ref(self):
        return C.byref(self.p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with %d" % (what, rc))


def primitives(case, U):
    U = _f64(U)
    out = np.empty((7,) + case.shape)
    _check(lib().orc_primitives(case.ref(), _ptr(U), _ptr(out)), "primitives")
    return out


def sensor(case, U):
    U = _f64(U)
    th = np.empty(case.shape)
    cls = np.empty(case.shape, dtype=np.uint8)
    _check(lib().orc_sensor(case.ref(), _ptr(U), _ptr(th), cls.ctypes.data_as(_ucp)), "sensor")
    return th, cls


def rhs(case, metrics, U, return_cls=False):
    U = _f64(U)
    M = _f64(metrics)
    L = np.empty_like(U)
    cls = np.zeros(case.shape, dtype=np.uint8)
    _check(lib().orc_rhs(case.ref(), _ptr(M), _ptr(U), _ptr(L), cls.ctypes.data_as(_ucp)), "rhs")
    return (L, cls) if return_cls else L


def apply_bc(case, metrics, U, t=0.0):
    U = _f64(U).copy()
    _check(lib().orc_apply_bc(case.ref(), _ptr(_f64(metrics)), _ptr(U), t), "apply_bc")
    return U


def rk3_stage(stage, Un, Uk, L, dt):
    Un, Uk, L = _f64(Un), _f64(Uk), _f64(L)
    out = np.empty_like(Un)
    _check(lib().orc_rk3_stage(stage, Un.size, _ptr(Un), _ptr(Uk), _ptr(L), dt, _ptr(out)), "rk3")
    return out


def step(case, metrics, U, dt, nsteps=1, t0=0.0):
    U = _f64(U).copy()
    _check(lib().orc_step(case.ref(), _ptr(_f64(metrics)), _ptr(U), dt, nsteps, t0), "step")
    return U


def cfl_dt(case, metrics, U, cfl=0.5):
    return lib().orc_cfl_dt(case.ref(), _ptr(_f64(metrics)), _ptr(_f64(U)), cfl)


def sw_split(gamma, rho, u, v, w, c, a1, a2, a3):
    fp = np.empty(5)
    fm = np.empty(5)
    lib().orc_sw_split(gamma, rho, u, v, w, c, a1, a2, a3, _ptr(fp), _ptr(fm))
    return fp, fm


def ud7(a):
    a = _f64(a)
    assert a.size == 7
    return lib().orc_ud7(_ptr(a))


def weno_tables(r):
    c = np.empty((r, r))
    d = np.empty(r)
    Q = np.empty((r, r, r))
    cf = np.empty(2 * r - 1)
    _check(lib().orc_weno_tables(r, _ptr(c), _ptr(d), _ptr(Q), _ptr(cf)), "weno_tables")
    return c, d, Q, cf


def weno(r, a, mask=None, eps=1e-6, return_omega=False, scale=1.0):
    a = _f64(a)
    assert a.size == 2 * r - 1
    om = np.empty(r)
    mptr = None
    if mask is not None:
        m = (C.c_int * r)(*[int(x) for x in mask])
        mptr = C.cast(m, C.POINTER(C.c_int))
    v = lib().orc_weno(r, _ptr(a), mptr, eps, scale, _ptr(om))
    return (v, om) if return_omega else v


def char_matrices(gamma, U, n):
    """(S, S^-1) of Sec. 2.2.2 (Eq. 34-40) at conserved state U, normal n."""
    U, n = _f64(U), _f64(n)
    S, Si = np.empty((5, 5)), np.empty((5, 5))
    _check(lib().orc_char_matrices(gamma, _ptr(U), _ptr(n), _ptr(S), _ptr(Si)), "char_matrices")
    return S, Si


def weno_beta(r, k, a):
    a = _f64(a)
    return lib().orc_weno_beta(r, k, _ptr(a))


def central_deriv(order, g, periodic):
    g = _f64(g)
    out = np.empty_like(g)
    _check(lib().orc_central_deriv(order, g.size, int(periodic), _ptr(g), _ptr(out)), "central")
    return out


def midpoint_weights():
    w = np.empty(8)
    lib().orc_midpoint_weights(_ptr(w))
    return w


def viscosity(case, T):
    return lib().orc_viscosity(case.ref(), T)


def nthreads_default():
    return os.cpu_count() or 1
