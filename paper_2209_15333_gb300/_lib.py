"""Thin ctypes binding of the C ABI in include/cfd.h (argument marshalling only).

Every step of the right-hand side and the RK3 update runs in the CUDA library
``_build/libcfd_gb300.so``; there is no CPU path here.  Loading fails loudly
when the library has not been built.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# CFD_GB300_LIB selects another build of the same library (the bounds-checked
# one in its test); there is no fallback when the library is missing
LIB_PATH = os.environ.get("CFD_GB300_LIB") or os.path.join(HERE, "_build", "libcfd_gb300.so")

CFD_OK, CFD_EINVAL, CFD_ENOMEM, CFD_ECUDA, CFD_ENONPHYS, CFD_ETIMEOUT, CFD_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
BC_PERIODIC, BC_WALL_ISOTHERMAL, BC_INFLOW, BC_OUTFLOW_EXTRAP, BC_HALO, BC_NONREFLECT = 0, 1, 2, 3, 4, 5
HALO_WIDTH = 8
METRICS_3D, METRICS_2D, METRICS_UNIFORM = 0, 1, 2
SUTHERLAND, POWER = 0, 1
UD7, WENO5, WENO7, HYBRID = 0, 1, 2, 3
METRIC_NODAL, METRIC_FSP = 0, 1
FP64, FP32_BULK = 0, 1
SENSOR_PLAIN, SENSOR_MLP = 0, 1

STATUS_NAMES = {0: "CFD_OK", -1: "CFD_EINVAL", -2: "CFD_ENOMEM", -3: "CFD_ECUDA", -4: "CFD_ENONPHYS",
                -5: "CFD_ETIMEOUT", -6: "CFD_EUNSUPPORTED"}

# every entry point declared in include/cfd.h
EXPORTS = ["cfd_default_params", "cfd_create", "cfd_create_batch", "cfd_set_inflow", "cfd_set_blowing", "cfd_set_state",
           "cfd_get_state", "cfd_rhs", "cfd_step", "cfd_cfl_dt", "cfd_get_flags", "cfd_force_flags",
           "cfd_get_time", "cfd_set_time", "cfd_sync", "cfd_last_error", "cfd_launch_count", "cfd_fma_peak",
           "cfd_check_conversions", "cfd_eval_viscosity", "cfd_profile_stage", "cfd_rhs_noalloc", "cfd_set_sweep_variant", "cfd_get_sweep_variant",
           "cfd_set_sensor_mlp", "cfd_sensor_features", "cfd_sensor_fallbacks", "cfd_set_halo_links",
           "cfd_destroy"]


class CfdGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc_lo", C.c_int * 3),
                ("bc_hi", C.c_int * 3), ("metric_layout", C.c_int)]


class CfdParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("Re", C.c_double), ("Ma", C.c_double), ("Pr", C.c_double),
                ("T_wall", C.c_double), ("T_ref", C.c_double), ("visc_law", C.c_int),
                ("visc_omega", C.c_double), ("scheme", C.c_int), ("theta1", C.c_double),
                ("theta2", C.c_double), ("visc_order", C.c_int), ("metric_mode", C.c_int),
                ("precision", C.c_int), ("sensor", C.c_int), ("weno_eps", C.c_double),
                ("recon_vars", C.c_int)]


class CfdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run paper_2209_15333_gb300/build.py" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, dp, ucp = C.c_void_p, C.POINTER(C.c_double), C.c_void_p
        L.cfd_default_params.argtypes = [C.POINTER(CfdParams)]
        L.cfd_default_params.restype = None
        L.cfd_create.argtypes = [C.POINTER(vp), C.POINTER(CfdGrid), vp, C.c_int, C.POINTER(CfdParams), vp]
        L.cfd_create_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(CfdGrid), C.POINTER(vp), C.c_int,
                                       C.POINTER(CfdParams), vp]
        L.cfd_set_inflow.argtypes = [vp, vp]
        L.cfd_set_blowing.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                      C.c_double, vp, vp]
        L.cfd_set_state.argtypes = [vp, C.c_int, vp, C.c_int]
        L.cfd_get_state.argtypes = [vp, C.c_int, vp, C.c_int]
        L.cfd_rhs.argtypes = [vp, C.c_int, vp, C.c_int]
        L.cfd_step.argtypes = [vp, C.c_double, C.c_int]
        L.cfd_cfl_dt.argtypes = [vp, C.c_int, C.c_double, dp]
        L.cfd_get_flags.argtypes = [vp, C.c_int, ucp, C.c_int]
        L.cfd_force_flags.argtypes = [vp, C.c_int, ucp, C.c_int]
        L.cfd_get_time.argtypes = [vp, dp]
        L.cfd_set_time.argtypes = [vp, C.c_double]
        L.cfd_sync.argtypes = [vp, C.c_double]
        L.cfd_last_error.argtypes = [vp]
        L.cfd_last_error.restype = C.c_char_p
        L.cfd_launch_count.argtypes = [vp]
        L.cfd_launch_count.restype = C.c_longlong
        L.cfd_fma_peak.argtypes = [C.c_int, dp]
        L.cfd_check_conversions.argtypes = [C.POINTER(C.c_ulonglong)]
        L.cfd_eval_viscosity.argtypes = [C.POINTER(CfdParams), vp, vp, C.c_int]
        L.cfd_profile_stage.argtypes = [vp, C.c_int, dp]
        L.cfd_set_sensor_mlp.argtypes = [vp, vp, vp, C.c_float]
        L.cfd_sensor_features.argtypes = [vp, C.c_int, vp, C.c_int]
        L.cfd_sensor_fallbacks.argtypes = [vp, C.POINTER(C.c_ulonglong)]
        L.cfd_set_sweep_variant.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.cfd_get_sweep_variant.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.cfd_rhs_noalloc.argtypes = [C.POINTER(CfdGrid), C.POINTER(CfdParams), vp, vp, vp, vp]
        L.cfd_set_halo_links.argtypes = [vp, vp]
        L.cfd_destroy.argtypes = [vp]
        L.cfd_destroy.restype = None
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("cfd_default_params", "cfd_last_error", "cfd_launch_count", "cfd_destroy"):
                f.restype = C.c_int
        _lib = L
    return _lib


def check(status, ctx=None):
    if status != CFD_OK:
        msg = lib().cfd_last_error(ctx).decode()
        raise CfdError(status, msg)


def check_conversions():
    """Device self-check of the integer-pipe binary64 <-> binary32
    conversions (cfd_check_conversions): dict of the five counts."""
    out = (C.c_ulonglong * 5)()
    check(lib().cfd_check_conversions(out))
    keys = ("floats", "f2d_mismatch", "doubles_ok", "d2f_mismatch", "ok_flag_wrong")
    return dict(zip(keys, (int(v) for v in out)))


def eval_viscosity(T, **params):
    """mu(T) on the device by the viscous kernels' routine (cfd_eval_viscosity)."""
    import numpy as np
    T = np.ascontiguousarray(T, dtype=np.float64)
    mu = np.empty_like(T)
    p = default_params(**params)
    check(lib().cfd_eval_viscosity(C.byref(p), C.c_void_p(T.ctypes.data), C.c_void_p(mu.ctypes.data), T.size))
    return mu


def default_params(**kw):
    p = CfdParams()
    lib().cfd_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def make_grid(nx, ny, nz, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), metric_layout=METRICS_3D):
    g = CfdGrid()
    g.nx, g.ny, g.nz = nx, ny, nz
    for d in range(3):
        g.bc_lo[d], g.bc_hi[d] = bc_lo[d], bc_hi[d]
    g.metric_layout = metric_layout
    return g
