"""cfd_rhs_noalloc: the allocation-free right-hand side, for callers that
cannot call cudaMalloc (their device memory belongs to another allocator or
budget, or they must not stall the device the way cudaFree does).

Called through the C ABI with caller-owned device buffers and compared, on
consecutive calls, with the context-based cfd_rhs and with the FP64 oracle
(so that contents the shared scratch array keeps from one call cannot leak
into the next, and so that a fault shared by both GPU entry points is still
caught).  The cases cover periodic boxes and a walled curved ramp grid whose
state already carries its boundary values (the call applies no boundary
conditions).  This file is collected last; it passes alone in a fresh process
and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import field_rel_err, turbulence_field

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()
    return torch


def _case(name, orc=None):
    """(shape, metrics, params, U, bc_lo, bc_hi) of a case; U already carries
    its boundary values."""
    if name == "ramp_walls":
        nx, ny, nz = 40, 24, 8
        rc = cases.ramp_case(nx, ny, nz, 24.0, 2.9, Tw=2.8)
        params = dict(scheme=3, Re=2000.0, Ma=2.9, T_wall=2.8, visc_law=0, T_ref=108.1)
        bc_lo, bc_hi = (2, 1, 0), (3, 3, 0)
        U = rc["U"].copy()
        rng = np.random.default_rng(11)
        U[1:4] += 0.01 * rng.standard_normal(U[1:4].shape) * U[0]
        c = orc.Case(nx, ny, nz, Ma=2.9, T_wall=2.8, visc_law=0, T_ref=108.1, Re=2000.0, scheme=3,
                     bc_lo=bc_lo, bc_hi=bc_hi, inflow=rc["inflow"])
        U = orc.apply_bc(c, cases.expand_metrics(rc["metrics2d"], (nz, ny, nx)), U)
        return (nx, ny, nz), rc["metrics2d"], params, U, bc_lo, bc_hi
    return _periodic_case(name) + ((0, 0, 0), (0, 0, 0))


def _periodic_case(name):
    if name == "tgv32_hybrid":
        n = 32
        return (n, n, n), cases.uniform_metrics(n, n, n), dict(scheme=3, Re=400.0, theta1=0.004,
                                                               theta2=0.012), cases.taylor_green(n)
    if name == "wavy_weno7":
        n = 20
        met, _ = cases.wavy_grid(n, amp=0.05)
        return (n, n, n), met, dict(scheme=2, Re=150.0, visc_law=0, T_ref=108.1), turbulence_field((n, n, n), 41)
    if name == "ragged_ud7_inviscid":
        sh = (29, 13, 17)
        return sh, cases.uniform_metrics(*sh), dict(scheme=0, Re=0.0), turbulence_field(sh, 42)
    raise KeyError(name)


def _noalloc(torch, shape, met, params, U, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0)):
    from paper_2209_15333_gb300 import _lib as L
    nx, ny, nz = shape
    m = np.asarray(met)
    layout = {1: L.METRICS_UNIFORM, 3: L.METRICS_2D, 4: L.METRICS_3D}[m.ndim]
    grid = L.make_grid(nx, ny, nz, bc_lo=bc_lo, bc_hi=bc_hi, metric_layout=layout)
    prm = L.default_params(**params)
    dm = torch.tensor(m, device="cuda", dtype=torch.float64).contiguous()
    dU = torch.tensor(U, device="cuda", dtype=torch.float64).contiguous()
    dL = torch.full_like(dU, float("nan"))
    stream = torch.cuda.current_stream()
    st = L.lib().cfd_rhs_noalloc(C.byref(grid), C.byref(prm), C.c_void_p(dm.data_ptr()), C.c_void_p(dU.data_ptr()),
                                 C.c_void_p(dL.data_ptr()), C.c_void_p(stream.cuda_stream))
    L.check(st)
    stream.synchronize()
    return dL.cpu().numpy()


def _with_context(shape, met, params, U, bc_lo, bc_hi):
    from paper_2209_15333_gb300.solver import Solver
    with Solver(shape, met, bc_lo=bc_lo, bc_hi=bc_hi, **params) as s:
        s.set_state(U)
        return s.rhs()


def _oracle(orc, shape, met, params, U, bc_lo, bc_hi):
    nx, ny, nz = shape
    c = orc.Case(nx, ny, nz, bc_lo=bc_lo, bc_hi=bc_hi, **params)
    return orc.rhs(c, cases.expand_metrics(met, (nz, ny, nx)), U)


def test_noalloc_matches_context_rhs_and_oracle_on_consecutive_calls(torch_cuda, orc):
    for name in ("tgv32_hybrid", "ramp_walls", "wavy_weno7", "ragged_ud7_inviscid", "ramp_walls", "tgv32_hybrid"):
        shape, met, params, U, lo, hi = _case(name, orc)
        got = _noalloc(torch_cuda, shape, met, params, U, lo, hi)
        assert np.isfinite(got).all(), name
        ref = _with_context(shape, met, params, U, lo, hi)
        assert field_rel_err(got, ref) <= TOL, name
        ora = _oracle(orc, shape, met, params, U, lo, hi)
        assert field_rel_err(got, ora) <= TOL, name


def test_noalloc_allocates_no_device_memory(torch_cuda, orc):
    """After a first call (its one-time set-up, and the lazy loading of its
    kernels), further calls leave the device's free memory unchanged (the
    test's own buffers come back from torch's caching allocator)."""
    shape, met, params, U, lo, hi = _case("ramp_walls", orc)
    _noalloc(torch_cuda, shape, met, params, U, lo, hi)
    torch_cuda.cuda.synchronize()
    free0 = torch_cuda.cuda.mem_get_info()[0]
    for _ in range(3):
        _noalloc(torch_cuda, shape, met, params, U, lo, hi)
    torch_cuda.cuda.synchronize()
    assert torch_cuda.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_the_learned_sensor(torch_cuda):
    """The call holds no network weights: asking for the learned sensor is an
    error, not a silent switch to the plain sensor."""
    from paper_2209_15333_gb300 import _lib as L
    n = 16
    grid = L.make_grid(n, n, n, metric_layout=L.METRICS_UNIFORM)
    prm = L.default_params(sensor=L.SENSOR_MLP)
    dummy = torch_cuda.zeros(5 * n ** 3, device="cuda", dtype=torch_cuda.float64)
    p = C.c_void_p(dummy.data_ptr())
    st = L.lib().cfd_rhs_noalloc(C.byref(grid), C.byref(prm), p, p, p, None)
    assert st == L.CFD_EUNSUPPORTED
    assert b"learned-sensor" in L.lib().cfd_last_error(None)


def test_noalloc_rejects_grids_beyond_the_limit(torch_cuda):
    from paper_2209_15333_gb300 import _lib as L
    n = 33  # 33^3 > CFD_NOALLOC_MAX_NODES = 32^3
    grid = L.make_grid(n, n, n, metric_layout=L.METRICS_UNIFORM)
    prm = L.default_params()
    dummy = torch_cuda.zeros(8, device="cuda", dtype=torch_cuda.float64)
    p = C.c_void_p(dummy.data_ptr())
    st = L.lib().cfd_rhs_noalloc(C.byref(grid), C.byref(prm), p, p, p, None)
    assert st == L.CFD_ENOMEM
    assert b"CFD_NOALLOC_MAX_NODES" in L.lib().cfd_last_error(None)
