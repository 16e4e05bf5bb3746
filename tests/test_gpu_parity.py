"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerance: field-max relative error <= 1e-11 on the
conserved variables (and on L(U)); sensor classes bit-exact."""
import math

import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import field_rel_err, make_pair, turbulence_field

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()
    torch.cuda.init()


def _box(shape):
    nx, ny, nz = shape
    return cases.uniform_metrics(nx, ny, nz)


def rhs_case(name, orc):
    """(solver, case, metrics, U) for a named parity configuration."""
    if name == "tgv32_ud7":
        s, c, M = make_pair(orc, (32, 32, 32), _box((32, 32, 32)), scheme="UD7", Re=400.0)
        return s, c, M, cases.taylor_green(32)
    if name == "ragged_hybrid_v6":
        sh = (37, 19, 23)
        s, c, M = make_pair(orc, sh, _box(sh), scheme="HYBRID", Re=200.0, visc_order=6, theta1=0.004,
                            theta2=0.012)
        return s, c, M, turbulence_field(sh, 1)
    if name == "ragged_weno5_inviscid":
        sh = (29, 33, 17)
        s, c, M = make_pair(orc, sh, _box(sh), scheme="WENO5", Re=0.0)
        return s, c, M, turbulence_field(sh, 2)
    if name == "ragged_weno7_sutherland":
        sh = (41, 13, 26)
        s, c, M = make_pair(orc, sh, _box(sh), scheme="WENO7", Re=150.0, visc_law=0, T_ref=108.1)
        return s, c, M, turbulence_field(sh, 3)
    if name == "wavy_3d_metrics":
        n = 20
        met, _ = cases.wavy_grid(n, amp=0.05)
        s, c, M = make_pair(orc, (n, n, n), met, scheme="HYBRID", Re=300.0, theta1=0.004, theta2=0.012)
        return s, c, M, turbulence_field((n, n, n), 4)
    if name == "long_x_tiles":
        sh = (300, 3, 5)
        s, c, M = make_pair(orc, sh, _box(sh), scheme="HYBRID", Re=100.0, theta1=0.004, theta2=0.012)
        return s, c, M, turbulence_field(sh, 5)
    if name == "two_d_nz1":
        sh = (24, 40, 1)
        s, c, M = make_pair(orc, sh, _box(sh), scheme="UD7", Re=80.0)
        return s, c, M, turbulence_field(sh, 6)
    if name == "all_outflow_3d_metrics":
        sh = (22, 12, 10)
        n = 22
        met, _ = cases.wavy_grid(n, amp=0.04)
        met = np.ascontiguousarray(met[:, :10, :12, :22])
        s, c, M = make_pair(orc, sh, met, scheme="HYBRID", Re=120.0, bc_lo=(3, 3, 3), bc_hi=(3, 3, 3),
                            theta1=0.004, theta2=0.012)
        U = turbulence_field(sh, 7)
        return s, c, M, U
    if name == "ramp_walls":
        return ramp_pair(orc)
    if name == "ramp_nonreflect":
        # the outlet and the top characteristic non-reflecting boundaries
        return ramp_pair(orc, bc_hi=(5, 5, 0))
    raise KeyError(name)


def ramp_pair(orc, nx=40, ny=24, nz=8, blowing=True, bc_hi=(3, 3, 0)):
    rc = cases.ramp_case(nx, ny, nz, 24.0, 2.9, Tw=2.8)
    bl = None
    if blowing:
        bl = dict(amp=0.05, x0=-15.0, x1=-10.0, omega=2.0, m=1, Lz=4.0, wall_x=rc["wall_x"], wall_z=rc["wall_z"])
    s, c, M = make_pair(orc, (nx, ny, nz), rc["metrics2d"], scheme="HYBRID", Re=2000.0, Ma=2.9, T_wall=2.8,
                        visc_law=0, T_ref=108.1, bc_lo=(2, 1, 0), bc_hi=bc_hi, inflow=rc["inflow"], blowing=bl)
    U = rc["U"].copy()
    # a smooth disturbance so that all terms are exercised
    rng = np.random.default_rng(11)
    U[1:4] += 0.01 * rng.standard_normal(U[1:4].shape) * U[0]
    return s, c, M, U


RHS_CASES = ["tgv32_ud7", "ragged_hybrid_v6", "ragged_weno5_inviscid", "ragged_weno7_sutherland", "wavy_3d_metrics",
             "long_x_tiles", "two_d_nz1", "all_outflow_3d_metrics", "ramp_walls", "ramp_nonreflect"]


@pytest.mark.parametrize("name", RHS_CASES)
def test_rhs_parity(orc, name):
    s, c, M, U = rhs_case(name, orc)
    with s:
        s.set_state(U)
        Ub = orc.apply_bc(c, M, U)
        Ug = s.get_state()
        assert field_rel_err(Ug, Ub) <= TOL
        Lg = s.rhs()
        Lo, co = orc.rhs(c, M, Ub, return_cls=True)
        if c.p.scheme == 3:
            assert np.array_equal(s.flags(), co)
            if name != "tgv32_ud7":
                assert (co > 0).any()
        err = field_rel_err(Lg, Lo)
        assert err <= TOL, err


def test_step_parity_tgv_config1(orc):
    """Taylor-Green 32^3, UD7, Re 400, CFL 0.5, 10 RK3 steps."""
    n = 32
    s, c, M = make_pair(orc, (n, n, n), _box((n, n, n)), scheme="UD7", Re=400.0)
    U = cases.taylor_green(n)
    with s:
        s.set_state(U)
        dt = s.cfl_dt(0.5)
        dto = orc.cfl_dt(c, M, U, 0.5)
        assert abs(dt - dto) <= 1e-14 * dto
        s.step(dt, 10)
        Ug = s.get_state()
    Uo = orc.step(c, M, U, dt, 10)
    err = field_rel_err(Ug, Uo)
    assert err <= TOL, err


@pytest.mark.parametrize("forced", [True, False])
def test_step_parity_hybrid(orc, forced):
    sh = (24, 20, 16)
    kw = dict(scheme="HYBRID", Re=200.0, theta1=0.004, theta2=0.012)
    s, c, M = make_pair(orc, sh, _box(sh), **kw)
    U = turbulence_field(sh, 21)
    _, cls0 = orc.sensor(c, U)
    if forced:
        c = orc.Case(*sh, Re=200.0, Ma=0.5, scheme=3, theta1=0.004, theta2=0.012, forced_cls=cls0)
    with s:
        s.set_state(U)
        if forced:
            s.force_flags(cls0)
        dt = s.cfl_dt(0.5)
        s.step(dt, 10)
        Ug = s.get_state()
    Uo = orc.step(c, M, U, dt, 10)
    err = field_rel_err(Ug, Uo)
    assert err <= TOL, err


@pytest.mark.parametrize("bc_hi", [(3, 3, 0), (5, 5, 0)])
def test_step_parity_ramp_with_walls(orc, bc_hi):
    """Walls, inflow, blowing and (second case) non-reflecting outlet and top:
    5 RK3 steps against the oracle."""
    s, c, M, U = ramp_pair(orc, bc_hi=bc_hi)
    with s:
        s.set_state(U)
        Ub = orc.apply_bc(c, M, U)
        dt = 0.3 * s.cfl_dt(0.5)
        s.step(dt, 5)
        Ug = s.get_state()
        t = s.time()
    assert abs(t - 5 * dt) <= 1e-15 * t
    Uo = orc.step(c, M, Ub, dt, 5)
    err = field_rel_err(Ug, Uo)
    assert err <= TOL, err


def test_determinism_and_resume(orc):
    sh = (24, 20, 16)
    s, c, M = make_pair(orc, sh, _box(sh), scheme="HYBRID", Re=200.0, theta1=0.004, theta2=0.012)
    U = turbulence_field(sh, 31)
    with s:
        s.set_state(U)
        dt = s.cfl_dt(0.5)
        s.step(dt, 10)
        A = s.get_state()
        s.set_state(U)
        s.set_time(0.0)
        s.step(dt, 10)
        B = s.get_state()
        s.set_state(U)
        s.set_time(0.0)
        s.step(dt, 5)
        mid = s.get_state()
        t5 = s.time()
        s.set_state(mid)
        s.set_time(t5)
        s.step(dt, 5)
        C = s.get_state()
    assert np.array_equal(A, B)
    assert np.array_equal(A, C)


def test_nonphysical_state_reported(orc):
    from paper_2209_15333_gb300 import _lib
    sh = (16, 16, 16)
    s, c, M = make_pair(orc, sh, _box(sh), scheme="UD7")
    U = cases.taylor_green(16)
    U[0, 3, 4, 5] = -1.0
    with s:
        s.set_state(U)
        with pytest.raises(_lib.CfdError) as ei:
            s.rhs()
        assert ei.value.status == _lib.CFD_ENONPHYS
        U2 = cases.taylor_green(16)
        U2[4, 1, 1, 1] = float("nan")
        s.set_state(U2)
        s.step(1e-3, 1)
        with pytest.raises(_lib.CfdError) as ei:
            s.sync(30.0)
        assert ei.value.status == _lib.CFD_ENONPHYS
        # the context stays usable
        s.set_state(cases.taylor_green(16))
        s.rhs()


def test_sync_timeout_returns(orc):
    """A wait that runs out returns CFD_ETIMEOUT; the work still completes."""
    from paper_2209_15333_gb300 import _lib
    n = 64
    s, c, M = make_pair(orc, (n, n, n), _box((n, n, n)), scheme="WENO7", Re=100.0)
    with s:
        s.set_state(cases.taylor_green(n))
        s.step(1e-3, 20)
        with pytest.raises(_lib.CfdError) as ei:
            s.sync(0.0)
        assert ei.value.status == _lib.CFD_ETIMEOUT
        s.sync(120.0)


def test_device_pointers_and_stream(orc):
    torch = pytest.importorskip("torch")
    from paper_2209_15333_gb300.solver import Solver
    n = 16
    U = cases.taylor_green(n)
    st = torch.cuda.Stream()
    s = Solver((n, n, n), torch.tensor(_box((n, n, n)), device="cuda"), stream=st, scheme=0, Re=400.0)
    with s:
        Ud = torch.tensor(U, device="cuda")
        s.set_state(Ud)
        Ld = torch.empty_like(Ud)
        s.rhs(out=Ld)
        st.synchronize()
        c = orc.Case(n, n, n, Re=400.0, Ma=0.5, scheme=0)
        Lo = orc.rhs(c, cases.expand_metrics(_box((n, n, n)), (n, n, n)), U)
        assert field_rel_err(Ld.cpu().numpy(), Lo) <= TOL


# (xi kind, xi segment), (eta/zeta kind, param), viscous kind
SWEEP_VARIANTS = [((0, 0), (0, 128), 0), ((1, 0), (0, 5), 1), ((1, 128), (1, 32), 2), ((1, 100), (1, 16), 1),
                  ((0, 0), (2, 0), 3), ((1, 0), (2, 8), 0), ((1, 256), (2, 13), 3)]


@pytest.mark.parametrize("precision,walled", [(0, True), (1, True), (1, False)])
def test_sweep_variants_bit_identical(orc, precision, walled):
    """The per-segment and walking xi sweeps, the streaming, tiled and
    walking eta/zeta sweeps (any segment / tile length) and the node-parallel
    and 2.5-D viscous kernels give identical bits, and so do the sensor
    classes (in FP32 the node-parallel and tiled viscous kernels also form the
    plain sensor's classes, the 2.5-D ones leave them to the sensor kernel);
    the autotuner only changes speed.  Lines of 300 xi nodes span several
    walking chunks and segments; the periodic box takes the instantiations
    for periodic lines with 8th-order viscous terms."""
    from paper_2209_15333_gb300.solver import Solver
    sh = (300, 21, 26)
    # one non-periodic direction too, or every direction periodic
    bc = dict(bc_lo=(0, 3, 0), bc_hi=(0, 3, 0)) if walled else dict(bc_lo=(0, 0, 0), bc_hi=(0, 0, 0))
    met = cases.uniform_metrics(*sh)
    U = turbulence_field(sh, 61)
    outs = []
    for (xk, xs), (kind, param), vk in SWEEP_VARIANTS:
        with Solver(sh, met, precision=precision, scheme=3, Re=150.0, theta1=0.004, theta2=0.012, **bc) as s:
            s.set_state(U)
            for d in (1, 2):
                s.set_sweep_variant(d, kind, param)
            s.set_sweep_variant(3, xk, xs)
            s.set_sweep_variant(0, vk, 0)
            assert s.sweep_variant(3) == (xk, xs)
            L = s.rhs()
            cls = s.flags()
            s.step(1e-3, 2)
            outs.append((L, s.get_state(), cls, s.flags()))
    assert len(np.unique(outs[0][2])) >= 2  # UD7 and WENO nodes occur
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
    if precision == 0:
        c = orc.Case(*sh, Re=150.0, Ma=0.5, scheme=3, theta1=0.004, theta2=0.012, **bc)
        Lo = orc.rhs(c, cases.expand_metrics(met, sh[::-1]), orc.apply_bc(c, cases.expand_metrics(met, sh[::-1]), U))
        assert field_rel_err(outs[0][0], Lo) <= TOL


@pytest.mark.parametrize("case", ["hybrid_viscous", "walled_inviscid_ud7"])
def test_tma_staged_sweeps_bit_identical(case):
    """The FP32 walking eta/zeta sweeps whose rows arrive by tensor-memory-
    accelerator copies (kind 3; several segments, periodic and walled lines,
    with and without classes and viscous fluxes) give the bits of the tiled
    sweeps.  Pinning kind 3 succeeds only where the TMA kernel runs."""
    from paper_2209_15333_gb300 import _lib as L
    from paper_2209_15333_gb300.solver import Solver
    if case == "hybrid_viscous":
        sh, bc = (96, 21, 26), dict(bc_lo=(0, 3, 0), bc_hi=(0, 3, 0))
        prm = dict(scheme=3, Re=150.0, theta1=0.004, theta2=0.012)
    else:
        sh, bc = (64, 40, 17), dict(bc_lo=(3, 1, 3), bc_hi=(3, 3, 3))
        prm = dict(scheme=0, Re=0.0, T_wall=1.2)
    met = cases.uniform_metrics(*sh)
    U = turbulence_field(sh, 64)
    outs = []
    for kind, param in ((1, 16), (3, 0), (3, 8), (3, 13), (2, 0)):
        with Solver(sh, met, precision=1, **bc, **prm) as s:
            s.set_state(U)
            for d in (1, 2):
                s.set_sweep_variant(d, kind, param)
            L_ = s.rhs()
            s.step(1e-3, 2)
            outs.append((L_, s.get_state()))
    for L_, V in outs[1:]:
        assert np.array_equal(L_, outs[0][0])
        assert np.array_equal(V, outs[0][1])
    # not available where rows are not 32-node multiples, nor in FP64
    with Solver((40, 8, 8), cases.uniform_metrics(40, 8, 8), precision=1) as s:
        with pytest.raises(L.CfdError) as e:
            s.set_sweep_variant(1, 3, 0)
        assert e.value.status == L.CFD_EUNSUPPORTED
    with Solver((32, 8, 8), cases.uniform_metrics(32, 8, 8), precision=0) as s:
        with pytest.raises(L.CfdError) as e:
            s.set_sweep_variant(2, 3, 0)
        assert e.value.status == L.CFD_EUNSUPPORTED


@pytest.mark.parametrize("n", [(17, 9, 5), (16, 8, 4)])
def test_pinned_host_state_round_trip(n):
    """State copies from and to pinned (device-mapped) host memory, which
    the SMs move themselves, are exact; odd and even element counts."""
    import torch
    from paper_2209_15333_gb300.solver import Solver
    met = cases.uniform_metrics(*n)
    U = turbulence_field(n, 71)
    host_in = torch.from_numpy(U.copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    with Solver(n, met, scheme=0, Re=0.0) as s:
        s.set_state(host_in)
        s.get_state(out=host_out)
        assert np.array_equal(host_out.numpy(), U)
        s.step(1e-3, 1)
        ref = s.get_state()            # pageable numpy: copy engine
        s.get_state(out=host_out)      # pinned: mapped copy
        assert np.array_equal(host_out.numpy(), ref)
