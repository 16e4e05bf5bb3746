"""Characteristic-variable reconstruction (Sec. 2.2.2, Eq. 31-40) on the GPU
against the FP64 oracle: field-max relative error <= 1e-11 on L(U) and on
the state after 10 steps (FP64), rounding-model bound for the FP32-bulk
form."""
import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import field_rel_err, turbulence_field

pytestmark = pytest.mark.gpu

TOL = 1e-11
CHAR = 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def _pair(orc, name, precision=0):
    from paper_2209_15333_gb300.solver import Solver
    bl = inflow = None
    bc_lo = bc_hi = (0, 0, 0)
    if name == "ragged_weno5":
        sh = (37, 19, 23)
        met, U = cases.uniform_metrics(*sh), turbulence_field(sh, 41, amp=1.5)
        kw = dict(scheme=1, Re=0.0, Ma=0.5)
    elif name == "ragged_weno7_viscous":
        sh = (29, 33, 17)
        met, U = cases.uniform_metrics(*sh), turbulence_field(sh, 42, amp=1.5)
        kw = dict(scheme=2, Re=150.0, Ma=0.5, visc_law=0, T_ref=108.1)
    elif name == "wavy_hybrid":
        n = 20
        met, _ = cases.wavy_grid(n, amp=0.05)
        sh, U = (n, n, n), turbulence_field((n, n, n), 43, amp=1.2)
        kw = dict(scheme=3, Re=300.0, Ma=0.5, theta1=0.004, theta2=0.012)
    elif name == "ramp_walls":
        sh = (40, 24, 8)
        rc = cases.ramp_case(*sh, 24.0, 2.9, Tw=2.8)
        met, U = rc["metrics2d"], rc["U"].copy()
        rng = np.random.default_rng(12)
        U[1:4] += 0.01 * rng.standard_normal(U[1:4].shape) * U[0]
        inflow = rc["inflow"]
        bl = dict(amp=0.05, x0=-15.0, x1=-10.0, omega=2.0, m=1, Lz=4.0, wall_x=rc["wall_x"], wall_z=rc["wall_z"])
        bc_lo, bc_hi = (2, 1, 0), (3, 3, 0)
        kw = dict(scheme=3, Re=2000.0, Ma=2.9, T_wall=2.8, visc_law=0, T_ref=108.1, theta1=0.005, theta2=0.02)
    else:
        raise KeyError(name)
    s = Solver(sh, met, bc_lo=bc_lo, bc_hi=bc_hi, precision=precision, recon_vars=CHAR, **kw)
    if inflow is not None:
        s.set_inflow(inflow)
    if bl is not None:
        s.set_blowing(bl["amp"], bl["x0"], bl["x1"], bl["omega"], bl["m"], bl["Lz"], bl["wall_x"], bl["wall_z"])
    c = orc.Case(*sh, bc_lo=bc_lo, bc_hi=bc_hi, inflow=inflow, blowing=bl, recon_vars=orc.RECON_CHARACTERISTIC,
                 **kw)
    M = cases.expand_metrics(met, sh[::-1])
    return s, c, M, U


NAMES = ["ragged_weno5", "ragged_weno7_viscous", "wavy_hybrid", "ramp_walls"]


@pytest.mark.parametrize("name", NAMES)
def test_char_rhs_parity(orc, name):
    s, c, M, U = _pair(orc, name)
    with s:
        s.set_state(U)
        Ug = s.get_state()   # boundary conditions applied by the library
        Lg = s.rhs()
        cls = s.flags()
    Uo = orc.apply_bc(c, M, U)
    assert field_rel_err(Ug, Uo) <= 1e-14
    Lo, co = orc.rhs(c, M, Uo, return_cls=True)
    if c.p.scheme == 3:
        assert np.array_equal(cls, co)
        print("%s: non-UD7 nodes %d of %d" % (name, int((co > 0).sum()), co.size))
    err = field_rel_err(Lg, Lo)
    print("char RHS %s: %.3g" % (name, err))
    assert err <= TOL


@pytest.mark.parametrize("name", ["ragged_weno5", "wavy_hybrid", "ramp_walls"])
def test_char_ten_steps_parity(orc, name):
    s, c, M, U = _pair(orc, name)
    with s:
        s.set_state(U)
        U0 = s.get_state()
        dt = s.cfl_dt(0.4)
        s.step(dt, 10)
        Ug = s.get_state()
    Uo = orc.step(c, M, U0, dt, 10)
    err = field_rel_err(Ug, Uo)
    print("char 10-step %s: %.3g" % (name, err))
    assert err <= TOL


def test_char_differs_from_component(orc):
    """The option really changes the WENO faces (and nothing else for UD7)."""
    from paper_2209_15333_gb300.solver import Solver
    s, c, M, U = _pair(orc, "ragged_weno5")
    with s:
        s.set_state(U)
        Lc = s.rhs()
    with Solver((37, 19, 23), cases.uniform_metrics(37, 19, 23), scheme=1, Re=0.0, Ma=0.5) as s0:
        s0.set_state(U)
        L0 = s0.rhs()
    assert field_rel_err(Lc, L0) > 1e-6


def test_char_mixed_within_rounding_model(orc):
    s, c, M, U = _pair(orc, "wavy_hybrid", precision=1)
    with s:
        s.set_state(U)
        U0 = s.get_state()
        _, cls = orc.sensor(c, U0)
        s.force_flags(cls)
        Lg = s.rhs()
    kw = {f: getattr(c.p, f) for f in ("gamma", "Re", "Ma", "Pr", "T_wall", "T_ref", "visc_law", "visc_omega",
                                       "scheme", "theta1", "theta2", "visc_order")}
    cf = orc.Case(c.p.nx, c.p.ny, c.p.nz, forced_cls=cls, recon_vars=orc.RECON_CHARACTERISTIC, **kw)
    Lo = orc.rhs(cf, M, U0)
    Lm = orc.rhs(cf, M, U0.astype(np.float32).astype(np.float64))
    for q in range(5):
        bound = 50.0 * np.abs(Lm[q] - Lo[q]).max() + 1e-12 * np.abs(Lo[q]).max()
        err = np.abs(Lg[q] - Lo[q]).max()
        print("char mixed L q%d: %.3g (bound %.3g)" % (q, err, bound))
        assert err <= bound


def test_char_rejected_where_unsupported():
    from paper_2209_15333_gb300 import _lib as L
    from paper_2209_15333_gb300.solver import BatchSolver
    sh = (16, 16, 16)
    p = dict(scheme=1, recon_vars=CHAR)
    with pytest.raises(L.CfdError) as e:
        BatchSolver([sh, sh], [cases.uniform_metrics(*sh)] * 2, [p, p])
    assert e.value.status == L.CFD_EUNSUPPORTED
