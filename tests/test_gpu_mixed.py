"""FP32-bulk / FP64-state path against the FP64 oracle.

Error bounds from the arithmetic, case by case: how much FP32 rounding costs
depends on how strongly the flux difference cancels (at low Mach number the
split fluxes carry the background pressure 1/(gamma Ma^2) while the RHS
carries its small gradient).  The bound is therefore a rounding model: the
oracle's own response to rounding the state to FP32 (one rounding of every
input, unit roundoff 6e-8), times C = 50 for the few hundred FP32 operations
of each node whose rounding errors add up.  For the state after n steps the
model response of L is integrated over the 3n stages.  The tests print the
measured errors and the bounds.
"""
import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import field_rel_err, make_pair, turbulence_field

pytestmark = pytest.mark.gpu

C_MODEL = 50.0


def round32(U):
    return U.astype(np.float32).astype(np.float64)


def l_model(orc, c, M, U, Lo):
    """per-field max |L(round32(U)) - L(U)| from the oracle"""
    Lm = orc.rhs(c, M, round32(U))
    return np.array([np.abs(Lm[q] - Lo[q]).max() for q in range(5)])


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def _pair(orc, name, precision):
    from paper_2209_15333_gb300.solver import Solver
    if name == "tgv32_hybrid":
        n = 32
        sh, met, U = (n, n, n), cases.uniform_metrics(n, n, n), cases.taylor_green(n)
        kw = dict(scheme=3, Re=400.0, theta1=0.004, theta2=0.012)
    elif name == "ragged_weno7":
        sh = (37, 19, 23)
        met, U = cases.uniform_metrics(*sh), turbulence_field(sh, 51)
        kw = dict(scheme=2, Re=200.0, visc_order=6)
    elif name == "wavy_hybrid":
        n = 20
        met, _ = cases.wavy_grid(n, amp=0.05)
        sh, U = (n, n, n), turbulence_field((n, n, n), 52)
        kw = dict(scheme=3, Re=300.0, theta1=0.004, theta2=0.012)
    else:
        raise KeyError(name)
    s = Solver(sh, met, precision=precision, **kw)
    c = orc.Case(*sh, Ma=0.5, **kw)
    return s, c, cases.expand_metrics(met, sh[::-1]), U


def _force_oracle_classes(orc, s, c, U):
    """Hold the hybrid switch at the oracle's classes on both sides, so that
    only arithmetic differs (a class flip near a threshold changes the face
    flux by the difference between two schemes, not by rounding)."""
    if c.p.scheme != 3:
        return c
    _, cls = orc.sensor(c, U)
    s.force_flags(cls)
    kw = {f: getattr(c.p, f) for f in ("gamma", "Re", "Ma", "Pr", "T_wall", "T_ref", "visc_law", "visc_omega",
                                       "scheme", "theta1", "theta2", "visc_order")}
    return orc.Case(c.p.nx, c.p.ny, c.p.nz, forced_cls=cls, **kw)


@pytest.mark.parametrize("name", ["tgv32_hybrid", "ragged_weno7", "wavy_hybrid"])
def test_mixed_rhs_error_vs_fp64_oracle(orc, name):
    s, c, M, U = _pair(orc, name, 1)
    with s:
        s.set_state(U)
        c = _force_oracle_classes(orc, s, c, U)
        Lg = s.rhs()
    Lo = orc.rhs(c, M, U)
    dl = l_model(orc, c, M, U, Lo)
    for q in range(5):
        den = np.abs(Lo[q]).max()
        err = np.abs(Lg[q] - Lo[q]).max()
        bound = C_MODEL * dl[q] + 1e-12 * den
        print("mixed L error %s q%d: %.3g (bound %.3g, rel %.3g)" % (name, q, err, bound, err / max(den, 1e-300)))
        assert err <= bound


def test_mixed_free_sensor_class_mismatch_reported(orc):
    """Free mode: the FP32 sensor may flip classes where theta sits within
    FP32 rounding of a threshold; count the flips (a small fraction)."""
    s, c, M, U = _pair(orc, "tgv32_hybrid", 1)
    with s:
        s.set_state(U)
        s.rhs()
        g = s.flags()
    _, co = orc.sensor(c, U)
    mism = int((g != co).sum())
    print("mixed free-mode class mismatches: %d of %d (oracle non-UD7 nodes: %d)" % (mism, co.size, int((co > 0).sum())))
    assert mism <= 0.01 * co.size


@pytest.mark.parametrize("name", ["tgv32_hybrid", "ragged_weno7"])
def test_mixed_ten_steps_error_vs_fp64_oracle(orc, name):
    s, c, M, U = _pair(orc, name, 1)
    with s:
        s.set_state(U)
        c = _force_oracle_classes(orc, s, c, U)
        dt = orc.cfl_dt(c, M, U, 0.5)
        s.step(dt, 10)
        Ug = s.get_state()
    Uo = orc.step(c, M, U, dt, 10)
    dl = l_model(orc, c, M, U, orc.rhs(c, M, U))
    for q in range(5):
        err = np.abs(Ug[q] - Uo[q]).max()
        bound = C_MODEL * 3 * 10 * dt * dl[q] + 1e-13 * np.abs(Uo[q]).max()
        print("mixed 10-step U error %s q%d: %.3g (bound %.3g)" % (name, q, err, bound))
        assert err <= bound


@pytest.mark.parametrize("bc_hi", [(3, 3, 0), (5, 5, 0)])
def test_mixed_ramp_with_walls(orc, bc_hi):
    """Walls, inflow, extrapolation (or non-reflecting outlet and top), 2-D
    metrics, Sutherland; FP64 recovery near the wall and at flagged nodes."""
    rc = cases.ramp_case(40, 24, 8, 24.0, 2.9, Tw=2.8)
    kw = dict(scheme="HYBRID", Re=2000.0, Ma=2.9, T_wall=2.8, visc_law=0, T_ref=108.1, bc_lo=(2, 1, 0),
              bc_hi=bc_hi, inflow=rc["inflow"])
    s64, c, M = make_pair(orc, (40, 24, 8), rc["metrics2d"], **kw)
    s64.close()
    from paper_2209_15333_gb300.solver import Solver
    s = Solver((40, 24, 8), rc["metrics2d"], bc_lo=(2, 1, 0), bc_hi=bc_hi, precision=1, scheme=3, Re=2000.0,
               Ma=2.9, T_wall=2.8, visc_law=0, T_ref=108.1)
    s.set_inflow(rc["inflow"])
    U = rc["U"].copy()
    rng = np.random.default_rng(11)
    U[1:4] += 0.01 * rng.standard_normal(U[1:4].shape) * U[0]
    with s:
        s.set_state(U)
        Ub = orc.apply_bc(c, M, U)
        dt = 0.3 * orc.cfl_dt(c, M, Ub, 0.5)
        s.step(dt, 5)
        Ug = s.get_state()
    Uo = orc.step(c, M, Ub, dt, 5)
    dl = l_model(orc, c, M, Ub, orc.rhs(c, M, Ub))
    for q in range(5):
        err = np.abs(Ug[q] - Uo[q]).max()
        bound = C_MODEL * 3 * 5 * dt * dl[q] + 1e-13 * np.abs(Uo[q]).max()
        print("mixed ramp 5-step U error q%d: %.3g (bound %.3g)" % (q, err, bound))
        assert err <= bound


def test_mixed_is_deterministic(orc):
    s, c, M, U = _pair(orc, "tgv32_hybrid", 1)
    with s:
        s.set_state(U)
        s.step(1e-3, 5)
        A = s.get_state()
        s.set_state(U)
        s.set_time(0.0)
        s.step(1e-3, 5)
        B = s.get_state()
    assert np.array_equal(A, B)


def test_integer_pipe_conversions_match_hardware():
    """The mixed form rounds the FP64 state to float and widens float
    residuals to double with integer operations; on the device they agree
    bit for bit with the hardware conversion on every float and on 2^32
    doubles that sweep float's exponent range and the rounding edges, and
    the double -> float path accepts exactly zero and 2^-126 <= |x| < 2^128."""
    from paper_2209_15333_gb300 import _lib
    c = _lib.check_conversions()
    print(c)
    assert c["floats"] == 1 << 32
    assert c["f2d_mismatch"] == 0
    # about 260/512 of the draws fall in float's range (exponent sweep) and
    # the special exponents add a few more
    assert c["doubles_ok"] > 0.45 * (1 << 32)
    assert c["d2f_mismatch"] == 0
    assert c["ok_flag_wrong"] == 0
