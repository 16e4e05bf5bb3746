"""Parity at full size: the 256^3 decaying isotropic-turbulence workload
(seed 20220930, turbulent Mach 0.5, Re_lambda ~ 72, hybrid scheme, 8th-order
viscous terms, power-law viscosity) in the launch configuration the benchmark
times: cfd_step with the autotuned sweeps replayed as a CUDA graph.

FP64: every node after 10 steps against the oracle on all host cores,
field-max relative error <= 1e-11 (free sensor, classes bit-exact).
FP32-bulk: one step against the oracle with the initial classes held on both
sides, bounded by the rounding model of the mixed-precision tests."""
import os

import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import field_rel_err

pytestmark = pytest.mark.gpu

N = 256
SEED = 20220930
MT = 0.5
C_MODEL = 50.0


@pytest.fixture(scope="module")
def workload():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()
    U, Re = cases.isotropic_turbulence(N, SEED, Mt=MT)
    met = cases.uniform_metrics(N, N, N)
    params = dict(gamma=1.4, Re=Re, Ma=MT, Pr=0.72, visc_law=1, visc_omega=0.76, scheme=3, theta1=0.02,
                  theta2=0.1, visc_order=8)
    return U, met, params


def _oracle_case(orc, params, forced_cls=None):
    return orc.Case(N, N, N, nthreads=os.cpu_count() or 1, forced_cls=forced_cls, **params)


def test_fp64_ten_steps_full_size(orc, workload):
    from paper_2209_15333_gb300.solver import Solver
    U, met, params = workload
    with Solver((N, N, N), met, **params) as s:
        s.set_state(U)
        dt = s.cfl_dt(0.5)
        s.step(dt, 10)
        Ug = s.get_state()
        cls_g = s.flags()
    c = _oracle_case(orc, params)
    M = cases.expand_metrics(met, (N, N, N))
    assert abs(dt - orc.cfl_dt(c, M, U, 0.5)) <= 1e-15 * dt
    Uo = orc.step(c, M, U, dt, 10)
    err = field_rel_err(Ug, Uo)
    _, cls_o = orc.sensor(c, Uo)
    print("256^3 FP64 10-step field-max relative error %.3g; non-UD7 nodes %d" % (err, int((cls_o > 0).sum())))
    assert err <= 1e-11
    # classes of the final state's last stage are those of a stage state, not
    # of Uo itself, so compare the share only
    assert abs(float((cls_g > 0).mean()) - float((cls_o > 0).mean())) < 0.01


def test_mixed_one_step_full_size(orc, workload):
    from paper_2209_15333_gb300.solver import Solver
    U, met, params = workload
    M = cases.expand_metrics(met, (N, N, N))
    c0 = _oracle_case(orc, params)
    _, cls = orc.sensor(c0, U)
    c = _oracle_case(orc, params, forced_cls=cls)
    with Solver((N, N, N), met, precision=1, **params) as s:
        s.set_state(U)
        s.force_flags(cls)
        dt = s.cfl_dt(0.5)
        s.step(dt, 1)
        Ug = s.get_state()
    Uo = orc.step(c, M, U, dt, 1)
    Lo = orc.rhs(c, M, U)
    Lm = orc.rhs(c, M, U.astype(np.float32).astype(np.float64))
    for q in range(5):
        dl = np.abs(Lm[q] - Lo[q]).max()
        err = np.abs(Ug[q] - Uo[q]).max()
        bound = C_MODEL * 3 * dt * dl + 1e-13 * np.abs(Uo[q]).max()
        print("256^3 mixed 1-step U error q%d: %.3g (bound %.3g, relative %.3g)"
              % (q, err, bound, err / np.abs(Uo[q]).max()))
        assert err <= bound


@pytest.mark.skipif(os.environ.get("CFD_LONG_PARITY") != "1",
                    reason="about 20 minutes of host cores for the oracle; set CFD_LONG_PARITY=1")
def test_two_hundred_steps_full_size(orc, workload):
    """The benchmark workload's full run: 200 RK3 steps of the 256^3 field in
    both forms against 200 oracle steps (free sensor on every side)."""
    from paper_2209_15333_gb300.solver import Solver
    U, met, params = workload
    M = cases.expand_metrics(met, (N, N, N))
    out = {}
    for prec in (0, 1):
        with Solver((N, N, N), met, precision=prec, **params) as s:
            s.set_state(U)
            dt = s.cfl_dt(0.5)
            s.step(dt, 200)
            out[prec] = s.get_state()
            cls = s.flags()
    Uo = orc.step(_oracle_case(orc, params), M, U, dt, 200)
    e64 = field_rel_err(out[0], Uo)
    e32 = field_rel_err(out[1], Uo)
    print("256^3 after 200 steps: FP64 %.3g, FP32-bulk %.3g field-max relative error; non-UD7 nodes %.4f"
          % (e64, e32, float((cls > 0).mean())))
    # stated, not a parity bound (10 steps is): over 200 steps a hybrid class
    # that flips at a threshold between two rounding-different states changes
    # a face by the difference of two schemes
    assert e64 <= 1e-8
    assert e32 <= 1e-3
