"""The free-stream-preserving metric mode on the GPU (reading R17): every
interface splits its eight stencil nodes with one interface metric, the
8-point midpoint interpolation of alpha = grad(d)/J.

- L(U) and 10 RK3 steps against the oracle's FSP mode on a curved (wavy)
  3-D grid at 1e-11 (hybrid scheme, viscous).
- Uniform flow over the curved grid: |L| <= 1e-13 of the flux scale, where
  the paper's nodal mode leaves a residual above 1e-6.
- Non-periodic lines, characteristic reconstruction, ensembles and the
  allocation-free call reject the mode.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import field_rel_err, turbulence_field

pytestmark = pytest.mark.gpu

TOL = 1e-11
PRM = dict(Re=300.0, Ma=0.5, scheme=3, theta1=0.004, theta2=0.012)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def _flux_scale(met, U):
    """max|J| max|grad d| max|U|: the size of L = J R with R ~ alpha . F,
    the scale the oracle's own free-stream pin uses."""
    return np.abs(met[9]).max() * np.abs(met[:9]).max() * np.abs(U).max()


def test_fsp_rhs_and_steps_match_oracle(orc):
    from paper_2209_15333_gb300.solver import Solver
    n = 20
    met, _ = cases.wavy_grid(n, amp=0.05)
    U = turbulence_field((n, n, n), 4)
    c = orc.Case(n, n, n, metric_mode=orc.METRIC_FSP, **PRM)
    with Solver((n, n, n), met, metric_mode=1, **PRM) as s:
        s.set_state(U)
        Lg = s.rhs()
        dt = s.cfl_dt(0.5)
        s.step(dt, 10)
        Ug = s.get_state()
    Lo = orc.rhs(c, met, U)
    assert field_rel_err(Lg, Lo) <= TOL
    Uo = orc.step(c, met, U, dt, 10)
    assert field_rel_err(Ug, Uo) <= TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_fsp_preserves_a_free_stream_on_a_curved_grid(precision):
    from paper_2209_15333_gb300.solver import Solver
    n = 16
    met, _ = cases.wavy_grid(n, amp=0.06)
    o = np.ones((n, n, n))
    U = cases.conserved(1.1 * o, 0.6 * o, -0.3 * o, 0.25 * o, 2.0 * o, 1.4)
    res = {}
    for mode in (0, 1):
        with Solver((n, n, n), met, metric_mode=mode, precision=precision, Re=500.0, Ma=0.6, scheme=3) as s:
            s.set_state(U)
            res[mode] = np.abs(s.rhs()).max() / _flux_scale(met, U)
    if precision == 0:
        assert res[1] <= 1e-13, res
        assert res[0] > 1e-6, res
    else:
        # FP32 bulk: a free stream to FP32 round-off, the nodal residual stays
        assert res[1] <= 1e-5 and res[1] < 1e-2 * res[0], res


def test_fsp_rejected_where_not_defined():
    from paper_2209_15333_gb300 import _lib as L
    from paper_2209_15333_gb300.solver import BatchSolver, Solver
    n = 16
    met = cases.uniform_metrics(n, n, n)
    with pytest.raises(L.CfdError) as e:
        Solver((n, n, n), met, metric_mode=1, bc_lo=(3, 0, 0), bc_hi=(3, 0, 0))
    assert e.value.status == L.CFD_EUNSUPPORTED
    with pytest.raises(L.CfdError) as e:
        Solver((n, n, n), met, metric_mode=1, recon_vars=1)
    assert e.value.status == L.CFD_EUNSUPPORTED
    with pytest.raises(L.CfdError) as e:
        BatchSolver([(n, n, n)], [met], [dict(metric_mode=1)])
    assert e.value.status == L.CFD_EUNSUPPORTED
    grid = L.make_grid(n, n, n, metric_layout=L.METRICS_UNIFORM)
    prm = L.default_params(metric_mode=1)
    import torch
    dummy = torch.zeros(5 * n ** 3, device="cuda", dtype=torch.float64)
    p = C.c_void_p(dummy.data_ptr())
    assert L.lib().cfd_rhs_noalloc(C.byref(grid), C.byref(prm), p, p, p, None) == L.CFD_EUNSUPPORTED
