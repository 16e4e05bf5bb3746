"""Multi-block domains on one GPU (cfd_set_halo_links): a periodic box split
into blocks with ghost layers evolves exactly as the undivided box, on the GPU
and in the FP64 oracle (the gathered interiors against the oracle's undivided
periodic box, field-max relative error <= 1e-11)."""
import numpy as np
import pytest

from paper_2209_15333_gb300 import cases
from paper_2209_15333_gb300 import multiblock as mb

from gpu_helpers import field_rel_err, turbulence_field

pytestmark = pytest.mark.gpu

PARAMS = dict(scheme=3, Re=250.0, Ma=0.5, visc_law=1, visc_omega=0.76, theta1=0.004, theta2=0.012)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def _run_split(U, shape, parts, dt, nsteps, precision):
    from paper_2209_15333_gb300.solver import BatchSolver
    blocks, links = mb.decompose_box(shape, parts)
    Ub = mb.scatter(U, blocks)
    with BatchSolver([b["grid"] for b in blocks], [cases.uniform_metrics(*shape)] * len(blocks),
                     [dict(PARAMS, precision=precision)] * len(blocks),
                     bcs=[(b["bc_lo"], b["bc_hi"]) for b in blocks]) as s:
        for b, u in enumerate(Ub):
            s.set_state(u, block=b)
        s.set_halo_links(links)
        s.step(dt, nsteps)
        out = [s.get_state(block=b) for b in range(len(blocks))]
    return mb.gather(out, blocks, shape)


def _run_single(U, shape, nsteps, precision, dt=None):
    from paper_2209_15333_gb300.solver import Solver
    with Solver(shape, cases.uniform_metrics(*shape), precision=precision, **PARAMS) as s:
        s.set_state(U)
        dt = dt or s.cfl_dt(0.5)
        s.step(dt, nsteps)
        return s.get_state(), dt


@pytest.fixture(scope="module")
def oracle_box(orc):
    """The oracle's undivided periodic 40 x 36 x 24 box after 5 RK3 steps."""
    shape = (40, 36, 24)
    nx, ny, nz = shape
    U = turbulence_field(shape, 61, amp=1.2)
    _, dt = _run_single(U, shape, 0, 0)
    c = orc.Case(nx, ny, nz, **PARAMS)
    M = cases.expand_metrics(cases.uniform_metrics(*shape), (nz, ny, nx))
    return U, dt, orc.step(c, M, U, dt, 5)


@pytest.mark.parametrize("parts", [(2, 2, 1), (1, 1, 2), (3, 1, 1)])
def test_split_box_matches_undivided_fp64(parts, oracle_box):
    shape = (40, 36, 24)
    U, dt, Uo = oracle_box
    ref, _ = _run_single(U, shape, 5, 0, dt=dt)
    got = _run_split(U, shape, parts, dt, 5, 0)
    err = field_rel_err(got, ref)
    print("split %s FP64: rel err %.3g, bit-identical %s" % (parts, err, np.array_equal(got, ref)))
    assert err <= 1e-13
    err_o = field_rel_err(got, Uo)
    print("split %s FP64 against the oracle's undivided box: rel err %.3g" % (parts, err_o))
    assert err_o <= 1e-11


def test_self_linked_block_is_periodic():
    """One block whose x faces are linked to itself behaves as periodic in x."""
    from paper_2209_15333_gb300.solver import BatchSolver
    shape = (40, 20, 18)
    U = turbulence_field(shape, 62)
    ref, dt = _run_single(U, shape, 4, 0)
    blocks, _ = mb.decompose_box(shape, (2, 1, 1))
    H = mb.HALO_WIDTH
    ext = (shape[0] + 2 * H, shape[1], shape[2])
    idx = np.arange(-H, shape[0] + H) % shape[0]
    Ue = np.ascontiguousarray(U[:, :, :, idx])
    links = -np.ones((1, 3, 2), np.int32)
    links[0, 0, :] = 0
    with BatchSolver([ext], [cases.uniform_metrics(*shape)], [PARAMS], bcs=[((4, 0, 0), (4, 0, 0))]) as s:
        s.set_state(Ue, block=0)
        s.set_halo_links(links)
        s.step(dt, 4)
        got = s.get_state(block=0)[:, :, :, H:H + shape[0]]
    err = field_rel_err(got, ref)
    print("self-linked: rel err %.3g, bit-identical %s" % (err, np.array_equal(got, ref)))
    assert err <= 1e-13


def test_split_box_mixed_precision():
    """FP32-bulk: the same up to FP32 rounding (a ghost node at the end of an
    extended line takes the boundary rule of the sensor, so the mixed
    recovery may take FP64 there where the undivided box took FP32)."""
    shape = (40, 36, 24)
    U = turbulence_field(shape, 63, amp=1.2)
    ref, dt = _run_single(U, shape, 5, 1)
    got = _run_split(U, shape, (2, 2, 1), dt, 5, 1)
    err = field_rel_err(got, ref)
    print("split (2,2,1) mixed: rel err %.3g" % err)
    assert err <= 1e-6


def test_bad_links_rejected():
    from paper_2209_15333_gb300 import _lib as L
    from paper_2209_15333_gb300.solver import BatchSolver
    shape = (40, 20, 18)
    blocks, links = mb.decompose_box(shape, (2, 1, 1))
    with BatchSolver([b["grid"] for b in blocks], [cases.uniform_metrics(*shape)] * 2, [PARAMS] * 2,
                     bcs=[(b["bc_lo"], b["bc_hi"]) for b in blocks]) as s:
        bad = links.copy()
        bad[0, 0, 0] = 7
        with pytest.raises(L.CfdError) as e:
            s.set_halo_links(bad)
        assert e.value.status == L.CFD_EINVAL
        bad = links.copy()
        bad[1, 0, 1] = -1   # a HALO face left without a neighbour
        with pytest.raises(L.CfdError) as e:
            s.set_halo_links(bad)
        assert e.value.status == L.CFD_EINVAL
        bad = links.copy()
        bad[0, 1, 0] = 1    # a periodic face cannot be linked
        with pytest.raises(L.CfdError) as e:
            s.set_halo_links(bad)
        assert e.value.status == L.CFD_EINVAL
