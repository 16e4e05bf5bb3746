"""Ensembles of uneven blocks (cfd_create_batch): one persistent launch per
kernel kind runs every block; each block must evolve exactly as it does in a
context of its own (same operations, so identical bits), and as the oracle."""
import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import field_rel_err, turbulence_field

pytestmark = pytest.mark.gpu

SHAPES = [(24, 20, 16), (32, 16, 24), (17, 33, 9), (40, 12, 20), (22, 12, 10)]
BCS = [((0, 0, 0), (0, 0, 0))] * 4 + [((3, 3, 0), (3, 3, 0))]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def _blocks(precision):
    mets, params, states = [], [], []
    for b, sh in enumerate(SHAPES):
        if b == 4:
            met, _ = cases.wavy_grid(22, amp=0.04)
            met = np.ascontiguousarray(met[:, :10, :12, :22])
        else:
            met = cases.uniform_metrics(*sh)
        mets.append(met)
        params.append(dict(scheme=3, Re=150.0 + 40 * b, Ma=0.3 + 0.1 * b, theta1=0.004, theta2=0.012,
                           precision=precision))
        states.append(turbulence_field(sh, 70 + b, Mt=0.3 + 0.1 * b))
    return mets, params, states


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_single_block_contexts(orc, precision):
    from paper_2209_15333_gb300.solver import BatchSolver, Solver
    mets, params, states = _blocks(precision)
    dt = 5e-4
    with BatchSolver(SHAPES, mets, params, bcs=BCS) as bs:
        for b, U in enumerate(states):
            bs.set_state(U, block=b)
        bs.step(dt, 4)
        got = [bs.get_state(block=b) for b in range(len(SHAPES))]
        assert abs(bs.time() - 4 * dt) <= 1e-15
        # (mixed precision picks FP64 recovery from the previous classes, which
        # set_state resets: compare right-hand sides right after set_state)
        bs.set_state(got[2], block=2)
        Lb = bs.rhs(block=2)
    for b, sh in enumerate(SHAPES):
        lo, hi = BCS[b]
        with Solver(sh, mets[b], bc_lo=lo, bc_hi=hi, **params[b]) as s:
            s.set_state(states[b])
            s.step(dt, 4)
            ref = s.get_state()
            if b == 2:
                s.set_state(got[2])
                assert np.array_equal(s.rhs(), Lb)
        assert np.array_equal(got[b], ref), b
    if precision == 0:
        for b in (0, 4):
            lo, hi = BCS[b]
            c = orc.Case(*SHAPES[b], bc_lo=lo, bc_hi=hi, **{k: v for k, v in params[b].items() if k != "precision"})
            M = cases.expand_metrics(mets[b], SHAPES[b][::-1])
            Uo = orc.step(c, M, orc.apply_bc(c, M, states[b]), dt, 4)
            assert field_rel_err(got[b], Uo) <= 1e-11


def _mlp_weights(seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(0, 10.0, (32, 42)), rng.normal(0, 0.5, (32, 32)), rng.normal(0, 0.5, (3, 32)),
            rng.normal(0, 0.1, 32), rng.normal(0, 0.1, 32), rng.normal(0, 0.1, 3))


@pytest.mark.parametrize("precision,impl", [(0, 0), (1, 0), (1, 1)])
def test_batch_learned_sensor_matches_single_block_contexts(precision, impl):
    """The learned sensor in an ensemble (one launch walks the zeta columns
    of all blocks, with partial columns, clamped lines and ragged segments)
    gives every block the classes, fallbacks and state of its own context."""
    from paper_2209_15333_gb300.solver import BatchSolver, Solver
    mets, params, states = _blocks(precision)
    W = _mlp_weights(11)
    dt = 5e-4
    with BatchSolver(SHAPES, mets, params, bcs=BCS) as bs:
        for b, U in enumerate(states):
            bs.set_state(U, block=b)
        bs.set_sensor_mlp(*W, conf_min=0.6)
        bs.set_sweep_variant(4, impl, 0)
        bs.sensor_fallbacks()
        bs.step(dt, 3)
        got = [bs.get_state(block=b) for b in range(len(SHAPES))]
        cls = [bs.flags(block=b) for b in range(len(SHAPES))]
        fb = bs.sensor_fallbacks()
    fb_ref = 0
    kinds = set()
    for b, sh in enumerate(SHAPES):
        lo, hi = BCS[b]
        with Solver(sh, mets[b], bc_lo=lo, bc_hi=hi, **params[b]) as s:
            s.set_state(states[b])
            s.set_sensor_mlp(*W, conf_min=0.6)
            s.set_sweep_variant(4, impl, 0)
            s.step(dt, 3)
            assert np.array_equal(s.flags(), cls[b]), b
            assert np.array_equal(s.get_state(), got[b]), b
            fb_ref += s.sensor_fallbacks()
        kinds |= set(np.unique(cls[b]).tolist())
    assert fb == fb_ref and fb > 0
    assert len(kinds) >= 2


def test_batch_classifier_timed_once():
    """With the learned sensor and no classifier fixed, an ensemble times both
    classifiers on its first step and keeps one; the run then gives the bits
    (states, classes, fallbacks) of the same ensemble with that classifier fixed."""
    from paper_2209_15333_gb300.solver import BatchSolver
    mets, params, states = _blocks(1)
    W = _mlp_weights(12)
    runs = []
    for fixed in (None, "picked"):
        with BatchSolver(SHAPES, mets, params, bcs=BCS) as bs:
            for b, U in enumerate(states):
                bs.set_state(U, block=b)
            bs.set_sensor_mlp(*W, conf_min=0.6)
            if fixed is not None:
                bs.set_sweep_variant(4, runs[0][0], 0)
            bs.sensor_fallbacks()
            bs.step(5e-4, 2)
            impl = bs.sweep_variant(4)[0]
            runs.append((impl, [bs.get_state(block=b) for b in range(len(SHAPES))],
                         [bs.flags(block=b) for b in range(len(SHAPES))], bs.sensor_fallbacks()))
    assert runs[0][0] in (0, 1) and runs[1][0] == runs[0][0]
    for b in range(len(SHAPES)):
        assert np.array_equal(runs[0][1][b], runs[1][1][b]), b
        assert np.array_equal(runs[0][2][b], runs[1][2][b]), b
    assert runs[0][3] == runs[1][3]


# ensemble variants as (kind, param): viscous (dir 0), xi (dir 3), eta/zeta (dirs 1, 2)
VISC_V = [(2, 32), (1, 64), (3, 0)]
XI_V = [(0, 64), (0, 128), (1, 0)]
ETA_V = [(1, 16), (1, 32), (2, 64)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_variants_bit_identical(precision):
    """Every ensemble kernel variant the autotuner may pick (2.5-D viscous
    fluxes with 32 / 64 planes or 32 x 4 node tiles; xi in 64- / 128-node
    segments or walking whole lines; eta and zeta in 16- / 32-node tiles or
    walking 64-node segments) gives the same bits."""
    from paper_2209_15333_gb300.solver import BatchSolver
    mets, params, states = _blocks(precision)
    outs = []
    for v in ((0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (2, 0, 1, 2), (0, 2, 2, 1)):
        with BatchSolver(SHAPES, mets, params, bcs=BCS) as bs:
            for b, U in enumerate(states):
                bs.set_state(U, block=b)
            bs.set_sweep_variant(0, *VISC_V[v[0]])
            bs.set_sweep_variant(3, *XI_V[v[1]])
            bs.set_sweep_variant(1, *ETA_V[v[2]])
            bs.set_sweep_variant(2, *ETA_V[v[3]])
            got = bs.batch_variants()
            assert got == {"visc": VISC_V[v[0]], "xi": XI_V[v[1]], "eta": ETA_V[v[2]], "zeta": ETA_V[v[3]]}
            bs.step(5e-4, 3)
            outs.append([bs.get_state(block=b) for b in range(len(SHAPES))])
    for o in outs[1:]:
        for b in range(len(SHAPES)):
            assert np.array_equal(o[b], outs[0][b]), b


@pytest.mark.parametrize("precision", [0, 1])
def test_periodic_batch_matches_single_block_contexts(orc, precision):
    """An ensemble whose blocks are all periodic with 8th-order viscous terms
    takes the instantiations for periodic lines (viscous tiles; FP32 xi and
    tile sweeps): every variant still gives each block the bits of its own
    context, and the FP64 form matches the oracle."""
    from paper_2209_15333_gb300.solver import BatchSolver, Solver
    mets, params, states = _blocks(precision)
    shapes, bcs = SHAPES[:4], BCS[:4]
    mets, params, states = mets[:4], params[:4], states[:4]
    dt = 5e-4
    refs = []
    for b, sh in enumerate(shapes):
        with Solver(sh, mets[b], **params[b]) as s:
            s.set_state(states[b])
            s.step(dt, 3)
            refs.append(s.get_state())
    for v in ((2, 0, 0, 0), (2, 1, 1, 1), (0, 2, 2, 2)):
        with BatchSolver(shapes, mets, params, bcs=bcs) as bs:
            for b, U in enumerate(states):
                bs.set_state(U, block=b)
            bs.set_sweep_variant(0, *VISC_V[v[0]])
            bs.set_sweep_variant(3, *XI_V[v[1]])
            bs.set_sweep_variant(1, *ETA_V[v[2]])
            bs.set_sweep_variant(2, *ETA_V[v[3]])
            bs.step(dt, 3)
            for b in range(len(shapes)):
                assert np.array_equal(bs.get_state(block=b), refs[b]), (v, b)
    if precision == 0:
        c = orc.Case(*shapes[1], **{k: v for k, v in params[1].items() if k != "precision"})
        M = cases.expand_metrics(mets[1], shapes[1][::-1])
        Uo = orc.step(c, M, states[1], dt, 3)
        assert field_rel_err(refs[1], Uo) <= 1e-11


def test_batch_rejects_mismatched_blocks():
    from paper_2209_15333_gb300 import _lib
    from paper_2209_15333_gb300.solver import BatchSolver
    mets, params, _ = _blocks(0)
    params[1] = dict(params[1], scheme=0)
    with pytest.raises(_lib.CfdError) as ei:
        BatchSolver(SHAPES, mets, params, bcs=BCS)
    assert ei.value.status == _lib.CFD_EINVAL
