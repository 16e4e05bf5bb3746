"""Learned shock sensor: features, tensor-core MLP and plain-sensor fallback.

The features are checked against a numpy evaluation of their definition; the
MLP classes against a numpy forward pass with the same roundings (features
and hidden activations to bf16, FP32 accumulation), on nodes whose logit
margin exceeds the accumulation-order tolerance.
"""
import numpy as np
import pytest

from paper_2209_15333_gb300 import cases

from gpu_helpers import turbulence_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def features_numpy(U, gamma, per):
    """42 features per node from the definition (float64 here)."""
    rho = U[0]
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    out = []
    for d in range(3):
        ax = 2 - d                      # arrays are [z][y][x]
        n = p.shape[ax]
        idx = np.arange(n)
        for q in (p, rho):
            vals = []
            for t in range(7):
                j = idx + t - 3
                j = j % n if per[d] else np.clip(j, 0, n - 1)
                vals.append(np.take(q, j, axis=ax))
            for t in range(6):
                out.append((vals[t + 1] - vals[t]) / vals[3])
            out.append((vals[2] - 2 * vals[3] + vals[4]) / (vals[2] + 2 * vals[3] + vals[4]))
    return np.stack(out)


def bf16(a):
    from paper_2209_15333_gb300.solver import from_bf16_bits, to_bf16_bits
    return from_bf16_bits(to_bf16_bits(np.asarray(a, np.float32)))


def mlp_numpy(F, W):
    x = bf16(F.reshape(42, -1).T)
    h = np.maximum(x @ bf16(W["w1"]).T + W["b1"], 0.0)
    h = np.maximum(bf16(h) @ bf16(W["w2"]).T + W["b2"], 0.0)
    return bf16(h) @ bf16(W["w3"]).T + W["b3"]


def random_weights(seed, scale=10.0):
    rng = np.random.default_rng(seed)
    # features are O(0.01-0.3): a wide first layer makes several classes occur
    return dict(w1=rng.normal(0, scale, (32, 42)), w2=rng.normal(0, 0.5, (32, 32)), w3=rng.normal(0, 0.5, (3, 32)),
                b1=rng.normal(0, 0.1, 32), b2=rng.normal(0, 0.1, 32), b3=rng.normal(0, 0.1, 3))


@pytest.mark.parametrize("precision", [0, 1])
def test_features_match_definition(precision):
    from paper_2209_15333_gb300.solver import Solver
    sh = (37, 19, 23)
    U = turbulence_field(sh, 91)
    bc = dict(bc_lo=(3, 0, 0), bc_hi=(3, 0, 0))
    with Solver(sh, cases.uniform_metrics(*sh), precision=precision, scheme=3, Re=100.0, **bc) as s:
        s.set_state(U)
        Ub = s.get_state()
        F = s.sensor_features()
    ref = features_numpy(Ub, 1.4, (0, 1, 1))
    tol = 1e-5 if precision else 1e-6
    assert np.abs(F - ref).max() <= tol * max(1.0, np.abs(ref).max())


def steep_field(sh, seed):
    """turbulence_field with p and rho scaled by tanh steps across z and x
    (width 1.5 nodes), so that the features of the finer lines still span
    several classes of the random network"""
    U = turbulence_field(sh, seed)
    nx, ny, nz = sh
    k = np.arange(nz)[:, None, None]
    i = np.arange(nx)[None, None, :]
    s = 1.0 + 0.25 * np.tanh((k - 0.5 * nz) / 1.5) + 0.15 * np.tanh((i - 0.4 * nx) / 1.5)
    u, v, w = U[1] / U[0], U[2] / U[0], U[3] / U[0]
    p = 0.4 * (U[4] - 0.5 * U[0] * (u * u + v * v + w * w))
    return cases.conserved(U[0] * s, u, v, w, p * s, 1.4)


# (precision, shape, x and z boundaries): the kernel walks zeta in 32 x 8
# (x, y) columns over segments of at most 64 planes; these shapes leave
# partial columns in x and y and a ragged last segment, and the clamped x and
# z line ends of non-periodic faces (3: outflow) fall inside a column or a
# segment; the first case runs the FP64 form
MLP_CASES = [(0, (40, 24, 20), 0, 0), (1, (40, 24, 20), 0, 0), (1, (132, 12, 10), 3, 0), (1, (37, 16, 12), 3, 0),
             (1, (45, 13, 27), 0, 3), (1, (33, 9, 70), 3, 3)]


# the classifier: 0 mma.sync per warp, 1 tcgen05 per CTA (tensor memory)
IMPLS = [0, 1]


@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("precision,sh,xbc,zbc", MLP_CASES)
def test_mlp_classes_match_numpy_forward_pass(precision, sh, xbc, zbc, impl):
    from paper_2209_15333_gb300.solver import Solver
    U = turbulence_field(sh, 92) if zbc == 0 else steep_field(sh, 92)
    W = random_weights(5)
    with Solver(sh, cases.uniform_metrics(*sh), precision=precision, scheme=3, Re=100.0, bc_lo=(xbc, 0, zbc),
                bc_hi=(xbc, 0, zbc)) as s:
        s.set_state(U)
        F = s.sensor_features()
        s.set_sensor_mlp(W["w1"], W["w2"], W["w3"], W["b1"], W["b2"], W["b3"], conf_min=0.0)
        s.set_sweep_variant(4, impl, 0)
        assert s.sweep_variant(4) == (impl, 0)
        s.rhs()
        got = s.flags().ravel()
        assert s.sensor_fallbacks() == 0
    logits = mlp_numpy(F, W)
    want = logits.argmax(axis=1)
    srt = np.sort(logits, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    sure = margin > 1e-2 * (1.0 + np.abs(logits).max(axis=1))
    assert sure.mean() > 0.9
    assert np.array_equal(got[sure], want[sure])
    assert len(np.unique(want)) >= 2


@pytest.mark.parametrize("impl", IMPLS)
def test_mlp_fallback_to_plain_sensor(impl):
    from paper_2209_15333_gb300.solver import Solver
    sh = (32, 16, 16)
    U = turbulence_field(sh, 93)
    kw = dict(scheme=3, Re=100.0, theta1=0.004, theta2=0.012)
    with Solver(sh, cases.uniform_metrics(*sh), **kw) as s:
        s.set_state(U)
        s.rhs()
        plain = s.flags()
        W = random_weights(6, scale=0.5)
        # small logits: no softmax probability rounds to 1, so every node falls back
        s.set_sensor_mlp(W["w1"], W["w2"], W["w3"], W["b1"], W["b2"], W["b3"], conf_min=1.0)
        s.set_sweep_variant(4, impl, 0)
        s.rhs()
        assert np.array_equal(s.flags(), plain)
        assert s.sensor_fallbacks() == plain.size
        s.set_sensor_mlp(None, None, None, None, None, None)
        s.rhs()
        assert np.array_equal(s.flags(), plain)


def test_packaged_model_against_plain_sensor():
    """The packaged weights on a held-out ensemble block (seed not used in
    training) after it has evolved: learned classes against the plain
    sensor's on the same state (rates over all nodes)."""
    from paper_2209_15333_gb300.solver import Solver
    from paper_2209_15333_gb300.train_sensor import load
    W, conf, report = load()
    blk = cases.ensemble_blocks(1, seed=777)[0]
    with Solver(blk["shape"], blk["metrics"], scheme=3, Re=blk["Re"], Ma=blk["Mt"], visc_law=1, visc_omega=0.76,
                precision=1) as s:
        s.set_state(blk["U"])
        s.step(s.cfl_dt(0.5), 60)
        s.rhs()
        plain = s.flags()
        s.set_sensor_mlp(W["w1"], W["w2"], W["w3"], W["b1"], W["b2"], W["b3"], conf_min=conf)
        s.sensor_fallbacks()
        s.rhs()
        learned = s.flags()
        fb = s.sensor_fallbacks() / plain.size
    mis = float((learned != plain).mean())
    unsafe = float((learned < plain).mean())
    print("packaged model: non-UD7 %.4f, misclassification %.4g, unsafe %.4g, fallback %.4g"
          % ((plain > 0).mean(), mis, unsafe, fb))
    assert (plain > 0).any()
    assert mis < 0.01 and unsafe < 0.002 and fb < 0.05


def test_mlp_classifier_forms_agree():
    """The two classifiers (mma.sync per warp, tcgen05 per CTA) on the same
    features: the same classes wherever the top logit leads by more than the
    accumulation-order tolerance, over several planes and partial columns."""
    from paper_2209_15333_gb300.solver import Solver
    sh = (70, 20, 40)
    U = steep_field(sh, 94)
    W = random_weights(8)
    got = []
    for impl in IMPLS:
        with Solver(sh, cases.uniform_metrics(*sh), precision=1, scheme=3, Re=100.0) as s:
            s.set_state(U)
            F = s.sensor_features()
            s.set_sensor_mlp(W["w1"], W["w2"], W["w3"], W["b1"], W["b2"], W["b3"], conf_min=0.0)
            s.set_sweep_variant(4, impl, 0)
            s.rhs()
            got.append(s.flags().ravel())
    logits = mlp_numpy(F, W)
    srt = np.sort(logits, axis=1)
    sure = (srt[:, -1] - srt[:, -2]) > 1e-2 * (1.0 + np.abs(logits).max(axis=1))
    assert sure.mean() > 0.9
    assert np.array_equal(got[0][sure], got[1][sure])
    assert (got[0] != got[1]).mean() < 1e-3
    with Solver(sh, cases.uniform_metrics(*sh), precision=1) as s:
        from paper_2209_15333_gb300 import _lib as L
        with pytest.raises(L.CfdError):
            s.set_sweep_variant(4, 2, 0)
