"""Host logic of the learned sensor (no GPU): bf16 rounding, node-weighted
rates and the calibration of the confidence threshold."""
import numpy as np

from paper_2209_15333_gb300.solver import from_bf16_bits, to_bf16_bits
from paper_2209_15333_gb300.train_sensor import calibrate, scores


def test_bf16_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 1.0 + 2.0 ** -9], dtype=np.float32)
    bits = to_bf16_bits(x)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to the even mantissa (1.0)
    assert list(bits) == [0x3F80, 0x3F80, 0x3F82, 0xC020, 0x3F80]
    assert np.array_equal(from_bf16_bits(bits), np.array([1.0, 1.0, 1.0 + 2.0 ** -6, -2.5, 1.0], np.float32))


def test_scores_are_node_weighted():
    # three samples: a confident correct UD7 standing for 100 nodes, a
    # confident unsafe call (UD7 for a WENO5 node), an unsure WENO7 node
    logits = np.array([[5.0, 0.0, 0.0], [5.0, 0.0, 0.0], [0.1, 0.0, 0.05]])
    y = np.array([0, 2, 1])
    w = np.array([100.0, 1.0, 1.0])
    sc = scores(logits, y, 0.0, w)
    assert abs(sc["misclassification"] - 2 / 102) < 1e-12
    assert abs(sc["unsafe_rate"] - 2 / 102) < 1e-12
    sc = scores(logits, y, 0.9, w)
    # the unsure node falls back to the plain class (correct); the confident
    # unsafe call stays
    assert abs(sc["fallback_rate"] - 1 / 102) < 1e-12
    assert abs(sc["misclassification"] - 1 / 102) < 1e-12
    assert abs(sc["unsafe_rate"] - 1 / 102) < 1e-12


def test_calibration_respects_the_unsafe_bound():
    rng = np.random.default_rng(0)
    n = 4000
    y = rng.integers(0, 3, n)
    logits = rng.normal(0, 1, (n, 3))
    logits[np.arange(n), y] += 2.5
    w = np.ones(n)
    off, conf, sc = calibrate(logits, y, w, unsafe_max=0.01)
    assert sc["unsafe_rate"] <= 0.01
    # nothing with a smaller fallback rate meets the bound on the searched grid
    for o in np.linspace(0.0, 6.0, 25):
        lg = logits.copy()
        lg[:, 0] += o
        for c in (0.5, 0.6, 0.7, 0.8, 0.9, 0.95, 0.98, 0.99):
            s2 = scores(lg, y, c, w)
            if s2["unsafe_rate"] <= 0.01:
                assert s2["fallback_rate"] >= sc["fallback_rate"] - 1e-15
