"""Values the paper prints, kept as text fixtures under tests/golden/ (each
file cites its equation or table), checked against the oracle, the C ABI's
defaults and the ramp set-up."""
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    rows = []
    for line in open(os.path.join(HERE, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


def test_ud7_coefficients_eq41(orc):
    num, (den,) = _rows("eq41_ud7.txt")
    coef = np.array(num) / den
    for k in range(7):
        e = np.zeros(7)
        e[k] = 1.0
        assert abs(orc.ud7(e) - coef[k]) <= 1e-16
    assert abs(coef.sum() - 1.0) < 1e-15


def test_hybrid_thresholds_are_the_defaults(orc):
    (t1, t2), = _rows("hybrid_thresholds.txt")
    c = orc.Case(8, 8, 8)
    assert (c.p.theta1, c.p.theta2) == (t1, t2)
    from paper_2209_15333_gb300 import _lib
    p = _lib.default_params()
    assert (p.theta1, p.theta2) == (t1, t2)


def test_mach_2_9_ramp_follows_table8():
    (ma, re_mm, t_inf, t_w), = _rows("table8_incoming_flow.txt")
    from paper_2209_15333_gb300.ramp import CASES
    c = CASES[4]
    assert c["Ma"] == ma and c["T_ref"] == t_inf
    # the wall temperature ratio 307 / 108.1 = 2.84, taken as 2.8
    assert abs(c["Tw"] - t_w / t_inf) < 0.05


def test_oracle_tgv_regression_fixture():
    """The oracle reproduces its own stored 10-step Taylor-Green summary
    (written by tests/golden/make_tgv_reference.py); a change of the oracle's
    arithmetic shows up here."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_tgv_reference", os.path.join(HERE, "make_tgv_reference.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    stored = {}
    for line in open(os.path.join(HERE, "tgv32_10steps.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            stored[k] = float(v)
    for k, v in m.summary():
        assert abs(v - stored[k]) <= 1e-12 * max(1.0, abs(stored[k])), k
