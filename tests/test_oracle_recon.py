"""Pins of the oracle's reconstructions: UD7 (Eq. 41), WENO5, WENO7 and the
masked WENO5 boundary closure (Sections 2.2.3-2.2.4, readings R8 and R10).

The oracle derives its WENO tables from definitions; these tests check them
against the paper's printed Eq. 41, the published linear weights, a symbolic
integration of the smoothness indicators (sympy), exactness on polynomials,
convergence order and the essentially non-oscillatory property.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

EQ41 = np.array([-3.0, 25.0, -101.0, 319.0, 214.0, -38.0, 4.0]) / 420.0


def test_linear_weights_and_full_stencils(orc):
    c5, d5, _, cf5 = orc.weno_tables(3)
    c7, d7, _, cf7 = orc.weno_tables(4)
    assert np.allclose(d5, np.array([1, 6, 3]) / 10.0, rtol=0, atol=1e-12)
    assert np.allclose(d7, np.array([1, 12, 18, 4]) / 35.0, rtol=0, atol=1e-12)
    # WENO7's underlying linear scheme is the paper's seventh-order upwind scheme
    assert np.allclose(cf7, EQ41, rtol=0, atol=1e-12)
    assert np.allclose(cf5, np.array([2, -13, 47, 27, -3]) / 60.0, rtol=0, atol=1e-12)
    # the linear combination of the candidates reproduces the full stencil
    for r, c, d, cf in ((3, c5, d5, cf5), (4, c7, d7, cf7)):
        acc = np.zeros(2 * r - 1)
        for k in range(r):
            acc[k:k + r] += d[k] * c[k]
        assert np.allclose(acc, cf, atol=1e-12)
    # textbook third-order candidates of WENO5
    assert np.allclose(c5[2], np.array([2, 5, -1]) / 6.0, atol=1e-12)
    assert np.allclose(c5[0], np.array([2, -7, 11]) / 6.0, atol=1e-12)


def _beta_symbolic(r, k, vals):
    """beta_k by exact integration of the cell-average interpolant (sympy)."""
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    coeffs = sp.symbols("a0:%d" % r)
    poly = sum(coeffs[p] * x ** p for p in range(r))
    eqs = []
    for l in range(r):
        o = -(r - 1) + k + l
        eqs.append(sp.integrate(poly, (x, o - sp.Rational(1, 2), o + sp.Rational(1, 2))) - vals[l])
    sol = sp.solve(eqs, coeffs)
    q = poly.subs(sol)
    beta = 0
    for l in range(1, r):
        beta += sp.integrate(sp.diff(q, x, l) ** 2, (x, -sp.Rational(1, 2), sp.Rational(1, 2)))
    return float(beta)


@pytest.mark.parametrize("r", [3, 4])
def test_smoothness_indicators_symbolic(orc, r):
    rng = np.random.default_rng(10 + r)
    for k in range(r):
        vals = [Fraction(int(v), 7) for v in rng.integers(-20, 20, size=r)]
        ref = _beta_symbolic(r, k, vals)
        got = orc.weno_beta(r, k, np.array([float(v) for v in vals]))
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


def test_weno5_beta_jiang_shu_form(orc):
    rng = np.random.default_rng(5)
    for _ in range(20):
        f = rng.normal(size=5)
        b0 = 13 / 12 * (f[0] - 2 * f[1] + f[2]) ** 2 + 0.25 * (f[0] - 4 * f[1] + 3 * f[2]) ** 2
        b1 = 13 / 12 * (f[1] - 2 * f[2] + f[3]) ** 2 + 0.25 * (f[1] - f[3]) ** 2
        b2 = 13 / 12 * (f[2] - 2 * f[3] + f[4]) ** 2 + 0.25 * (3 * f[2] - 4 * f[3] + f[4]) ** 2
        for k, b in enumerate((b0, b1, b2)):
            assert abs(orc.weno_beta(3, k, f[k:k + 3]) - b) <= 1e-13 * (1 + b)


def test_large_eps_gives_linear_scheme(orc):
    rng = np.random.default_rng(6)
    for _ in range(20):
        a7 = rng.normal(size=7)
        assert abs(orc.weno(4, a7, eps=1e30) - orc.ud7(a7)) <= 1e-14 * (1 + np.abs(a7).max())
        assert abs(orc.ud7(a7) - EQ41 @ a7) <= 1e-14 * (1 + np.abs(a7).max())
        a5 = rng.normal(size=5)
        lin5 = np.array([2, -13, 47, 27, -3]) / 60.0 @ a5
        assert abs(orc.weno(3, a5, eps=1e30) - lin5) <= 1e-14 * (1 + np.abs(a5).max())


def _cell_avg_poly(deg):
    """Cell averages over unit cells centred at integers of x^deg, and the
    exact face value at 1/2 of the function with those averages (x^deg)."""
    def avg(i):
        return (Fraction(2 * i + 1, 2) ** (deg + 1) - Fraction(2 * i - 1, 2) ** (deg + 1)) / (deg + 1)
    return avg


@pytest.mark.parametrize("deg", range(0, 9))
def test_ud7_polynomial_exactness(orc, deg):
    """Reconstruction of x^deg from its cell averages is exact at the face
    for deg <= 6 (seventh order), and not for deg = 7."""
    avg = _cell_avg_poly(deg)
    a = np.array([float(avg(i)) for i in range(-3, 4)])
    exact = 0.5 ** deg
    err = abs(orc.ud7(a) - exact)
    if deg <= 6:
        assert err <= 1e-12 * max(1.0, np.abs(a).max())
    else:
        assert err > 1e-6


@pytest.mark.parametrize("r,order", [(3, 5), (4, 7)])
def test_weno_convergence_order(orc, r, order):
    """Face values of a smooth function from its cell averages converge at
    the design order (point values of the flux = cell averages of h)."""
    errs = []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        x0 = 0.3
        # h(x) = sin(x): cell average over [x-h/2, x+h/2] is sin(x) sinc
        offs = np.arange(-(r - 1), r)
        xc = x0 + offs * h
        avg = (np.cos(xc - h / 2) - np.cos(xc + h / 2)) / h
        got = orc.weno(r, avg, eps=1e-6)
        errs.append(abs(got - math.sin(x0 + h / 2)))
    rates = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert rates[-1] > order - 0.6, (errs, rates)


@pytest.mark.parametrize("r", [3, 4])
def test_weno_non_oscillatory_on_step(orc, r):
    n = 2 * r - 1
    for jump_at in range(1, n):
        a = np.where(np.arange(n) < jump_at, 0.0, 1.0)
        v, om = orc.weno(r, a, return_omega=True)
        assert -1e-3 <= v <= 1 + 1e-3
        # sub-stencils that straddle the jump get a negligible weight
        for k in range(r):
            cells = range(k, k + r)
            crosses = any(c < jump_at for c in cells) and any(c >= jump_at for c in cells)
            smooth_exists = any(
                not (any(c < jump_at for c in range(kk, kk + r)) and any(c >= jump_at for c in range(kk, kk + r)))
                for kk in range(r))
            if crosses and smooth_exists:
                assert om[k] < 1e-6


def test_masked_weno5(orc):
    rng = np.random.default_rng(7)
    for _ in range(20):
        a = rng.normal(size=5)
        # only the right sub-stencil: third-order candidate (2 f_j + 5 f_j+1 - f_j+2)/6
        v, om = orc.weno(3, a, mask=[1, 1, 0], return_omega=True)
        assert np.allclose(om, [0, 0, 1])
        assert abs(v - (2 * a[2] + 5 * a[3] - a[4]) / 6.0) <= 1e-14 * (1 + np.abs(a).max())
        v, om = orc.weno(3, a, mask=[1, 0, 0], return_omega=True)
        assert om[0] == 0.0 and abs(om.sum() - 1.0) <= 1e-15
        # renormalised linear weights 6:3 on smooth (linear) data
        lin = np.arange(5) * 0.7 + 0.1
        v, om = orc.weno(3, lin, mask=[1, 0, 0], return_omega=True)
        assert np.allclose(om, [0, 2 / 3, 1 / 3], atol=1e-12)


def test_midpoint_weights(orc):
    w = orc.midpoint_weights()
    assert np.allclose(w * 2048, [-5, 49, -245, 1225, 1225, -245, 49, -5], atol=1e-11)
    x = np.arange(-3, 5, dtype=float)
    for deg in range(8):
        assert abs(w @ x ** deg - 0.5 ** deg) <= 1e-12


@pytest.mark.parametrize("r", [3, 4])
def test_weno_invariant_to_flux_scale(orc, r):
    """Reading R23: the weights are measured on the flux per unit face area,
    so scaling the values and the face scale together scales the result and
    leaves the weights unchanged (the values straddle a jump, where the
    weights are far from linear)."""
    a = np.array([1.0, 1.02, 0.97, 1.1, 3.0, 3.05, 2.9])[:2 * r - 1]
    v1, w1 = orc.weno(r, a, return_omega=True)
    for lam in (1e-7, 1e-3, 1e4):
        v2, w2 = orc.weno(r, lam * a, return_omega=True, scale=lam)
        assert abs(v2 / lam - v1) < 1e-14 * abs(v1)
        assert np.allclose(w2, w1, rtol=1e-13, atol=0)
    # the unscaled call on tiny values degenerates to the linear weights
    _, d, _, _ = orc.weno_tables(r)
    _, w3 = orc.weno(r, 1e-7 * a, return_omega=True)
    assert np.allclose(w3, d, atol=1e-3)
    assert not np.allclose(w1, d, atol=1e-2)
