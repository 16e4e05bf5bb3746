"""Derive the WENO5/WENO7 constants used by the CUDA kernels (exact rationals).

Conservative finite differences treat node values as cell averages of a
function h on unit cells; a sub-stencil's candidate is the degree r-1
polynomial with those averages, evaluated at the right face x = 1/2, and its
smoothness indicator is sum_{l=1}^{r-1} int_{-1/2}^{1/2} (d^l q/dx^l)^2 dx
(Jiang and Shu 1996; Balsara and Shu 2000 for r = 4).  The linear weights
make the candidates' combination equal the full-stencil reconstruction.

Run:  python derive_weno.py > weno_coeffs.cuh
The output is committed; this script documents where every number comes from.
"""
import sympy as sp


def candidate(offsets):
    """Face coefficients, and the smoothness indicator written as a weighted
    sum of squares sum_i D_i (h_i . f)^2: the indicator is a^T B a in the
    derivative coefficients a_1..a_{r-1} of the polynomial (each a linear
    combination of f that annihilates constants), and B = L D L^T."""
    x = sp.symbols("x")
    r = len(offsets)
    a = sp.symbols("a0:%d" % r)
    f = sp.symbols("f0:%d" % r)
    poly = sum(a[p] * x ** p for p in range(r))
    eqs = [sp.integrate(poly, (x, o - sp.Rational(1, 2), o + sp.Rational(1, 2))) - f[l]
           for l, o in enumerate(offsets)]
    sol = sp.solve(eqs, a)
    q = sp.expand(poly.subs(sol))
    face = sp.expand(q.subs(x, sp.Rational(1, 2)))
    coef = [face.coeff(f[l]) for l in range(r)]
    if r == 1 or len(offsets) > 4:
        return coef, None
    beta_a = 0
    for l in range(1, r):
        beta_a += sp.integrate(sp.diff(poly, x, l) ** 2, (x, -sp.Rational(1, 2), sp.Rational(1, 2)))
    beta_a = sp.expand(beta_a)
    m = r - 1
    B = sp.Matrix(m, m, lambda i, j: beta_a.coeff(a[i + 1], 2) if i == j
                  else beta_a.coeff(a[i + 1], 1).coeff(a[j + 1], 1) / 2)
    Lm, Dm = B.LDLdecomposition()
    g = [[sp.expand(sol[a[p]]).coeff(f[l]) for l in range(r)] for p in range(1, r)]
    rows = []
    for i in range(m):
        h = [sum(Lm[p, i] * g[p][l] for p in range(m)) for l in range(r)]
        rows.append((Dm[i, i], h))
    return coef, rows


def tables(r):
    cands = [candidate([-(r - 1) + k + l for l in range(r)]) for k in range(r)]
    full, _ = candidate([-(r - 1) + l for l in range(2 * r - 1)])
    d = []
    for k in range(r):
        s = full[k] - sum(d[kk] * cands[kk][0][k - kk] for kk in range(k))
        d.append(sp.nsimplify(s / cands[k][0][0]))
    return cands, d, full


def c_num(v):
    v = sp.Rational(v)
    if v.q == 1:
        return "%d.0" % v.p
    return "(%d.0 / %d.0)" % (v.p, v.q)


def emit(r, name):
    cands, d, full = tables(r)
    print("/* WENO%d (r = %d): linear weights, candidate face coefficients and"
          " smoothness-indicator rows (see candidate()). */" % (2 * r - 1, r))
    print("#define %s_D {%s}" % (name, ", ".join(c_num(v) for v in d)))
    print("/* smoothness indicator beta_k = sum_i SD[i] * (S_k[i] . f)^2 */")
    print("#define %s_SD {%s}" % (name, ", ".join(c_num(dd) for dd, _ in cands[0][1])))
    for k, (coef, rows) in enumerate(cands):
        print("#define %s_C%d {%s}" % (name, k, ", ".join(c_num(v) for v in coef)))
        assert all(dd == cands[0][1][i][0] for i, (dd, _) in enumerate(rows))
        flat = [c_num(v) for _, h in rows for v in h]
        print("#define %s_S%d {%s}" % (name, k, ", ".join(flat)))
    print("/* full-stencil linear reconstruction: %s */" % ", ".join(str(v) for v in full))


if __name__ == "__main__":
    print("/* generated by derive_weno.py -- do not edit */")
    print("#pragma once")
    emit(3, "W5")
    emit(4, "W7")
