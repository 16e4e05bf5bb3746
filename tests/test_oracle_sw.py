"""Pins of the oracle's Steger-Warming splitting (Eqs. 19-30, reading R7).

The closed form of Eq. 23 (as corrected) is checked against
  * the exact flux of Eq. 6: f+ + f- = F;
  * the defining property of flux-vector splitting: f+- = A+- U with
    A+- = R diag(max/min(lambda, 0)) R^-1 from an eigendecomposition of the
    flux Jacobian A = dF/dU (computed here by complex-step differentiation);
  * one-sidedness for supersonic normal velocity and homogeneity in alpha.
"""
import numpy as np
import pytest

G = 1.4


def exact_flux(U, a, gamma=G):
    rho, mu, mv, mw, E = U
    u, v, w = mu / rho, mv / rho, mw / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w))
    V = a[0] * u + a[1] * v + a[2] * w
    return np.array([rho * V, mu * V + a[0] * p, mv * V + a[1] * p, mw * V + a[2] * p, (E + p) * V])


def prim_of(U, gamma=G):
    rho = U[0]
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    c = np.sqrt(gamma * p / rho)
    return rho, u, v, w, p, c


def random_state(rng, mach_max=3.0):
    rho = rng.uniform(0.2, 3.0)
    p = rng.uniform(0.2, 3.0)
    c = np.sqrt(G * p / rho)
    vel = rng.normal(size=3)
    vel *= rng.uniform(0.0, mach_max) * c / np.linalg.norm(vel)
    E = p / (G - 1) + 0.5 * rho * vel @ vel
    return np.array([rho, rho * vel[0], rho * vel[1], rho * vel[2], E])


def split(orc, U, a):
    rho, u, v, w, p, c = prim_of(U)
    return orc.sw_split(G, rho, u, v, w, c, *a)


def test_split_sums_to_exact_flux(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        U = random_state(rng)
        a = rng.normal(size=3) * rng.uniform(0.1, 10.0)
        fp, fm = split(orc, U, a)
        F = exact_flux(U, a)
        scale = np.abs(F).max() + np.abs(fp).max()
        assert np.abs(fp + fm - F).max() <= 1e-13 * scale


def jacobian_complex_step(U, a, h=1e-30):
    A = np.zeros((5, 5))
    for k in range(5):
        Uc = U.astype(complex)
        Uc[k] += 1j * h
        A[:, k] = np.imag(exact_flux(Uc, a)) / h
    return A


def test_split_equals_eigen_splitting(orc):
    """f+- = R Lambda+- R^-1 U: the definition of Steger-Warming splitting."""
    rng = np.random.default_rng(2)
    for _ in range(100):
        U = random_state(rng)
        a = rng.normal(size=3) * rng.uniform(0.1, 5.0)
        A = jacobian_complex_step(U, a)
        lam, R = np.linalg.eig(A)
        lam = lam.real
        Rinv = np.linalg.inv(R)
        Ap = (R @ np.diag(np.maximum(lam, 0.0)) @ Rinv).real
        Am = (R @ np.diag(np.minimum(lam, 0.0)) @ Rinv).real
        fp, fm = split(orc, U, a)
        scale = np.abs(exact_flux(U, a)).max() + np.abs(Ap @ U).max()
        assert np.abs(fp - Ap @ U).max() <= 1e-10 * scale
        assert np.abs(fm - Am @ U).max() <= 1e-10 * scale
        # eigenvalues of Eq. 20
        rho, u, v, w, p, c = prim_of(U)
        V = a @ np.array([u, v, w])
        sig = np.linalg.norm(a)
        expect = np.sort([V, V, V, V - c * sig, V + c * sig])
        assert np.allclose(np.sort(lam), expect, rtol=1e-9, atol=1e-9 * (abs(V) + c * sig))


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_supersonic_one_sided(orc, sign):
    rng = np.random.default_rng(3)
    for _ in range(50):
        a = rng.normal(size=3)
        sig = np.linalg.norm(a)
        rho, p = rng.uniform(0.5, 2.0, size=2)
        c = np.sqrt(G * p / rho)
        # normal velocity beyond the sound speed along a
        vel = sign * a / sig * c * rng.uniform(1.01, 3.0) + np.cross(a, rng.normal(size=3)) * 0.3
        E = p / (G - 1) + 0.5 * rho * vel @ vel
        U = np.array([rho, *(rho * vel), E])
        fp, fm = split(orc, U, a)
        F = exact_flux(U, a)
        if sign > 0:
            assert np.all(fm == 0.0)
            assert np.allclose(fp, F, rtol=1e-13, atol=1e-13 * np.abs(F).max())
        else:
            assert np.all(fp == 0.0)
            assert np.allclose(fm, F, rtol=1e-13, atol=1e-13 * np.abs(F).max())


def test_homogeneous_in_alpha(orc):
    rng = np.random.default_rng(4)
    for _ in range(50):
        U = random_state(rng)
        a = rng.normal(size=3)
        s = rng.uniform(0.1, 10.0)
        fp1, fm1 = split(orc, U, a)
        fp2, fm2 = split(orc, U, s * a)
        sc = np.abs(fp1).max() + np.abs(fm1).max()
        assert np.abs(fp2 - s * fp1).max() <= 1e-13 * s * sc
        assert np.abs(fm2 - s * fm1).max() <= 1e-13 * s * sc
