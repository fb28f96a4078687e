"""Pins of the oracle's angular and radial functions and of its Gaunt table.

Y_lm: scipy's complex spherical harmonics (converted to the real form), the addition
theorem with scipy's Legendre polynomials, orthonormality by an independent numpy
quadrature, gradients by central differences.  Radial basis: numpy's Chebyshev series.
Gaunt: sympy's complex Gaunt coefficients transformed to the real basis.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre, sph_harm_y

rng = np.random.default_rng(42)


def _unit(n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


def _real_ylm_scipy(l, m, v):
    theta = np.arccos(v[2] / np.linalg.norm(v))
    phi = np.arctan2(v[1], v[0])
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    y = sph_harm_y(l, abs(m), theta, phi)
    return np.sqrt(2) * (-1) ** m * (y.real if m > 0 else y.imag)


def test_ylm_matches_scipy_real_form(orc):
    for v in _unit(20) * 2.3:
        Y, _ = orc.ylm(v)
        for l in range(5):
            for m in range(-l, l + 1):
                assert abs(Y[l * l + l + m] - _real_ylm_scipy(l, m, v)) < 1e-13


def test_ylm_addition_theorem(orc):
    U = _unit(30)
    for a, b in zip(U[:15], U[15:]):
        Ya, _ = orc.ylm(a)
        Yb, _ = orc.ylm(b)
        for l in range(5):
            s = sum(Ya[l * l + l + m] * Yb[l * l + l + m] for m in range(-l, l + 1))
            assert abs(s - (2 * l + 1) / (4 * np.pi) * eval_legendre(l, a @ b)) < 1e-13


def test_ylm_orthonormal(orc):
    xs, ws = np.polynomial.legendre.leggauss(12)
    nph = 24
    M = np.zeros((25, 25))
    for ct, wt in zip(xs, ws):
        st = np.sqrt(1 - ct * ct)
        for k in range(nph):
            ph = 2 * np.pi * (k + 0.37) / nph
            Y, _ = orc.ylm([st * np.cos(ph), st * np.sin(ph), ct])
            M += wt * (2 * np.pi / nph) * np.outer(Y, Y)
    assert np.abs(M - np.eye(25)).max() < 1e-13


def test_ylm_gradient(orc):
    for v in _unit(8) * rng.uniform(1.5, 5.0, size=(8, 1)):
        Y, G = orc.ylm(v)
        # Y depends on the direction only: r . grad Y = 0
        assert np.abs(G @ v).max() < 1e-12
        h = 1e-6
        for k in range(3):
            e = np.zeros(3); e[k] = h
            fd = (orc.ylm(v + e)[0] - orc.ylm(v - e)[0]) / (2 * h)
            assert np.abs(fd - G[:, k]).max() < 1e-8


def test_radial_basis_is_chebyshev_times_cosine_cutoff(orc):
    rc = 5.0
    for r in (0.3, 1.7, 2.74, 4.2, 4.999):
        g, dg = orc.radial(r, rc)
        x = 2 * r / rc - 1
        fc = 0.5 * (1 + np.cos(np.pi * r / rc))
        for n in range(8):
            c = np.zeros(n + 1); c[n] = 1
            assert abs(g[n] - np.polynomial.chebyshev.chebval(x, c) * fc) < 1e-14
        h = 1e-6
        fd = (orc.radial(r + h, rc)[0] - orc.radial(r - h, rc)[0]) / (2 * h)
        assert np.abs(fd - dg).max() < 1e-7
    g, dg = orc.radial(rc, rc)
    assert np.all(g == 0) and np.all(dg == 0)


def _complex_to_real(l):
    """U with Y_real[m] = sum_m' U[m, m'] Y_complex[m'] (Condon-Shortley complex Y)."""
    U = np.zeros((2 * l + 1, 2 * l + 1), dtype=complex)
    for m in range(-l, l + 1):
        i = m + l
        if m == 0:
            U[i, l] = 1
        elif m > 0:
            U[i, -m + l] = 1 / np.sqrt(2)
            U[i, m + l] = (-1) ** m / np.sqrt(2)
        else:
            U[i, m + l] = 1j / np.sqrt(2)
            U[i, -m + l] = -1j * (-1) ** m / np.sqrt(2)
    return U


def test_gaunt_matches_sympy_complex_gaunt(orc):
    sympy = pytest.importorskip("sympy")
    from sympy.physics.wigner import gaunt
    for (l1, l2, l3) in [(1, 1, 2), (2, 2, 2), (1, 3, 4), (2, 3, 3), (4, 4, 4), (0, 2, 2)]:
        Gc = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1))
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                for m3 in range(-l3, l3 + 1):
                    Gc[m1 + l1, m2 + l2, m3 + l3] = float(sympy.N(gaunt(l1, l2, l3, m1, m2, m3), 20))
        U1, U2, U3 = _complex_to_real(l1), _complex_to_real(l2), _complex_to_real(l3)
        Gr = np.einsum("ai,bj,ck,ijk->abc", U1, U2, U3, Gc)
        assert np.abs(Gr.imag).max() < 1e-13
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                for m3 in range(-l3, l3 + 1):
                    assert abs(orc.gaunt(l1, m1, l2, m2, l3, m3) - Gr.real[m1 + l1, m2 + l2, m3 + l3]) < 1e-13


def test_gaunt_selection_rules_and_count(orc):
    nz = 0
    for l1 in range(5):
        for l2 in range(5):
            for l3 in range(5):
                ok = (l1 + l2 + l3) % 2 == 0 and abs(l1 - l2) <= l3 <= l1 + l2
                cnt = sum(orc.gaunt(l1, m1, l2, m2, l3, m3) != 0.0
                          for m1 in range(-l1, l1 + 1) for m2 in range(-l2, l2 + 1) for m3 in range(-l3, l3 + 1))
                if not ok:
                    assert cnt == 0
                elif l1 <= l2 <= l3:
                    nz += cnt
    assert nz == 416          # nonzero (m1, m2, m3) entries over the 14 sorted l-triples
