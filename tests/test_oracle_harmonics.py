"""Pins for oracle.harmonics against the paper's appendix identities and library routines."""
from math import pi, sqrt

import numpy as np
import pytest

from oracle import harmonics as H


def _dirs(rng, n):
    u = rng.standard_normal((n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


@pytest.mark.parametrize("ell", range(0, 9))
def test_ylm_matches_scipy(rng, ell):
    sp = pytest.importorskip("scipy.special")
    u = _dirs(rng, 50)
    theta = np.arccos(u[:, 2])
    phi = np.arctan2(u[:, 1], u[:, 0])
    for m in range(-ell, ell + 1):
        ref = sp.sph_harm_y(ell, m, theta, phi)
        np.testing.assert_allclose(H.ylm(ell, m, u), ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("ell", range(0, 9))
def test_parity_and_conjugation(rng, ell):
    """Eq. sph_prop and Eq. sphiv."""
    u = _dirs(rng, 40)
    for m in range(-ell, ell + 1):
        np.testing.assert_allclose(H.ylm(ell, m, -u), (-1) ** ell * H.ylm(ell, m, u), atol=1e-12)
        np.testing.assert_allclose(H.ylm(ell, m, u), (-1) ** m * np.conj(H.ylm(ell, -m, u)),
                                   atol=1e-12)
        np.testing.assert_allclose(H.ylm(ell, -m, u), (-1) ** (ell + m) * np.conj(H.ylm(ell, m, -u)),
                                   atol=1e-12)


@pytest.mark.parametrize("ell", range(0, 9))
def test_special_values(rng, ell):
    """Y_l^m(z) = sqrt((2l+1)/4pi) delta_m0 and Y_l^0 = sqrt((2l+1)/4pi) L_l(cos theta)."""
    z = np.array([[0.0, 0.0, 1.0]])
    for m in range(-ell, ell + 1):
        want = sqrt((2 * ell + 1) / (4 * pi)) if m == 0 else 0.0
        np.testing.assert_allclose(H.ylm(ell, m, z), want, atol=1e-14)
    u = _dirs(rng, 30)
    np.testing.assert_allclose(H.ylm(ell, 0, u), sqrt((2 * ell + 1) / (4 * pi)) * H.legendre(ell, u[:, 2]),
                               atol=1e-13)


@pytest.mark.parametrize("ell", range(0, 9))
def test_addition_theorem(rng, ell):
    """Eq. add_theorem: L_l(r1.r2) = 4pi/(2l+1) sum_m Y*(r1) Y(r2)."""
    a, b = _dirs(rng, 64), _dirs(rng, 64)
    s = sum(np.conj(H.ylm(ell, m, a)) * H.ylm(ell, m, b) for m in range(-ell, ell + 1))
    np.testing.assert_allclose(4 * pi / (2 * ell + 1) * s, H.legendre(ell, np.sum(a * b, axis=1)),
                               atol=1e-13)


@pytest.mark.parametrize("ell", range(0, 7))
def test_addition_theorem_associated(rng, ell):
    """Eq. add_associated_L: for azimuths pi apart, L_l(r1.r2) = sum_m L_l^m(c1) L_l^{-m}(c2)."""
    t1 = rng.uniform(0, pi, 20)
    t2 = rng.uniform(0, pi, 20)
    phi = rng.uniform(0, 2 * pi, 20)
    r1 = np.stack([np.sin(t1) * np.cos(phi), np.sin(t1) * np.sin(phi), np.cos(t1)], 1)
    r2 = np.stack([np.sin(t2) * np.cos(phi + pi), np.sin(t2) * np.sin(phi + pi), np.cos(t2)], 1)
    lhs = H.legendre(ell, np.sum(r1 * r2, axis=1))
    rhs = sum(H.assoc_legendre(ell, m, np.cos(t1)) * H.assoc_legendre(ell, -m, np.cos(t2))
              for m in range(-ell, ell + 1))
    np.testing.assert_allclose(rhs, lhs, atol=1e-12)


def test_orthonormality():
    """Eq. ylm_orthonormal by Gauss-Legendre x uniform-phi quadrature (exact for l <= 8)."""
    xg, wg = np.polynomial.legendre.leggauss(20)
    nphi = 40
    phi = 2 * pi * np.arange(nphi) / nphi
    ct = xg[:, None] * np.ones((1, nphi))
    st = np.sqrt(1 - ct**2)
    u = np.stack([st * np.cos(phi), st * np.sin(phi), ct], -1)
    w = wg[:, None] * np.ones((1, nphi)) * (2 * pi / nphi)
    lm = [(l, m) for l in range(0, 7) for m in range(-l, l + 1)]
    Y = {key: H.ylm(key[0], key[1], u) for key in lm}
    for a in lm:
        for b in lm:
            val = np.sum(w * Y[a] * np.conj(Y[b]))
            np.testing.assert_allclose(val, 1.0 if a == b else 0.0, atol=1e-12)


def test_legendre_product_identities():
    """Eq. legendre: L4, L6, L8 in products of lower orders (polynomial identity at 64 points)."""
    x = np.linspace(-1, 1, 64)
    L = {l: H.legendre(l, x) for l in range(0, 9)}
    np.testing.assert_allclose(L[4], 35 / 18 * L[2] * L[2] - 5 / 9 * L[2] * L[0] - 7 / 18 * L[0] * L[0],
                               atol=1e-13)
    np.testing.assert_allclose(L[6], 11 / 5 * L[4] * L[2] - 4 / 7 * L[4] * L[0] - 22 / 35 * L[2] * L[0],
                               atol=1e-13)
    np.testing.assert_allclose(
        L[8],
        1287 / 490 * L[4] * L[4] - 286 / 245 * L[4] * L[2] - 209 / 1715 * L[4] * L[0]
        - 78 / 1715 * L[2] * L[0] - 143 / 490 * L[0] * L[0], atol=1e-13)


def test_wigner3j_against_sympy():
    wig = pytest.importorskip("sympy.physics.wigner")
    for j1 in range(0, 5):
        for j2 in range(0, 5):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                for m1 in range(-j1, j1 + 1):
                    for m2 in range(-j2, j2 + 1):
                        m3 = -m1 - m2
                        if abs(m3) > j3:
                            continue
                        ref = float(wig.wigner_3j(j1, j2, j3, m1, m2, m3))
                        assert abs(H.wigner3j(j1, j2, j3, m1, m2, m3) - ref) < 1e-14


def test_wigner3j_orthogonality_and_symmetry():
    """Eq. 3j-orthonormal and the sign-flip symmetry Eq. wigner_3j."""
    j1, j2 = 3, 2
    for j3 in range(1, 6):
        for j3p in range(1, 6):
            for m3 in range(-min(j3, j3p), min(j3, j3p) + 1):
                s = sum(H.wigner3j(j1, j2, j3, m1, m2, m3) * H.wigner3j(j1, j2, j3p, m1, m2, m3)
                        for m1 in range(-j1, j1 + 1) for m2 in range(-j2, j2 + 1))
                want = 1.0 if j3 == j3p else 0.0
                assert abs((2 * j3 + 1) * s - want) < 1e-13
    for (a, b, c) in [(2, 0, 2), (2, 2, 0), (1, 1, 2), (2, 2, 2), (4, 2, 2)]:
        for m1 in range(-a, a + 1):
            for m2 in range(-b, b + 1):
                v1 = H.wigner3j(a, b, c, m1, m2, -m1 - m2)
                v2 = H.wigner3j(a, b, c, -m1, -m2, m1 + m2)
                assert abs(v1 - (-1) ** (a + b + c) * v2) < 1e-14


def test_l0l_coefficients():
    """The values used to collapse the compressed estimator: (l 0 l; m 0 -m) = (-1)^{l-m}/sqrt(2l+1)."""
    for l in range(0, 6):
        for m in range(-l, l + 1):
            assert abs(H.wigner3j(l, 0, l, m, 0, -m) - (-1) ** (l - m) / sqrt(2 * l + 1)) < 1e-14


@pytest.mark.parametrize("ell", range(0, 5))
def test_g_closed_vs_integral(ell):
    """Eqs. g0-g4 against the practical integral form and the kappa form of Lemma 2."""
    for t in [0.05, 0.2, 0.5, 0.8, 0.97, 1.0, 1.03, 1.5, 2.0, 5.0, 30.0]:
        gc = H.g_closed(ell, t)
        assert abs(gc - H.g_integral(ell, t, 2000)) < 2e-6
        assert abs(gc - H.g_kappa(ell, t, 2000)) < 2e-6


def test_g_special_values():
    """Appendix H: g(1) values, g(0) = delta_l0, g -> 1 as t -> infinity."""
    assert abs(H.g_closed(1, 1.0) - 2 / 3) < 1e-15
    assert abs(H.g_closed(2, 1.0) - 0.25) < 1e-15
    assert abs(H.g_closed(3, 1.0) - 0.0) < 1e-15
    assert abs(H.g_closed(4, 1.0) + 1 / 24) < 1e-15
    for l in range(0, 5):
        assert H.g_closed(l, 0.0) == (1.0 if l == 0 else 0.0)
        assert abs(H.g_closed(l, 1e4) - 1.0) < 1e-3
    # t = 1: g_l(1) = 1/2 int_0^pi sin k L_l(cos(k/2)) dk
    for l in range(0, 5):
        kap = np.linspace(0, pi, 20001)
        f = 0.5 * np.sin(kap) * H.legendre(l, np.cos(kap / 2))
        assert abs(np.trapezoid(f, kap) - H.g_closed(l, 1.0)) < 1e-7
    # closed forms are continuous at t = 1 (the printed t = 1 values are the limits)
    for l in (2, 4):
        assert abs(H.g_closed(l, 1.0 + 1e-7) - H.g_closed(l, 1.0)) < 1e-5
