"""Angular functions (oracle; test infrastructure only).

Conventions
* Legendre polynomials L_l from their power-series coefficients (numpy.polynomial.legendre).
* Associated Legendre L_l^m(x) (Appendix A): for m >= 0, (-1)^m (1-x^2)^{m/2} d^m L_l/dx^m;
  for m < 0, L_l^{-m} = (-1)^m (l-m)!/(l+m)! L_l^m.
* Spherical harmonics with the Condon-Shortley phase (Sec. 2): for m >= 0
  Y_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) L_l^m(cos theta) e^{i m phi}, and Y_l^{-m} = (-1)^m Y_l^{m*}
  (Eq. sph_prop).  Appendix A's Eq. def_sph writes a further (-1)^m in front of L_l^m, which already
  carries one; the phase factor is applied once here, which is the Condon-Shortley convention the
  paper names.  Every estimator result is independent of this choice.
* Racah-normalised y_l^m = sqrt(4 pi/(2l+1)) Y_l^m (Sec. 2.3).
* Wigner 3j from the Racah closed form in exact rational arithmetic (Appendix F).
* g_l(t): closed forms for l <= 4 (Eqs. g0-g4) and the integral form of Lemma 2 (Appendix H).

Pinned by tests/test_oracle_harmonics.py against: scipy.special.sph_harm_y, the parity and
conjugation relations (Eqs. sph_prop, sphiv), special values Y_l^m(z), the addition theorems
(Eqs. add_theorem, add_associated_L), orthonormality by quadrature, sympy's exact 3j, 3j
orthogonality (Eq. 3j-orthonormal), the Legendre product identities (Eq. legendre), and g_l closed
forms versus the integral forms plus the limits and t = 1 values of Appendix H.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import factorial, pi, sqrt

import numpy as np
from numpy.polynomial import legendre as _npleg
from numpy.polynomial import polynomial as _nppoly


@lru_cache(maxsize=None)
def _legendre_coeffs(ell):
    c = np.zeros(ell + 1)
    c[ell] = 1.0
    return _npleg.leg2poly(c)


def legendre(ell, x):
    """Legendre polynomial L_ell(x)."""
    return _nppoly.polyval(np.asarray(x, dtype=np.float64), _legendre_coeffs(ell))


def assoc_legendre(ell, m, x):
    """Associated Legendre function L_ell^m(x) as defined in Appendix A (with the (-1)^m factor)."""
    x = np.asarray(x, dtype=np.float64)
    am = abs(m)
    if am > ell:
        return np.zeros_like(x)
    deriv = _nppoly.polyder(_legendre_coeffs(ell), am) if am else _legendre_coeffs(ell)
    s2 = np.clip(1.0 - x * x, 0.0, None)
    val = (-1.0) ** am * s2 ** (0.5 * am) * _nppoly.polyval(x, deriv)
    if m < 0:
        val = val * (-1.0) ** am * factorial(ell - am) / factorial(ell + am)
    return val


def _angles(u):
    u = np.asarray(u, dtype=np.float64)
    r = np.sqrt(np.sum(u * u, axis=-1))
    safe = np.where(r > 0, r, 1.0)
    ct = np.clip(u[..., 2] / safe, -1.0, 1.0)
    ct = np.where(r > 0, ct, 1.0)
    phi = np.arctan2(u[..., 1], u[..., 0])
    return ct, phi


def ylm(ell, m, u):
    """Complex Y_ell^m at the direction(s) u (..., 3); u need not be normalised."""
    ct, phi = _angles(u)
    if abs(m) > ell:
        return np.zeros(ct.shape, dtype=np.complex128)
    am = abs(m)
    norm = sqrt((2 * ell + 1) / (4.0 * pi) * factorial(ell - am) / factorial(ell + am))
    pos = norm * assoc_legendre(ell, am, ct) * np.exp(1j * am * phi)
    if m >= 0:
        return pos
    return (-1.0) ** am * np.conj(pos)


def ylm_racah(ell, m, u):
    """Racah-normalised y_ell^m = sqrt(4 pi/(2 ell+1)) Y_ell^m."""
    return sqrt(4.0 * pi / (2 * ell + 1)) * ylm(ell, m, u)


def wigner3j(j1, j2, j3, m1, m2, m3):
    """Wigner 3j symbol for integer arguments (Racah formula, exact rational arithmetic)."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    f = factorial
    tri = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pref = tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    tmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    tmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = Fraction(0)
    for t in range(tmin, tmax + 1):
        den = (f(t) * f(j3 - j2 + t + m1) * f(j3 - j1 + t - m2) * f(j1 + j2 - j3 - t)
               * f(j1 - t - m1) * f(j2 - t + m2))
        s += Fraction((-1) ** t, den)
    sign = -1.0 if (j1 - j2 - m3) % 2 else 1.0
    return sign * float(s) * sqrt(float(pref))


# ---------------------------------------------------------------------------------------------
# g_l(t), Lemma 2
# ---------------------------------------------------------------------------------------------

def g_closed(ell, t):
    """Closed forms of g_ell(t) for ell <= 4 (Appendix H, Eqs. g0-g4); scalar t >= 0."""
    t = float(t)
    if ell == 0:
        return 1.0
    if ell == 1:
        return 2.0 * t / 3.0 if t < 1.0 else 1.0 - 1.0 / (3.0 * t * t)
    if ell == 3:
        return 0.0 if t < 1.0 else (t * t - 1.0) ** 2 / t**4
    if ell == 2:
        if t == 0.0:
            return 0.0
        if t == 1.0:
            return 0.25
        lg = np.log((t + 1.0) / abs(t - 1.0))
        return (2.0 * t * (5.0 * t * t - 3.0) + 3.0 * (t * t - 1.0) ** 2 * lg) / (16.0 * t**3)
    if ell == 4:
        if t == 0.0:
            return 0.0
        if t == 1.0:
            return -1.0 / 24.0
        lg = np.log((t + 1.0) / abs(t - 1.0))
        return (2.0 * t * (81.0 * t**4 - 190.0 * t * t + 105.0)
                + 15.0 * (t * t - 7.0) * (t * t - 1.0) ** 2 * lg) / (192.0 * t**5)
    raise ValueError("closed form only for ell <= 4")


def g_integral(ell, t, npts=400):
    """g_ell(t) from the practical integral form of Appendix H,
    g(t) = 1/(2t) int_{|t-1|}^{t+1} x L_ell((x^2+t^2-1)/(2 x t)) dx, by Gauss-Legendre quadrature."""
    t = float(t)
    if t == 0.0:
        return 1.0 if ell == 0 else 0.0
    a, b = abs(t - 1.0), t + 1.0
    xg, wg = _npleg.leggauss(npts)
    x = 0.5 * (b - a) * xg + 0.5 * (b + a)
    arg = (x * x + t * t - 1.0) / (2.0 * x * t)
    return float(0.5 * (b - a) * np.sum(wg * x * legendre(ell, arg)) / (2.0 * t))


def g_kappa(ell, t, npts=400):
    """g_ell(t) from the kappa-integral of Lemma 2 (Eq. g_ell), split at kappa0 = arccos(-t) for
    t <= 1 with the (-1)^ell sign on the obtuse branch."""
    t = float(t)

    def integrand(kap):
        c = np.cos(kap)
        num = c * c + t * t + 2.0 * t * c
        den = 1.0 + t * t + 2.0 * t * c
        return 0.5 * np.sin(kap) * legendre(ell, np.sqrt(np.clip(num / den, 0.0, 1.0)))

    xg, wg = _npleg.leggauss(npts)

    def quad(a, b):
        if b <= a:
            return 0.0
        k = 0.5 * (b - a) * xg + 0.5 * (b + a)
        return float(0.5 * (b - a) * np.sum(wg * integrand(k)))

    if t <= 1.0:
        k0 = np.arccos(-t)
        return quad(0.0, k0) + (-1.0) ** ell * quad(k0, np.pi)
    return quad(0.0, np.pi)


def g_ell(ell, t):
    """g_ell(t) used by the shot-noise oracle: closed form for ell <= 4, integral form otherwise."""
    if ell <= 4:
        return g_closed(ell, t)
    return g_integral(ell, t)
