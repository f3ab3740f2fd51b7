"""Numbers the paper prints (tests/golden/printed_values.json, each entry with its location) against
mathematics and the oracle."""
import json
import os
from fractions import Fraction

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

from helpers import ROOT
from oracle import power as P

GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "printed_values.json")))


def _leg(ell):
    return npleg.leg2poly([0] * ell + [1])


def test_legendre_product_identities():
    """Eq. legendre: each printed combination of products L_a L_b is the polynomial L_l."""
    for key, terms in GOLD["legendre_products"].items():
        if key == "cite":
            continue
        acc = np.zeros(1)
        for a, b, num, den in terms:
            acc = nppoly.polyadd(acc, (num / den) * nppoly.polymul(_leg(a), _leg(b)))
        want = _leg(int(key))
        acc = np.pad(acc, (0, max(0, len(want) - len(acc))))
        assert np.max(np.abs(acc[:len(want)] - want)) < 1e-12 and np.max(np.abs(acc[len(want):]), initial=0) < 1e-12, key


def test_modified_multipole_coefficients_follow_from_the_products():
    """Eq. Plnew from Eq. legendre: with P_ab = (2(a+b)+1) <L_a L_b |F|^2> (P_a0 = P_a), the term
    c_ab L_a L_b of L_l enters P_lb = (2l+1) <L_l |F|^2> with c_ab (2l+1)/(2(a+b)+1).  The printed
    coefficients and the oracle's table both equal that."""
    for key, terms in GOLD["legendre_products"].items():
        if key == "cite":
            continue
        ell = int(key)
        derived = {(a, b): Fraction(num, den) * Fraction(2 * ell + 1, 2 * (a + b) + 1) for a, b, num, den in terms}
        printed = {(a, b): Fraction(num, den) for a, b, num, den in GOLD["modified_multipoles"][key]}
        assert derived == printed, ell
        oracle = {((0, a) if b == 0 else (a, b)): v for (a, b), v in printed.items()}
        assert oracle == P.PLB_COEFFS[ell], ell


def test_two_index_shot_noise():
    """N_ll = (2(2l)+1) N_0 <L_l^2> = (4l+1)/(2l+1) N_0: the printed 9/5 and 17/9, and the oracle."""
    for key, (num, den) in ((k, v) for k, v in GOLD["two_index_shot_noise"].items() if k != "cite"):
        ell = int(key[0])
        assert Fraction(4 * ell + 1, 2 * ell + 1) == Fraction(num, den)
        assert abs(P.n_shot_two_index(ell, ell, 1.0) - num / den) < 1e-15
    assert P.n_shot_two_index(4, 2, 1.0) == 0.0


def test_transform_counts_of_table_1():
    """Table 1: Cartesian monomials of every even degree (Scoccimarro'15), 2l+1 transforms per even l
    (Hand'17), l+1 with m >= 0 (Sec. 2), and the same up to l_max/2 with the modified multipoles
    (Sec. 3); the oracle's two forms count their transforms as they make them."""
    t = GOLD["fft_counts"]
    spec = dict(n=8, box=100.0, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=1)
    meshes = [np.zeros((8, 8, 8)), np.zeros((8, 8, 8))]
    for i, lmax in enumerate(t["l_max"]):
        evens = list(range(0, lmax + 1, 2))
        mono = sum(sum(1 for a in range(d + 1) for b in range(d + 1 - a)) for d in evens)
        assert mono == t["scoccimarro15"][i] == (lmax + 2) * (lmax + 4) * (2 * lmax + 3) // 24
        assert P.fields_plain(spec, meshes, evens)[1] == t["hand17"][i] == (lmax + 1) * (lmax + 2) // 2
        assert P.fields_symmetric(spec, meshes, evens)[1] == t["m_nonneg"][i] == (lmax + 2) ** 2 // 4
        half = list(range(0, lmax // 2 + 1, 2))
        assert P.fields_symmetric(spec, meshes, half)[1] == t["m_nonneg_plus_modified"][i] == (lmax + 4) ** 2 // 16
