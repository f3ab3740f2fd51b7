"""Pins for oracle.mesh: the k-binning against lattice-point counts and the mass assignment against
the textbook CIC / TSC weights (Sec. 3.1), independent of the binning and painting code."""
import itertools

import numpy as np
import pytest

from oracle import mesh as M


def _r3(m):
    """Number of integer vectors (i, j, l) with i^2 + j^2 + l^2 = m, signs and order counted, by
    enumeration of a cube that holds them all."""
    r = int(np.ceil(np.sqrt(m)))
    return sum(1 for v in itertools.product(range(-r, r + 1), repeat=3) if v[0] ** 2 + v[1] ** 2 + v[2] ** 2 == m)


def test_lattice_counts():
    """The enumeration against values worked out by hand (e.g. 9 = 3^2 in 6 ways plus 2^2 + 2^2 + 1^2
    in 3 x 8; 26 = 5^2 + 1^2 in 6 x 4 plus 4^2 + 3^2 + 1^2 in 6 x 8) and Legendre's three-square
    theorem (no representation of 4^a (8b + 7))."""
    by_hand = {0: 1, 1: 6, 2: 12, 3: 8, 4: 6, 5: 24, 6: 24, 8: 12, 9: 30, 10: 24, 11: 24, 12: 8, 13: 24,
               14: 48, 16: 6, 17: 48, 18: 36, 19: 24, 20: 24, 21: 48, 22: 24, 24: 24, 25: 30, 26: 72}
    for m, v in by_hand.items():
        assert _r3(m) == v, m
    for m in (7, 15, 23, 28, 31, 39, 47, 55, 60, 63):
        assert _r3(m) == 0, m


@pytest.mark.parametrize("n", [16, 24])
def test_shell_mode_counts_are_lattice_counts(n):
    """Bins 0.01 k_f wide isolate the shells |k|^2 = m k_f^2: each holds exactly r3(m) modes, for every
    shell whose vectors fit inside the Nyquist cube; the empty shells (m = 4^a (8b + 7)) hold none."""
    box = 2.0 * np.pi                       # k_f = 1
    kmin, dk = 0.005, 0.01                  # shell m at 100 sqrt(m) - 1/2 bin widths
    mmax = (n // 2 - 1) ** 2
    nbins = int(np.floor((np.sqrt(mmax) - kmin) / dk)) + 1
    b, _ = M.bin_index(n, box, kmin, dk, nbins)
    _, cnt = M.bin_average(np.ones(b.shape), b, nbins)
    expect = np.zeros(nbins)
    for m in range(1, mmax + 1):
        at = (np.sqrt(m) - kmin) / dk
        # the test's own design: no shell within 1e-7 bin widths of an edge (the rounding of |k| is
        # about 1e-13 bin widths), so the floor is the same in any exact evaluation
        assert abs(at - np.round(at)) > 1e-7
        expect[int(np.floor(at))] += _r3(m)
    np.testing.assert_array_equal(cnt, expect)


@pytest.mark.parametrize("n", [8, 16, 24])
def test_every_mode_inside_the_nyquist_cube_is_binned_once(n):
    """One bin covering every |k| > 0: (n - 1)^3 - 1 modes, the integer vectors with components in
    (-n/2, n/2) other than 0 (the Nyquist planes and the DC mode left out)."""
    box = 2.0 * np.pi
    b, _ = M.bin_index(n, box, 0.5, float(n), 1)
    assert int((b == 0).sum()) == (n - 1) ** 3 - 1
    assert int((b >= 0).sum()) == (n - 1) ** 3 - 1


def _one_d(n, cells):
    w = np.zeros(n)
    for c, v in cells.items():
        w[c % n] += v
    return w


@pytest.mark.parametrize("s,assign,cells", [
    (3.0, 3, {2: 0.125, 3: 0.75, 4: 0.125}),   # TSC on a grid point: 3/4 there, 1/8 on each side
    (3.5, 3, {3: 0.5, 4: 0.5}),                # TSC half-way: 1/2 on the two nearest points
    (3.25, 3, {2: 0.03125, 3: 0.6875, 4: 0.28125}),   # TSC at d = 1/4: (1/4)^2/2, 3/4 - 1/16, (3/4)^2/2
    (7.5, 3, {7: 0.5, 0: 0.5}),                # periodic wrap
    (0.0, 3, {-1: 0.125, 0: 0.75, 1: 0.125}),
    (3.0, 2, {3: 1.0}),                        # CIC on a grid point
    (3.25, 2, {3: 0.75, 4: 0.25}),             # CIC: linear in the distance to the two points
    (7.75, 2, {7: 0.25, 0: 0.75}),
])
def test_assignment_weights(s, assign, cells):
    """A unit particle at grid coordinate (s, s + 1, s + 2) paints the product of the one-dimensional
    CIC / TSC weights (Hockney and Eastwood's kernels) of each axis."""
    n = 8
    m = M.paint(np.array([[s, s + 1.0, s + 2.0]]), np.array([1.0]), n, assign)
    wx = _one_d(n, cells)
    wy = np.roll(wx, 1)
    wz = np.roll(wx, 2)
    np.testing.assert_allclose(m, np.einsum("i,j,k->ijk", wx, wy, wz), rtol=0, atol=1e-15)


@pytest.mark.parametrize("assign", [2, 3])
def test_assignment_conserves_mass_and_centre(assign):
    """Any particle away from the periodic edge (no tap wraps): the weights sum to 1 and their centre
    of mass is the particle (CIC and TSC both reproduce linear functions)."""
    rng = np.random.default_rng(4)
    n = 16
    s = rng.uniform(2.0, 13.0, size=(50, 3))
    for p in s:
        m = M.paint(p[None, :], np.array([1.0]), n, assign)
        assert m.sum() == pytest.approx(1.0, abs=1e-14)
        idx = np.arange(n, dtype=np.float64)
        for a in range(3):
            marg = m.sum(axis=tuple(x for x in range(3) if x != a))
            assert float(marg @ idx) == pytest.approx(p[a], abs=1e-12)


@pytest.mark.parametrize("assign", [2, 3])
def test_window_is_the_fourier_transform_of_the_kernel(assign):
    """Averaged over the particle's offset s within a cell, e^{i k.s} times the mesh DFT of one painted
    particle is the continuous Fourier transform of the assignment kernel, prod_a sinc^p(k_a H / 2):
    the compensation W(k) of Sec. 3.1.  By Poisson summation the M-point midpoint average over each
    axis differs from it only by the aliases k + 2 pi M m / H (m != 0), at most
    2 zeta(p) (pi (M - 1/2))^-p per axis; the tolerance is three times that (three axes)."""
    n, mo = 8, 48
    off = (np.arange(mo) + 0.5) / mo
    s = np.stack(np.meshgrid(off, off, off, indexing="ij"), -1).reshape(-1, 3) + np.array([3.0, 2.0, 5.0])
    w = M.window(n, assign)
    zeta = {2: np.pi ** 2 / 6, 3: 1.2020569031595942}[assign]
    tol = 3 * 2 * zeta * (np.pi * (mo - 0.5)) ** (-assign) * 1.01
    for i in [(1, 0, 0), (2, 1, 0), (3, 3, 1), (-3, 2, -1), (1, 1, 1), (3, -3, 3), (0, 0, 2)]:
        phase = s @ (2.0 * np.pi * np.array(i) / n)      # k.s with s in cells
        mesh_c = M.paint(s, np.cos(phase), n, assign)
        mesh_s = M.paint(s, np.sin(phase), n, assign)
        j = tuple(v % n for v in i)
        avg = (np.fft.fftn(mesh_c)[j] + 1j * np.fft.fftn(mesh_s)[j]) / len(s)
        assert abs(avg - w[j]) < tol, (i, avg, w[j], tol)
