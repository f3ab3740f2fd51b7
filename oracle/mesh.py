"""Mesh construction, Fourier grid and k-binning (oracle; test infrastructure only).

Mesh: cubic, n^3 cells of size H = box/n covering [origin, origin + box) (periodic index wrap).
Array index order is (x, y, z).  A particle at grid coordinate s = (pos - origin) n/box is assigned by
* CIC (assign = 2): base i0 = floor(s), d = s - i0, weights (1-d, d) at (i0, i0+1);
* TSC (assign = 3): base i0 = floor(s + 1/2), d = s - i0,
  weights (0.5(0.5-d)^2, 0.75-d^2, 0.5(0.5+d)^2) at (i0-1, i0, i0+1).
The interlaced second mesh (phase b) assigns s + 1/2, so its grid point j sits at
origin + (j - 1/2) H.  The paper applies the mass-assignment compensation of Sec. 3.1
(Eq. compensation, W = prod_i sinc(pi k_i / 2 k_N)^p with p = 2 for CIC, 3 for TSC) and cites the
standard interlacing scheme; the sample-point and half-cell conventions above are this oracle's
reading, stated once and shared in meaning (not in code) with the GPU library.

Fourier transforms use e^{-i k.x} with x measured from the mesh origin (numpy.fft.fftn); for
phase b the half-cell offset is restored by the factor e^{i H (kx+ky+kz)/2}.

k-bins: modes on the full grid with every integer index in (-n/2, n/2) (Nyquist planes excluded,
the paper notes they contribute nothing, Appendix G), DC excluded, bin
b = floor((k_f sqrt(i^2+j^2+l^2) - kmin)/dk), kept when 0 <= b < nbins (half-open bins).
The paper writes the shell boundaries both with strict and with non-strict inequalities (Sec. 2.3
and Appendix E); half-open is the reading used here.

Pinned by tests/test_oracle_mesh.py: mode counts per thin shell equal the number of integer vectors
of that length (enumerated; Legendre's three-square theorem for the empty shells), one bin over
every |k| > 0 holds the (n - 1)^3 - 1 modes inside the Nyquist cube, and the CIC / TSC weights at
grid points, half cells and quarter cells are the textbook values, conserve mass and reproduce the
particle's position, and the window W(k) is the Fourier transform of the painted kernel (the mesh
DFT of one particle averaged over its offset in the cell, to the alias bound of that average); by
tests/test_oracle_power.py: the painted mesh's DFT equals the per-particle
DFT (CIC on grid points exactly, compensated CIC / TSC at low k), the compensated Poisson spectrum
equals the closed-form alias sum of the window, and interlacing removes the leading alias.
"""
from __future__ import annotations

import numpy as np


def grid_coords(pos, origin, box, n, shift=0.0):
    """s = (pos - origin) * (n/box) (+ shift), float64.

    The cell a particle lands in is an integer decided in floating point; the GPU library makes
    the same decision with the same float64 expression (difference, then product with n/box)."""
    inv_h = n / box
    return (np.asarray(pos, dtype=np.float64) - np.asarray(origin, dtype=np.float64)) * inv_h + shift


def paint(s, weights, n, assign):
    """Sum of weight * window over particles at grid coordinates s (npart, 3); returns (n,n,n)."""
    s = np.asarray(s, dtype=np.float64)
    weights = np.asarray(weights, dtype=np.float64)
    mesh = np.zeros(n * n * n, dtype=np.float64)
    if s.shape[0] == 0:
        return mesh.reshape(n, n, n)
    if assign == 2:
        i0 = np.floor(s)
        d = s - i0
        taps = [(0, 1.0 - d), (1, d)]
    elif assign == 3:
        i0 = np.floor(s + 0.5)
        d = s - i0
        taps = [(-1, 0.5 * (0.5 - d) ** 2), (0, 0.75 - d * d), (1, 0.5 * (0.5 + d) ** 2)]
    else:
        raise ValueError("assign must be 2 (CIC) or 3 (TSC)")
    i0 = i0.astype(np.int64)
    for ox, wx in taps:
        ix = (i0[:, 0] + ox) % n
        for oy, wy in taps:
            iy = (i0[:, 1] + oy) % n
            wxy = wx[:, 0] * wy[:, 1]
            for oz, wz in taps:
                iz = (i0[:, 2] + oz) % n
                flat = (ix * n + iy) * n + iz
                mesh += np.bincount(flat, weights=weights * wxy * wz[:, 2], minlength=n**3)
    return mesh.reshape(n, n, n)


def sample_positions(n, box, origin, shift_cells=0.0):
    """Physical positions (n,n,n,3) of the grid points; shift_cells = 0 (phase a) or 0.5 (phase b)."""
    h = box / n
    j = (np.arange(n, dtype=np.float64) - shift_cells) * h
    o = np.asarray(origin, dtype=np.float64)
    x = o[0] + j[:, None, None] + 0.0 * j[None, :, None] + 0.0 * j[None, None, :]
    y = o[1] + 0.0 * j[:, None, None] + j[None, :, None] + 0.0 * j[None, None, :]
    z = o[2] + 0.0 * j[:, None, None] + 0.0 * j[None, :, None] + j[None, None, :]
    return np.stack([x, y, z], axis=-1)


def int_freqs(n):
    """Integer frequency index per axis in numpy fft order: 0..n/2-1, -n/2..-1."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def kvectors(n, box):
    """(kx, ky, kz) broadcastable arrays in h/Mpc and the integer index arrays."""
    kf = 2.0 * np.pi / box
    ii = int_freqs(n)
    ix, iy, iz = ii[:, None, None], ii[None, :, None], ii[None, None, :]
    return (kf * ix, kf * iy, kf * iz), (ix, iy, iz)


def window(n, assign):
    """W(k) = prod_i sinc(pi k_i/(2 k_N))^p on the full grid; pi k_i/(2 k_N) = pi i/n."""
    ii = int_freqs(n).astype(np.float64)
    a = np.pi * ii / n
    with np.errstate(invalid="ignore", divide="ignore"):
        sc = np.where(ii == 0, 1.0, np.sin(a) / np.where(ii == 0, 1.0, a))
    w1 = sc**assign
    return w1[:, None, None] * w1[None, :, None] * w1[None, None, :]


def interlace_phase(n):
    """e^{i H (kx+ky+kz)/2} = e^{i pi (i+j+l)/n} on the full grid."""
    ii = int_freqs(n).astype(np.float64)
    a = np.pi * ii / n
    return np.exp(1j * (a[:, None, None] + a[None, :, None] + a[None, None, :]))


def bin_index(n, box, kmin, dk, nbins):
    """Bin index per full-grid mode (-1 where excluded), and |k|."""
    _, (ix, iy, iz) = kvectors(n, box)
    kf = 2.0 * np.pi / box
    n2 = (ix * ix + iy * iy + iz * iz).astype(np.float64)
    kmag = kf * np.sqrt(n2)
    b = np.floor((kmag - kmin) / dk)
    ok = (b >= 0) & (b < nbins) & (n2 > 0)
    nyq = -(n // 2)
    ok &= (ix != nyq) & (iy != nyq) & (iz != nyq)
    b = np.where(ok, b, -1).astype(np.int64)
    return b, kmag


def bin_average(values, b, nbins):
    """Per-bin mean of ``values`` over modes with b >= 0; returns (mean, count)."""
    sel = b >= 0
    cnt = np.bincount(b[sel], minlength=nbins).astype(np.float64)
    s = np.bincount(b[sel], weights=np.asarray(values)[sel], minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(cnt > 0, s / np.where(cnt > 0, cnt, 1.0), 0.0)
    return mean, cnt
