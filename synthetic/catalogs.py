"""Seeded lognormal galaxy catalogues and uniform randoms.

Recipe (stand-in for the Patchy / Molino mocks the paper measures, which are not available here):

* a Gaussian field delta_G on a generation grid with P(k) = 2e4 (k/0.05)^-1.5 exp(-(k/0.5)^2)
  (Mpc/h)^3, each Fourier mode multiplied by the Kaiser factor (1 + beta mu^2), mu = k_z/|k|;
* the lognormal transform delta_LN = exp(delta_G - sigma_G^2/2) - 1;
* Poisson counts per generation cell with mean nbar V_cell (1 + delta_LN), points placed uniformly
  inside their cell, then exactly ``n`` points kept (a random subset, or extra points drawn from the
  same cell intensities when the Poisson total falls short);
* randoms uniform in the box.

Everything is driven by ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def power_law_pk(k):
    """Input power spectrum of the synthetic catalogues, (Mpc/h)^3; zero at k = 0."""
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros_like(k)
    nz = k > 0
    out[nz] = 2.0e4 * (k[nz] / 0.05) ** -1.5 * np.exp(-((k[nz] / 0.5) ** 2))
    return out


def _kgrid(n, box):
    kf = 2.0 * np.pi / box
    kx = np.fft.fftfreq(n, d=1.0 / n) * kf
    kz = np.fft.rfftfreq(n, d=1.0 / n) * kf
    return kx[:, None, None], kx[None, :, None], kz[None, None, :]


def gaussian_field(n, box, rng, kaiser=0.8, pk=power_law_pk):
    """Real Gaussian field on an n^3 grid (index order x, y, z) whose power is pk(k)(1+kaiser mu^2)^2."""
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    kx, ky, kz = _kgrid(n, box)
    kk = np.sqrt(kx**2 + ky**2 + kz**2)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(kk > 0, kz / np.where(kk > 0, kk, 1.0), 0.0)
    vcell = (box / n) ** 3
    amp = np.sqrt(pk(kk) / vcell) * (1.0 + kaiser * mu**2)
    return np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))


def lognormal_positions(n_obj, box, n_gen, seed, kaiser=0.8):
    """Exactly ``n_obj`` lognormal-Poisson points in [0, box)^3 (float64)."""
    rng = np.random.default_rng(seed)
    if n_obj == 0:
        return np.zeros((0, 3))
    dg = gaussian_field(n_gen, box, rng, kaiser=kaiser)
    sig2 = dg.var()
    dln = np.exp(dg - 0.5 * sig2) - 1.0
    vcell = (box / n_gen) ** 3
    lam = (n_obj / box**3) * vcell * (1.0 + dln)
    lam = lam.ravel()
    counts = rng.poisson(lam)
    total = int(counts.sum())
    if total < n_obj:
        p = lam / lam.sum()
        extra = rng.choice(lam.size, size=n_obj - total, p=p)
        counts = counts + np.bincount(extra, minlength=lam.size)
    cells = np.repeat(np.arange(lam.size), counts)
    if cells.size > n_obj:
        keep = rng.choice(cells.size, size=n_obj, replace=False)
        keep.sort()
        cells = cells[keep]
    ix = cells // (n_gen * n_gen)
    iy = (cells // n_gen) % n_gen
    iz = cells % n_gen
    h = box / n_gen
    pos = np.stack([ix, iy, iz], axis=1).astype(np.float64)
    pos += rng.random((cells.size, 3))
    pos *= h
    # keep strictly inside [0, box)
    np.clip(pos, 0.0, np.nextafter(box, 0.0), out=pos)
    return pos


def uniform_positions(n_obj, box, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n_obj, 3)) * box


def survey_box(box, distance):
    """Origin of a cubic box of side ``box`` whose centre sits at ``distance`` along (1,1,1)/sqrt(3)."""
    centre = distance * np.ones(3) / np.sqrt(3.0)
    return centre - 0.5 * box


@dataclass
class Catalog:
    """Positions (n,3), weights (n,), number densities (n,), all float32 by default."""

    pos: np.ndarray
    w: np.ndarray
    nbar: np.ndarray

    @property
    def n(self):
        return int(self.pos.shape[0])

    def astype(self, dtype):
        return Catalog(self.pos.astype(dtype), self.w.astype(dtype), self.nbar.astype(dtype))


def make_survey_catalogs(n_gal, n_ran, box, distance, n_gen, seed, fkp_p0=None,
                         kaiser=0.8, dtype=np.float32):
    """Galaxies + randoms in a box at ``distance`` from an observer at the origin.

    Weights are FKP, w = 1/(1 + nbar P0), when ``fkp_p0`` is given, else 1.  nbar = n_gal / box^3.
    Returns (galaxies, randoms, origin).
    """
    origin = survey_box(box, distance)
    gal = lognormal_positions(n_gal, box, n_gen, seed, kaiser=kaiser) + origin
    ran = uniform_positions(n_ran, box, seed + 7919) + origin
    nbar = n_gal / box**3
    wval = 1.0 / (1.0 + nbar * fkp_p0) if fkp_p0 else 1.0
    g = Catalog(gal.astype(dtype), np.full(n_gal, wval, dtype), np.full(n_gal, nbar, dtype))
    r = Catalog(ran.astype(dtype), np.full(n_ran, wval, dtype), np.full(n_ran, nbar, dtype))
    return g, r, origin


def make_periodic_catalog(n_gal, box, n_gen, seed, kaiser=0.8, dtype=np.float32):
    """A periodic-box lognormal catalogue with unit weights."""
    pos = lognormal_positions(n_gal, box, n_gen, seed, kaiser=kaiser)
    nbar = n_gal / box**3
    return Catalog(pos.astype(dtype), np.ones(n_gal, dtype), np.full(n_gal, nbar, dtype))


def fingerprint(*catalogs):
    """SHA-256 of the catalogues' arrays (positions, weights, densities, in order): identifies the
    exact inputs a stored set of expected values was computed from."""
    import hashlib

    h = hashlib.sha256()
    for c in catalogs:
        for a in (c.pos, c.w, c.nbar):
            a = np.ascontiguousarray(a)
            h.update(str(a.dtype).encode())
            h.update(str(a.shape).encode())
            h.update(a.tobytes())
    return h.hexdigest()
