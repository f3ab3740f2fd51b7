"""Yamamoto power-spectrum multipoles (oracle; test infrastructure only).

Follows Sec. 2.1 and Sec. 3 of the paper:
* catalogue scalars (Sec. 2.1): alpha = sum_g w / sum_r w, I22 = alpha sum_r nbar w^2,
  N_0 = (sum_g w^2 + alpha^2 sum_r w^2)/I22; for the bispectrum I33 = alpha sum_r nbar^2 w^3
  (Sec. 2.2) and the three-point self term S = sum_g w^3 - alpha^3 sum_r w^3 (the cube of the
  FKP field's random term carries (-alpha)^3; reading).  Periodic boxes (no randoms): with
  W = sum_g w and volume V, I22 = W^2/V, I33 = W^3/V^2, N_0 = sum_g w^2/I22, S = sum_g w^3.
* FKP field F(x) = sum_g w W(x - x_g) - alpha sum_r w W(x - x_r) on each interlacing phase; periodic:
  F = sum_g w W - W/n^3 per cell.
* S_l^m(k) = sum_x F(x) Y_l^m(xhat) e^{-i k.x} (Eq. key1) with xhat the unit vector from the
  observer to the grid point (endpoint line of sight), or the fixed line of sight for a global LOS;
  interlaced as 1/2 [S_a + e^{i H (kx+ky+kz)/2} S_b] and divided by W(k) (Eq. compensation).
* Hand+17 form (Eq. hand): F_l(k) = 4 pi/(2l+1) sum_{m=-l}^{l} Y_l^{m*}(khat) S_l^m(k)
  -- 2l+1 transforms; P_l = (2l+1)/I22 <Re F_0 F_l^*>_bin - delta_l0 N_0 (Eq. Hand17); for odd l
  the imaginary part (Sec. 2.1: odd multipoles replace the real part by the imaginary part).
* Symmetric form (Eqs. new_F_ell, pk_final): G_l = 4 pi/(2l+1) [f^0 + 2 sum_{m>=1} f^m] with
  f^m = Y_l^{m*}(khat) S_l^m -- l+1 transforms; P_l^E = Re[(2l+1)/I22 <F_0 G_l^*>] - N_l.
* Space inversion (Eq. F_and_new_G): F_l(k) = 1/2 [G_l(k) + (-1)^l G_l^*(-k)], grid index
  i -> (n - i) mod n (Appendix G).
* Two-index P_ll' = (2(l+l')+1)/I22 <Re F_l F_l'^*> - N_ll' (Eq. Pllp) with
  N_ll' = (2(l+l')+1) N_0 delta_ll'/(2l+1), so N_22 = 9N_0/5 and N_44 = 17N_0/9 (Sec. 3), and the
  modified multipoles of Eq. Plnew.

Pinned by tests/test_oracle_power.py: Hand+17 and symmetric forms agree to 1e-13; the Gaussian
field with fixed amplitudes gives P_0, P_2 exactly; Poisson catalogues give the shot-noise level;
with a global line of sight the modified multipoles equal the direct ones; the P_lb coefficients
follow from the Legendre product identities; the mesh DFT matches a direct per-particle DFT.
"""
from __future__ import annotations

from fractions import Fraction
from math import pi

import numpy as np

from . import harmonics as H
from . import mesh as M


def _fsum(a):
    return float(np.sum(np.asarray(a, dtype=np.float64)))


def catalog_scalars(data, randoms=None, box=None):
    """Scalars of Sec. 2.1 / 2.2.  ``data``/``randoms`` expose .pos, .w, .nbar."""
    wg = np.asarray(data.w, dtype=np.float64)
    if randoms is None:
        vol = float(box) ** 3
        wsum = _fsum(wg)
        i22 = wsum * wsum / vol
        i33 = wsum**3 / vol**2
        return dict(alpha=0.0, I22=i22, I33=i33, N0=_fsum(wg**2) / i22 if i22 > 0 else np.nan,
                    S3=_fsum(wg**3), sum_wg=wsum, sum_wr=0.0, sum_w2=_fsum(wg**2))
    wr = np.asarray(randoms.w, dtype=np.float64)
    nr = np.asarray(randoms.nbar, dtype=np.float64)
    alpha = _fsum(wg) / _fsum(wr)
    i22 = alpha * _fsum(nr * wr**2)
    i33 = alpha * _fsum(nr**2 * wr**3)
    n0 = (_fsum(wg**2) + alpha**2 * _fsum(wr**2)) / i22
    s3 = _fsum(wg**3) - alpha**3 * _fsum(wr**3)
    return dict(alpha=alpha, I22=i22, I33=i33, N0=n0, S3=s3, sum_wg=_fsum(wg), sum_wr=_fsum(wr),
                sum_w2=_fsum(wg**2) + alpha**2 * _fsum(wr**2))


def fkp_meshes(spec, data, randoms, scalars, weight_power=1):
    """FKP field meshes, one per interlacing phase.

    weight_power = 1: F = sum_g w W - alpha sum_r w W (periodic: minus the mean).
    weight_power = 2: the N-field sum_g w^2 W + alpha^2 sum_r w^2 W used by the shot noise (Sec. 5.2).
    """
    shifts = (0.0, 0.5) if spec.get("interlace", 0) else (0.0,)
    return [fkp_mesh_phase(spec, data, randoms, scalars, sh, weight_power) for sh in shifts]


def fkp_mesh_phase(spec, data, randoms, scalars, shift, weight_power=1):
    """One phase of ``fkp_meshes``: grid coordinates shifted by ``shift`` cells (0 or 1/2)."""
    n, box, origin, assign = spec["n"], spec["box"], spec["origin"], spec["assign"]
    sg = M.grid_coords(data.pos, origin, box, n, shift)
    wg = np.asarray(data.w, dtype=np.float64) ** weight_power
    mesh = M.paint(sg, wg, n, assign)
    if randoms is not None:
        sr = M.grid_coords(randoms.pos, origin, box, n, shift)
        coef = -scalars["alpha"] if weight_power == 1 else scalars["alpha"] ** 2
        wr = coef * np.asarray(randoms.w, dtype=np.float64) ** weight_power
        mesh = mesh + M.paint(sr, wr, n, assign)
    elif weight_power == 1:
        mesh = mesh - _fsum(wg) / n**3
    return mesh


def _xhat_dirs(spec, shift_cells):
    n = spec["n"]
    if spec.get("los", "endpoint") == "global":
        d = np.asarray(spec["los_dir"], dtype=np.float64)
        return np.broadcast_to(d / np.linalg.norm(d), (n, n, n, 3))
    pts = M.sample_positions(n, spec["box"], spec["origin"], shift_cells)
    return pts - np.asarray(spec.get("observer", (0.0, 0.0, 0.0)), dtype=np.float64)


def ylm_transform(spec, meshes, ell, m):
    """Interlaced, compensated S_l^m(k) on the full grid."""
    n = spec["n"]
    shifts = (0.0, 0.5) if len(meshes) == 2 else (0.0,)
    parts = []
    for mesh, sh in zip(meshes, shifts):
        y = H.ylm(ell, m, _xhat_dirs(spec, sh))
        parts.append(np.fft.fftn(mesh * y))
    if len(parts) == 2:
        s = 0.5 * (parts[0] + M.interlace_phase(n) * parts[1])
    else:
        s = parts[0]
    return s / M.window(n, spec["assign"])


def _khat(spec):
    (kx, ky, kz), _ = M.kvectors(spec["n"], spec["box"])
    return np.stack(np.broadcast_arrays(kx, ky, kz), axis=-1)


def fields_plain(spec, meshes, ells):
    """F_l(k) by the Hand+17 sum over all 2l+1 values of m (Eq. hand); also counts transforms."""
    kh = _khat(spec)
    out, nfft = {}, 0
    for ell in ells:
        acc = np.zeros((spec["n"],) * 3, dtype=np.complex128)
        for m in range(-ell, ell + 1):
            acc += np.conj(H.ylm(ell, m, kh)) * ylm_transform(spec, meshes, ell, m)
            nfft += 1
        out[ell] = 4.0 * pi / (2 * ell + 1) * acc
    return out, nfft


def fields_symmetric(spec, meshes, ells):
    """G_l(k) of Eq. new_F_ell from the m >= 0 transforms only; also counts transforms."""
    kh = _khat(spec)
    out, nfft = {}, 0
    for ell in ells:
        acc = np.conj(H.ylm(ell, 0, kh)) * ylm_transform(spec, meshes, ell, 0)
        nfft += 1
        for m in range(1, ell + 1):
            acc = acc + 2.0 * np.conj(H.ylm(ell, m, kh)) * ylm_transform(spec, meshes, ell, m)
            nfft += 1
        out[ell] = 4.0 * pi / (2 * ell + 1) * acc
    return out, nfft


def space_invert(g):
    """g(-k) on the fft grid: index i -> (n - i) mod n along every axis."""
    return np.roll(np.flip(g, axis=(0, 1, 2)), 1, axis=(0, 1, 2))


def f_from_g(g, ell):
    """F_l(k) = 1/2 [G_l(k) + (-1)^l G_l^*(-k)] (Eq. F_and_new_G)."""
    return 0.5 * (g + (-1.0) ** ell * np.conj(space_invert(g)))


# Coefficients of Eq. Plnew (modified multipoles from two-index spectra)
PLB_COEFFS = {
    4: {(2, 2): Fraction(35, 18), (0, 2): Fraction(-1), (0, 0): Fraction(-7, 2)},
    6: {(4, 2): Fraction(11, 5), (0, 4): Fraction(-52, 63), (0, 2): Fraction(-286, 175)},
    8: {(4, 4): Fraction(1287, 490), (4, 2): Fraction(-374, 245), (0, 4): Fraction(-3553, 15435),
        (0, 2): Fraction(-1326, 8575), (0, 0): Fraction(-2431, 490)},
}


def _part(ell, z):
    """Re z for even l, Im z for odd l (the odd-multipole estimator of Sec. 2.1)."""
    return np.imag(z) if ell % 2 else np.real(z)


def n_shot_two_index(ell, ellp, n0):
    """N_ll' = (2(l+l')+1) N_0 <L_l L_l'> over directions = (2(l+l')+1) N_0 delta_ll'/(2l+1)."""
    if ell != ellp:
        return 0.0
    return (2 * (ell + ellp) + 1) * n0 / (2 * ell + 1)


def power_from_fields(spec, fields, kbins, ells, scalars, modified=(), fields_kind="F"):
    """Binned P_l (and the modified multipoles) from Fourier fields.

    Bins without modes report 0 for every multipole (convention shared with the GPU library).

    fields_kind = "F": fields are F_l (Hand+17 or inverted); "G": fields are G_l and P_l uses
    Re<F_0 G_l^*> (Eq. pk_final) while the two-index spectra use F_l from Eq. F_and_new_G.
    """
    kmin, dk, nb = kbins
    b, kmag = M.bin_index(spec["n"], spec["box"], kmin, dk, nb)
    i22, n0 = scalars["I22"], scalars["N0"]
    f0 = fields[0]
    res = {"P": {}, "Pll": {}, "Pmod": {}}
    kmean, cnt = M.bin_average(kmag, b, nb)
    res["k_eff"], res["nmodes"] = kmean, cnt
    empty = cnt == 0
    internal = sorted(set(ells) | ({0, 2, 4} if modified else set()))
    pl = {}
    for ell in internal:
        v = _part(ell, f0 * np.conj(fields[ell]))
        mean, _ = M.bin_average(v, b, nb)
        pl[ell] = np.where(empty, 0.0, (2 * ell + 1) / i22 * mean - (n0 if ell == 0 else 0.0))
    for ell in ells:
        res["P"][ell] = pl[ell]
    if modified:
        if fields_kind == "G":
            ff = {ell: f_from_g(fields[ell], ell) for ell in fields}
        else:
            ff = fields
        need = {(2, 2), (4, 2), (4, 4)}
        for (a, c) in need:
            if a in ff and c in ff:
                v = np.real(ff[a] * np.conj(ff[c]))
                mean, _ = M.bin_average(v, b, nb)
                res["Pll"][(a, c)] = np.where(empty, 0.0, (2 * (a + c) + 1) / i22 * mean
                                              - n_shot_two_index(a, c, n0))
        for lb in modified:
            acc = 0.0
            for key, coef in PLB_COEFFS[lb].items():
                if key[0] == 0:
                    term = pl[key[1]]
                else:
                    term = res["Pll"][key]
                acc = acc + float(coef) * term
            res["Pmod"][lb] = acc
    return res


def power_multipoles(spec, data, randoms, kbins, ells=(0, 2, 4), modified=(), method="plain"):
    """Full oracle measurement: catalogue -> meshes -> transforms -> binned multipoles.

    method = "plain" (Hand+17, 2l+1 transforms per l) or "symmetric" (m >= 0 only).
    """
    sc = catalog_scalars(data, randoms, spec["box"])
    meshes = fkp_meshes(spec, data, randoms, sc)
    need = sorted(set(ells) | {0} | ({2, 4} if modified else set()))
    if method == "plain":
        fields, nfft = fields_plain(spec, meshes, need)
        res = power_from_fields(spec, fields, kbins, ells, sc, modified, "F")
    else:
        fields, nfft = fields_symmetric(spec, meshes, need)
        res = power_from_fields(spec, fields, kbins, ells, sc, modified, "G")
    res["scalars"] = sc
    res["n_transforms_per_phase"] = nfft
    return res


def cross_power_multipoles(spec, data_a, randoms_a, data_b, randoms_b, kbins, ells=(0, 2, 4)):
    """Cross multipoles of two tracers A and B (multi-tracer spectra; the paper's toolkit measures
    auto and cross spectra, Sec. 6, without printing the cross form).  Readings: the Y_lm weighting
    (line of sight) sits on tracer B, P_l^AB = (2l+1)/I22^AB <Re F_0^A F_l^B*>_bin with F_l^B the
    Hand+17 field of B; the normalisation I22^AB = sqrt(I22^A I22^B) (exact when the two
    selections n w have the same shape); no shot noise is subtracted (disjoint tracers share no
    object).  Pinned by: the cross spectrum of a tracer with itself equals its auto spectrum plus
    N_0 (l = 0); with a global line of sight P_l^AB = P_l^BA."""
    sa = catalog_scalars(data_a, randoms_a, spec["box"])
    sb = catalog_scalars(data_b, randoms_b, spec["box"])
    fa, _ = fields_plain(spec, fkp_meshes(spec, data_a, randoms_a, sa), [0])
    need = sorted(set(ells) | {0})
    fb, _ = fields_plain(spec, fkp_meshes(spec, data_b, randoms_b, sb), need)
    kmin, dk, nb = kbins
    b, kmag = M.bin_index(spec["n"], spec["box"], kmin, dk, nb)
    i22 = np.sqrt(sa["I22"] * sb["I22"])
    kmean, cnt = M.bin_average(kmag, b, nb)
    empty = cnt == 0
    res = {"P": {}, "k_eff": kmean, "nmodes": cnt, "I22": i22, "scalars_a": sa, "scalars_b": sb}
    for ell in ells:
        mean, _ = M.bin_average(_part(ell, fa[0] * np.conj(fb[ell])), b, nb)
        res["P"][ell] = np.where(empty, 0.0, (2 * ell + 1) / i22 * mean)
    return res


def power_monopole_rfft(spec, data, randoms, kbins):
    """P_0 alone (Eq. Hand17 with l = 0, where no Y_lm weighting is needed) from real-to-complex
    transforms, for meshes too large for the full-m path.  Each stored mode of the half grid
    (kz > 0) also stands for -k, whose |X|^2 is equal; the kz = 0 plane holds both members of each
    pair.  Returns (P_0, N_modes, scalars).  Pinned to power_multipoles in the tests."""
    n = spec["n"]
    sc = catalog_scalars(data, randoms, spec["box"])
    meshes = fkp_meshes(spec, data, randoms, sc)
    parts = [np.fft.rfftn(m) for m in meshes]
    ii = M.int_freqs(n)
    iz = np.arange(n // 2 + 1)
    a = np.pi * ii / n
    az = np.pi * iz / n
    if len(parts) == 2:
        ph = np.exp(1j * (a[:, None, None] + a[None, :, None] + az[None, None, :]))
        X = 0.5 * (parts[0] + ph * parts[1])
        del ph
    else:
        X = parts[0]
    del parts
    p = spec["assign"]
    s1 = np.where(ii == 0, 1.0, np.sin(a) / np.where(ii == 0, 1.0, a)) ** p
    sz = np.where(iz == 0, 1.0, np.sin(az) / np.where(iz == 0, 1.0, az)) ** p
    X /= s1[:, None, None] * s1[None, :, None] * sz[None, None, :]
    kmin, dk, nb = kbins
    kf = 2.0 * np.pi / spec["box"]
    n2 = (ii[:, None, None] ** 2 + ii[None, :, None] ** 2 + iz[None, None, :] ** 2).astype(np.float64)
    b = np.floor((kf * np.sqrt(n2) - kmin) / dk)
    ok = (b >= 0) & (b < nb) & (n2 > 0)
    nyq = -(n // 2)
    ok &= (ii[:, None, None] != nyq) & (ii[None, :, None] != nyq) & (iz[None, None, :] != n // 2)
    wgt = np.where(iz == 0, 1.0, 2.0)[None, None, :] * ok
    bb = np.where(ok, b, 0).astype(np.int64).ravel()
    cnt = np.bincount(bb, weights=wgt.ravel(), minlength=nb)
    s0 = np.bincount(bb, weights=(wgt * (X.real**2 + X.imag**2)).ravel(), minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        p0 = np.where(cnt > 0, s0 / np.where(cnt > 0, cnt, 1.0) / sc["I22"] - sc["N0"], 0.0)
    return p0, cnt, sc


def direct_dft(pos, weights, kvecs, origin):
    """sum_p w_p e^{-i k.(x_p - origin)} for a list of k vectors (brute force, for pins)."""
    x = np.asarray(pos, dtype=np.float64) - np.asarray(origin, dtype=np.float64)
    ph = np.asarray(kvecs) @ x.T
    return np.exp(-1j * ph) @ np.asarray(weights, dtype=np.float64)


class HalfSpectrumPower:
    """Symmetric-form multipoles (Eqs. new_F_ell, F_and_new_G, pk_final, Pllp, Plnew) evaluated on
    the half Fourier grid of real-to-complex transforms, for meshes too large for the full-grid
    forms above (the 512^3 survey workload).

    For m >= 0 the weighted field F(x) Y_l^m(xhat) is split into its real and imaginary parts, whose
    transforms A_l^m, B_l^m are Hermitian, so S_l^m = A_l^m + i B_l^m.  Inserting G_l of
    Eq. new_F_ell into the space inversion of Eq. F_and_new_G, with Y_l^m(-khat) = (-1)^l Y_l^m(khat)
    (Eq. sph_prop) and S_l^m(-k)^* = A_l^m(k) - i B_l^m(k), gives at every mode
        F_l(k) = 4 pi/(2l+1) [Y_l^0 A_l^0 + 2 sum_{m>=1} (Re Y_l^m(khat) A_l^m + Im Y_l^m(khat) B_l^m)],
    which obeys F_l(-k) = (-1)^l F_l(k)^*.  Hence for a mode pair (k, -k) both members carry the
    same Re F_0 F_l^* (even l), Im F_0 F_l^* (odd l) and Re F_l F_l'^*: a stored mode with
    0 < k_z < k_N stands for two modes of the full grid, a mode of the k_z = 0 plane for one (that
    plane holds both members of each pair); the Nyquist planes and DC are excluded as in
    ``mesh.bin_index``.  Interlacing and the compensation 1/W are per-mode factors, so each phase
    accumulates its own F_l before the phases are combined.  Same outputs as ``power_multipoles``.

    The work is a fixed list of stages (``stages()``): catalogue scalars and the painting of each
    interlacing phase, then one stage per phase and (l, m >= 0) pair (the Y_l^m-weighted transforms
    and their accumulation), then the phase combination and the binning.  ``workers`` is passed to
    scipy.fft.

    Pinned by tests/test_oracle_power.py: equal to the full-grid Hand+17 form (Eq. hand) and to
    the full-grid symmetric form to rounding, for even and odd l, the two-index and modified
    multipoles, endpoint and global lines of sight, CIC and interlaced TSC, meshes of 2^k and
    3 * 2^k cells."""

    def __init__(self, spec, data, randoms, kbins, ells=(0, 2, 4), modified=(), two_index=(),
                 workers=None):
        self.spec, self.data, self.randoms, self.kbins = spec, data, randoms, kbins
        self.ells = tuple(ells)
        self.modified = tuple(modified)
        self.two_index = tuple(tuple(p) for p in two_index)
        self.workers = workers
        need = set(self.ells) | {0}
        if self.modified:
            need |= {2, 4}
        for a, c in self.two_index:
            need |= {a, c}
        self.need = sorted(need)
        self.nph = 2 if spec.get("interlace", 0) else 1
        self.meshes = [None] * self.nph
        self.acc = [{} for _ in range(self.nph)]
        self.dirs = None
        self.result = None

    # --- half-grid geometry -------------------------------------------------------------------
    def _half_ints(self):
        n = self.spec["n"]
        ii = M.int_freqs(n)
        iz = np.arange(n // 2 + 1)
        return ii[:, None, None], ii[None, :, None], iz[None, None, :]

    def _khat_half(self):
        ix, iy, iz = self._half_ints()
        return np.stack(np.broadcast_arrays(ix, iy, iz), axis=-1).astype(np.float64)

    def _rfft(self, x):
        import scipy.fft as sfft

        return sfft.rfftn(x, workers=self.workers)

    # --- stages --------------------------------------------------------------------------------
    def stages(self):
        out = []
        for ph in range(self.nph):
            out.append((f"paint phase {ph}", lambda ph=ph: self._paint(ph)))
        for ph in range(self.nph):
            last = None
            for ell in self.need:
                for m in range(0, ell + 1):
                    last = (ell, m)
            for ell in self.need:
                for m in range(0, ell + 1):
                    out.append((f"transform phase {ph} l={ell} m={m}",
                                lambda ph=ph, ell=ell, m=m, fin=((ell, m) == last): self._transform(ph, ell, m, fin)))
        out.append(("combine and bin", self._finish))
        return out

    def _paint(self, ph):
        if ph == 0:
            self.scalars = catalog_scalars(self.data, self.randoms, self.spec["box"])
        self.meshes[ph] = fkp_mesh_phase(self.spec, self.data, self.randoms, self.scalars, 0.5 * ph)

    def _transform(self, ph, ell, m, last):
        if self.dirs is None:
            self.dirs = _xhat_dirs(self.spec, 0.5 * ph)
        y = H.ylm(ell, m, self.dirs)
        mesh = self.meshes[ph]
        kh = self._khat_half()
        yk = H.ylm(ell, m, kh)
        del kh
        c = 4.0 * pi / (2 * ell + 1) * (1.0 if m == 0 else 2.0)
        term = c * np.real(yk) * self._rfft(mesh * np.real(y))
        if m > 0:
            term += c * np.imag(yk) * self._rfft(mesh * np.imag(y))
        del y, yk
        if ell in self.acc[ph]:
            self.acc[ph][ell] += term
        else:
            self.acc[ph][ell] = term
        if last:
            self.dirs = None
            self.meshes[ph] = None

    def _finish(self):
        spec, n = self.spec, self.spec["n"]
        ix, iy, iz = self._half_ints()
        a = np.pi / n
        p = spec["assign"]

        def sinc_p(i):
            x = a * i.astype(np.float64)
            return np.where(i == 0, 1.0, np.sin(x) / np.where(i == 0, 1.0, x)) ** p

        win = sinc_p(ix) * sinc_p(iy) * sinc_p(iz)
        if self.nph == 2:
            ph = np.exp(1j * a * (ix + iy + iz))
            F = {ell: 0.5 * (self.acc[0][ell] + ph * self.acc[1][ell]) / win for ell in self.need}
            del ph
        else:
            F = {ell: self.acc[0][ell] / win for ell in self.need}
        self.acc = None
        kmin, dk, nb = self.kbins
        kf = 2.0 * np.pi / spec["box"]
        n2 = (ix * ix + iy * iy + iz * iz).astype(np.float64)
        kmag = kf * np.sqrt(n2)
        b = np.floor((kmag - kmin) / dk)
        ok = (b >= 0) & (b < nb) & (n2 > 0)
        ok &= (ix != -(n // 2)) & (iy != -(n // 2)) & (iz != n // 2)
        wgt = (np.where(iz == 0, 1.0, 2.0) * ok).ravel()
        bb = np.where(ok, b, 0).astype(np.int64).ravel()
        cnt = np.bincount(bb, weights=wgt, minlength=nb)
        ksum = np.bincount(bb, weights=wgt * np.broadcast_to(kmag, ok.shape).ravel(), minlength=nb)
        empty = cnt == 0
        safe = np.where(empty, 1.0, cnt)

        def bin_mean(v):
            return np.bincount(bb, weights=wgt * v.ravel(), minlength=nb) / safe

        sc = self.scalars
        i22, n0 = sc["I22"], sc["N0"]
        res = {"P": {}, "Pll": {}, "Pmod": {}, "k_eff": np.where(empty, 0.0, ksum / safe), "nmodes": cnt,
               "scalars": sc}
        internal = sorted(set(self.ells) | ({0, 2, 4} if self.modified else set()))
        pl = {}
        for ell in internal:
            mean = bin_mean(_part(ell, F[0] * np.conj(F[ell])))
            pl[ell] = np.where(empty, 0.0, (2 * ell + 1) / i22 * mean - (n0 if ell == 0 else 0.0))
        for ell in self.ells:
            res["P"][ell] = pl[ell]
        need2 = set(self.two_index)
        if self.modified:
            need2 |= {(2, 2), (4, 2), (4, 4)}
        for (l1, l2) in sorted(need2):
            mean = bin_mean(np.real(F[l1] * np.conj(F[l2])))
            res["Pll"][(l1, l2)] = np.where(empty, 0.0, (2 * (l1 + l2) + 1) / i22 * mean
                                            - n_shot_two_index(l1, l2, n0))
        for lb in self.modified:
            acc = 0.0
            for key, coef in PLB_COEFFS[lb].items():
                acc = acc + float(coef) * (pl[key[1]] if key[0] == 0 else res["Pll"][key])
            res["Pmod"][lb] = acc
        self.result = res


def power_multipoles_rfft(spec, data, randoms, kbins, ells=(0, 2, 4), modified=(), two_index=(),
                          workers=None):
    """Catalogue -> binned multipoles by ``HalfSpectrumPower`` (every stage in order)."""
    run = HalfSpectrumPower(spec, data, randoms, kbins, ells, modified, two_index, workers)
    for _, stage in run.stages():
        stage()
    return run.result
