"""Sugiyama TripoSH bispectrum multipoles B_{l1 l2 L}(k1, k2) (oracle; test infrastructure only).

Eq. sugi_estimator with the fields of Eq. F_and_G, discretised on the Fourier grid (the same
conventions as the compressed estimator in ``oracle.bispec``):

  F_l^m(x; k_i) = sum_{q in b_i} e^{i q.x} y_l^{m*}(qhat) X(q)          shell field of bin i
  G_L^M(x)      = sum_{all q}    e^{i q.x} dn_L^M(q) / W(q)              full-range field
  dn_L^M(q)     = interlaced FFT of F(x) y_L^{M*}(xhat)                  (Sec. 3.1 interlacing)

  B_{l1 l2 L}(i, j) = H N / (I33 N_i N_j n^3)
                      sum_{m1 m2 M} (l1 l2 L; m1 m2 M) sum_x F_l1^m1(x; k_i) F_l2^m2(x; k_j) G_L^M(x)

with H = (l1 l2 L; 0 0 0) (Eq. sugi_base), N = (2 l1 + 1)(2 l2 + 1)(2 L + 1), y = sqrt(4 pi/(2l+1)) Y
(Racah normalisation), N_i the number of modes in bin i (the shell averages of Eq. F_and_G), X the
compensated interlaced FKP spectrum and xhat the line of sight (global: the fixed direction;
survey geometry: observer to the grid point).  ``sugiyama_fft`` evaluates every sub-configuration
(m1, m2, M) with m1 + m2 + M = 0, in the catalogue's own coordinate frame; no pairing of
sub-configurations and no rotation of the line of sight onto an axis is used.

Analytic shot noise (Sec. 5.4, global line of sight; ``analytic_shot_noise``), four terms:
  i = j = k:        delta_{l1 0} delta_{l2 0} delta_{L 0} S / I33
  i != j = k (k1):  delta_{l1 L} delta_{l2 0} (2L+1)/I33 H_L(k1)
  i = k != j (k2):  delta_{l2 L} delta_{l1 0} (2L+1)/I33 H_L(k2)
  i = j != k:       H N / I33 * sum_m w_m q_{l1 l2 L}(c_i, c_j, c_m) Q_L(k_m) / sum_m w_m
over the shells m of width dk centred at c_m = (m + 1/2) dk with c_m in [|c_i - c_j| + dk/2,
c_i + c_j - dk/2], w_m = N_mode(m)/c_m (the mode-count weighting of the compressed estimator's
analytic shot noise), H_L and Q_L the shell terms of ``oracle.shot`` (global line of sight: both
<L_L(mu) Re X N^*> - S <L_L(mu)>), and
  q_{l1 l2 L}(k1, k2, k3) = sum_n (-1)^n cL_l1^n(cos t13) cL_l2^{-n}(cos t23) (l1 l2 L; n -n 0)
(Lemma 1 and Eq. q_ells) with cos t13 = (k2^2 - k1^2 - k3^2)/(2 k1 k3) and cos t23 = (k1^2 - k2^2 -
k3^2)/(2 k2 k3) for k1 + k2 + k3 = 0.  Reading: cL_l^n are the Racah-normalised associated Legendre
functions, y_l^n at azimuth 0, sqrt((l-n)!/(l+n)!) L_l^n for n >= 0 and (-1)^n cL_l^{|n|} for n < 0
(with the unnormalised L_l^n the closed form misses the ring average whenever l1 != l2 and n != 0).
Pinned by tests/test_oracle_sugiyama.py: the closed form against a direct quadrature of the ring
average of sum_m (l1 l2 L; m -m 0) y_l1^{m*}(k1hat) y_l2^{-m*}(k2hat) around k3 (= q L_L(mu3)), and
the monopole B_000 shot noise against the compressed estimator's analytic B_000 shot noise.

FFT-method (exact) shot noise (Sec. 5.4.2; ``fft_method_shot_noise``): the three two-object terms
and the pure term written out over the (q1, q2) mode pairs.  Pinned by the identity it must
satisfy: for uncompensated fields of two point objects every closed triple draws two legs from one
object, so the raw estimator equals it (tests, with a tilted line of sight).

Pinned by tests/test_oracle_sugiyama.py: the explicit (q1, q2) enumeration of the same sum in
Fourier space (brute force, tiny meshes); the l l 0 multipoles against the Legendre form that the
addition theorem gives (no Y_lm or 3j involved); B_000 against the compressed estimator B_000
(Sec. 6: the two monopoles coincide); the half-sum over paired sub-configurations of the boxed
estimator (Eq. sym_sugi); invariance under a cyclic permutation of the axes applied to the
catalogue and the line of sight together; for a global line of sight along z, the reduction of
B_l0l to (2l+1)/(I33 N_i N_j n^3) sum_x F_l(x; k_i) F_0(x; k_j) G(x) with F_l the L_l(mu) shell; and,
with the line of sight to each grid point, the global-line-of-sight result for a distant observer.
"""
from __future__ import annotations

import numpy as np

from . import harmonics as H
from . import mesh as M
from . import power as P


def valid_multipole(l1, l2, L):
    """Triangle rule and even l1 + l2 + L (H_{l1 l2 L} != 0)."""
    return abs(l1 - l2) <= L <= l1 + l2 and (l1 + l2 + L) % 2 == 0


def _transform(spec, meshes, weight_fn):
    """Interlaced, compensated FFT of the meshes times a per-sample-point weight."""
    n = spec["n"]
    shifts = (0.0, 0.5) if len(meshes) == 2 else (0.0,)
    parts = [np.fft.fftn(mm * weight_fn(sh)) for mm, sh in zip(meshes, shifts)]
    s = parts[0] if len(parts) == 1 else 0.5 * (parts[0] + M.interlace_phase(n) * parts[1])
    return s / M.window(n, spec["assign"])


def spectra(spec, meshes, ells_L):
    """X(q) and dn_L^M(q)/W for every L requested (Eq. F_and_G)."""
    X0 = _transform(spec, meshes, lambda sh: 1.0)
    dn = {}
    for L in ells_L:
        for Mm in range(-L, L + 1):
            dn[(L, Mm)] = _transform(spec, meshes,
                                     lambda sh, L=L, Mm=Mm: np.conj(H.ylm_racah(L, Mm, P._xhat_dirs(spec, sh))))
    return X0, dn


def shell_fields_lm(spec, X0, kbins, ell, m):
    """F_l^m(x; k_b) for every bin b (complex, unnormalised sums over the modes of the bin)."""
    n = spec["n"]
    b, _ = M.bin_index(n, spec["box"], *kbins)
    w = np.conj(H.ylm_racah(ell, m, P._khat(spec))) * X0
    out = np.empty((kbins[2], n, n, n), dtype=np.complex128)
    for ib in range(kbins[2]):
        out[ib] = np.fft.ifftn(np.where(b == ib, w, 0.0)) * n**3
    return out


def mode_counts(spec, kbins):
    n = spec["n"]
    b, _ = M.bin_index(n, spec["box"], *kbins)
    _, cnt = M.bin_average(np.zeros((n, n, n)), b, kbins[2])
    return cnt


def _normalise(spec, raw, cnt, i33):
    ni, nj = cnt[:, None], cnt[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(ni * nj > 0, raw / (i33 * np.where(ni * nj > 0, ni * nj, 1.0)), 0.0)


def sugiyama_fft(spec, meshes, kbins, multipoles, i33):
    """B_{l1 l2 L}(i, j) for every ordered bin pair (k1 = bin i, k2 = bin j), per multipole.

    Returns {(l1, l2, L): complex array (nb, nb)}; the imaginary part is zero up to rounding."""
    X0, dn = spectra(spec, meshes, sorted({L for _, _, L in multipoles}))
    return sugiyama_from_spectra(spec, X0, dn, kbins, multipoles, i33)


def sugiyama_from_spectra(spec, X0, dn, kbins, multipoles, i33):
    """The estimator from X(q) and dn_L^M(q)/W (the keys (L, M) of ``dn``)."""
    n = spec["n"]
    G = {key: np.fft.ifftn(v) * n**3 for key, v in dn.items()}
    cnt = mode_counts(spec, kbins)
    shells = {}

    def shell(ell, m):
        if (ell, m) not in shells:
            shells[(ell, m)] = shell_fields_lm(spec, X0, kbins, ell, m)
        return shells[(ell, m)]

    out = {}
    for l1, l2, L in multipoles:
        hN = H.wigner3j(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)
        acc = np.zeros((kbins[2], kbins[2]), dtype=np.complex128)
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                Mm = -m1 - m2
                if abs(Mm) > L:
                    continue
                w = H.wigner3j(l1, l2, L, m1, m2, Mm)
                if w == 0.0:
                    continue
                f1g = shell(l1, m1) * G[(L, Mm)][None]
                acc += w * np.einsum("ixyz,jxyz->ij", f1g, shell(l2, m2)) / n**3
        out[(l1, l2, L)] = _normalise(spec, hN * acc, cnt, i33)
    return out


def sugiyama_halved(spec, meshes, kbins, multipoles, i33):
    """The boxed form of the estimator (Eq. sym_sugi): one sub-configuration of each pair
    {(m1, m2, M), (-m1, -m2, -M)} (M < 0, or M = 0 with m1 <= 0), weight eta = 2 except for
    (0, 0, 0), real part only."""
    n = spec["n"]
    Ls = sorted({L for _, _, L in multipoles})
    X0, dn = spectra(spec, meshes, Ls)
    G = {key: np.fft.ifftn(v) * n**3 for key, v in dn.items()}
    cnt = mode_counts(spec, kbins)
    out = {}
    for l1, l2, L in multipoles:
        hN = H.wigner3j(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)
        acc = np.zeros((kbins[2], kbins[2]))
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                Mm = -m1 - m2
                if abs(Mm) > L or Mm > 0 or (Mm == 0 and m1 > 0):
                    continue
                w = H.wigner3j(l1, l2, L, m1, m2, Mm)
                if w == 0.0:
                    continue
                eta = 1.0 if (m1, m2, Mm) == (0, 0, 0) else 2.0
                f1g = shell_fields_lm(spec, X0, kbins, l1, m1) * G[(L, Mm)][None]
                s = np.einsum("ixyz,jxyz->ij", f1g, shell_fields_lm(spec, X0, kbins, l2, m2)) / n**3
                acc += w * eta * np.real(s)
        out[(l1, l2, L)] = _normalise(spec, hN * acc, cnt, i33)
    return out


def sugiyama_brute(spec, meshes, kbins, multipole, i33, prs):
    """The same sum enumerated over explicit (q1, q2) mode pairs in Fourier space:
    H N / (I33 N_i N_j) sum_{m1 m2 M} 3j sum_{q1 in b_i, q2 in b_j} y_l1^{m1*}(q1) y_l2^{m2*}(q2)
    X(q1) X(q2) dn_L^M(q3)/W(q3), q3 = -q1 - q2 taken modulo the grid (tiny meshes only)."""
    l1, l2, L = multipole
    n = spec["n"]
    X0, dn = spectra(spec, meshes, [L])
    b, _ = M.bin_index(n, spec["box"], *kbins)
    ii = M.int_freqs(n)
    kf = 2.0 * np.pi / spec["box"]
    hN = H.wigner3j(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)
    out = []
    for i, j in prs:
        i1 = np.argwhere(b == i)
        i2 = np.argwhere(b == j)
        q1 = np.stack([ii[i1[:, 0]], ii[i1[:, 1]], ii[i1[:, 2]]], axis=1).astype(np.float64)
        q2 = np.stack([ii[i2[:, 0]], ii[i2[:, 1]], ii[i2[:, 2]]], axis=1).astype(np.float64)
        # grid index of -q1 - q2: a grid index is its frequency modulo n
        i3 = (-i1[:, None, :] - i2[None, :, :]) % n
        x1 = X0[i1[:, 0], i1[:, 1], i1[:, 2]]
        x2 = X0[i2[:, 0], i2[:, 1], i2[:, 2]]
        acc = 0.0 + 0.0j
        for m1 in range(-l1, l1 + 1):
            y1 = np.conj(H.ylm_racah(l1, m1, kf * q1)) * x1
            for m2 in range(-l2, l2 + 1):
                Mm = -m1 - m2
                if abs(Mm) > L:
                    continue
                w = H.wigner3j(l1, l2, L, m1, m2, Mm)
                if w == 0.0:
                    continue
                y2 = np.conj(H.ylm_racah(l2, m2, kf * q2)) * x2
                d3 = dn[(L, Mm)][i3[..., 0], i3[..., 1], i3[..., 2]]
                acc += w * np.sum(y1[:, None] * y2[None, :] * d3)
        ni, nj = len(i1), len(i2)
        out.append(hN * acc / (i33 * ni * nj) if ni * nj > 0 else 0.0)
    return np.array(out)


def legendre_ll0(spec, meshes, kbins, ell, i33, prs):
    """B_{l l 0} from the addition theorem: (2l+1)/(I33 N_i N_j) sum_{q1, q2} L_l(q1hat . q2hat)
    X(q1) X(q2) X(-q1 - q2) (no spherical harmonics or 3j symbols involved)."""
    n = spec["n"]
    X0 = _transform(spec, meshes, lambda sh: 1.0)
    b, _ = M.bin_index(n, spec["box"], *kbins)
    ii = M.int_freqs(n)
    out = []
    for i, j in prs:
        i1 = np.argwhere(b == i)
        i2 = np.argwhere(b == j)
        q1 = np.stack([ii[i1[:, 0]], ii[i1[:, 1]], ii[i1[:, 2]]], axis=1).astype(np.float64)
        q2 = np.stack([ii[i2[:, 0]], ii[i2[:, 1]], ii[i2[:, 2]]], axis=1).astype(np.float64)
        u1 = q1 / np.linalg.norm(q1, axis=1)[:, None]
        u2 = q2 / np.linalg.norm(q2, axis=1)[:, None]
        leg = H.legendre(ell, u1 @ u2.T)
        i3 = (-i1[:, None, :] - i2[None, :, :]) % n
        x3 = X0[i3[..., 0], i3[..., 1], i3[..., 2]]
        s = np.sum(leg * X0[i1[:, 0], i1[:, 1], i1[:, 2]][:, None] * X0[i2[:, 0], i2[:, 1], i2[:, 2]][None, :] * x3)
        ni, nj = len(i1), len(i2)
        out.append((2 * ell + 1) * s / (i33 * ni * nj) if ni * nj > 0 else 0.0)
    return np.array(out)


def racah_assoc_legendre(ell, n, x):
    """cL_l^n(x) = y_l^n at polar cosine x and azimuth 0 (Racah-normalised associated Legendre)."""
    from math import factorial, sqrt

    an = abs(n)
    v = sqrt(factorial(ell - an) / factorial(ell + an)) * H.assoc_legendre(ell, an, x)
    return v if n >= 0 else (-1.0) ** an * v


def q_ring(l1, l2, L, k1, k2, k3):
    """q_{l1 l2 L}(k1, k2, k3) of Lemma 1 (Eq. q_ells) for the triangle k1 + k2 + k3 = 0."""
    c13 = (k2 * k2 - k1 * k1 - k3 * k3) / (2.0 * k1 * k3)
    c23 = (k1 * k1 - k2 * k2 - k3 * k3) / (2.0 * k2 * k3)
    c13, c23 = min(1.0, max(-1.0, c13)), min(1.0, max(-1.0, c23))
    s = 0.0
    for n in range(-min(l1, l2), min(l1, l2) + 1):
        s += (-1.0) ** n * float(racah_assoc_legendre(l1, n, c13)) * float(racah_assoc_legendre(l2, -n, c23)) \
            * H.wigner3j(l1, l2, L, n, -n, 0)
    return s


def analytic_shot_noise(spec, X0, N0, kbins, multipoles, sc):
    """Sec. 5.4 analytic shot noise of every multipole on every (k_i, k_j) pair (global line of
    sight).  Returns {(l1, l2, L): (nb, nb)}."""
    from . import shot as SH

    kmin, dk, nb = kbins
    cen = np.array([kmin + (b + 0.5) * dk for b in range(nb)])
    qb = SH.qgrid(kbins)
    cq = np.array([(m + 0.5) * dk for m in range(qb[2])])
    i33, s3 = sc["I33"], sc["S3"]
    Ls = sorted({L for _, _, L in multipoles})
    Hk = {L: SH.shell_terms(spec, X0, N0, kbins, L, s3)[0] for L in Ls}
    Qs = {}
    for L in Ls:
        _, Qs[L], nq = SH.shell_terms(spec, X0, N0, qb, L, s3)
    out = {}
    for l1, l2, L in multipoles:
        hN = H.wigner3j(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)
        sn = np.zeros((nb, nb))
        for i in range(nb):
            for j in range(nb):
                v = 0.0
                if l1 == 0 and l2 == 0 and L == 0:
                    v += s3 / i33
                if l1 == L and l2 == 0:
                    v += (2 * L + 1) / i33 * Hk[L][i]
                if l2 == L and l1 == 0:
                    v += (2 * L + 1) / i33 * Hk[L][j]
                lo = abs(cen[i] - cen[j]) + 0.5 * dk
                hi = cen[i] + cen[j] - 0.5 * dk
                num = den = 0.0
                for m in range(qb[2]):
                    if lo - 1e-9 * dk <= cq[m] <= hi + 1e-9 * dk and nq[m] > 0:
                        w = nq[m] / cq[m]
                        num += w * q_ring(l1, l2, L, cen[i], cen[j], cq[m]) * Qs[L][m]
                        den += w
                if den > 0:
                    v += hN / i33 * num / den
                sn[i, j] = v
        out[(l1, l2, L)] = sn
    return out


def fft_method_shot_noise(spec, X0, N0, kbins, multipoles, i33, s3):
    """FFT-method (exact) shot noise (Sec. 5.4.2) of every multipole and bin pair, global line of
    sight n, by enumerating the (q1, q2) mode pairs (q3 = -q1 - q2 on the grid):
      H N / (I33 N_i N_j) Re sum_{m1 m2 M} (l1 l2 L; m1 m2 M) y_L^{M*}(n)
        sum_{q1 in b_i, q2 in b_j} y_l1^{m1*}(q1) y_l2^{m2*}(q2) [XN(q3) + XN(q2) + XN(q1) - 2 S]
    with XN = X N^*: legs 1, 2 from one object leave X N^* on q3, legs 1, 3 on q2, legs 2, 3 on q1;
    each of the three contains the three-of-one-object part S once, the pure term once more.
    Tiny meshes only.  Returns {(l1, l2, L): (nb, nb)}."""
    n = spec["n"]
    b, _ = M.bin_index(n, spec["box"], *kbins)
    ii = M.int_freqs(n)
    kf = 2.0 * np.pi / spec["box"]
    d = np.asarray(spec["los_dir"], dtype=np.float64)
    d = d / np.linalg.norm(d)
    xn = X0 * np.conj(N0)
    nb = kbins[2]
    idx = [np.argwhere(b == i) for i in range(nb)]
    qv = [np.stack([ii[t[:, 0]], ii[t[:, 1]], ii[t[:, 2]]], axis=1).astype(np.float64) for t in idx]
    out = {}
    for l1, l2, L in multipoles:
        hN = H.wigner3j(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)
        sn = np.zeros((nb, nb))
        for i in range(nb):
            for j in range(nb):
                if len(idx[i]) == 0 or len(idx[j]) == 0:
                    continue
                i1, i2 = idx[i], idx[j]
                i3 = (-i1[:, None, :] - i2[None, :, :]) % n
                t = (xn[i3[..., 0], i3[..., 1], i3[..., 2]] + xn[i2[:, 0], i2[:, 1], i2[:, 2]][None, :]
                     + xn[i1[:, 0], i1[:, 1], i1[:, 2]][:, None] - 2.0 * s3)
                acc = 0.0 + 0.0j
                for m1 in range(-l1, l1 + 1):
                    y1 = np.conj(H.ylm_racah(l1, m1, kf * qv[i]))
                    for m2 in range(-l2, l2 + 1):
                        Mm = -m1 - m2
                        if abs(Mm) > L:
                            continue
                        w = H.wigner3j(l1, l2, L, m1, m2, Mm)
                        if w == 0.0:
                            continue
                        y2 = np.conj(H.ylm_racah(l2, m2, kf * qv[j]))
                        yL = np.conj(H.ylm_racah(L, Mm, d))
                        acc += w * yL * np.sum(y1[:, None] * y2[None, :] * t)
                sn[i, j] = hN * np.real(acc) / (i33 * len(i1) * len(i2))
        out[(l1, l2, L)] = sn
    return out


def bispectrum_sugiyama(spec, data, randoms, kbins, multipoles, shot=False):
    """Full oracle measurement: {(l1, l2, L): real (nb, nb) array} (raw), the analytic shot noise
    when ``shot``, mode counts and scalars."""
    sc = P.catalog_scalars(data, randoms, spec["box"])
    meshes = P.fkp_meshes(spec, data, randoms, sc)
    res = sugiyama_fft(spec, meshes, kbins, multipoles, sc["I33"])
    out = dict(B={k: np.real(v) for k, v in res.items()},
               imag=max(float(np.max(np.abs(np.imag(v)))) for v in res.values()),
               counts=mode_counts(spec, kbins), scalars=sc)
    if shot:
        nmeshes = P.fkp_meshes(spec, data, randoms, sc, weight_power=2)
        X0, _ = spectra(spec, meshes, [])
        N0, _ = spectra(spec, nmeshes, [])
        if shot == "fft":
            out["shot"] = fft_method_shot_noise(spec, X0, N0, kbins, multipoles, sc["I33"], sc["S3"])
        else:
            out["shot"] = analytic_shot_noise(spec, X0, N0, kbins, multipoles, sc)
    return out
