"""Bispectrum multipoles (oracle; test infrastructure only).

Scoccimarro estimator (Eq. bi_sco), discretised on the Fourier grid:
  B_l(i,j,k) = (2l+1)/I33 * (1/N_T) sum_{q1 in b_i, q2 in b_j, q3 in b_k, q1+q2+q3=0}
               X_l(q1) X_0(q2) X_0(q3)
with X = compensated, interlaced FKP spectra, X_l the Yamamoto field F_l/W (line of sight on the
first leg, which is the smallest side k1 for k1 <= k2 <= k3) and N_T the number of closed
triplets.  The closure sum is computed two ways: by plane-wave expansion of the Kronecker delta
(shell-filtered inverse transforms F_b(x) = sum_{q in b} X(q) e^{i q.x}, then sum_x F_i F_j F_k,
Sec. 2.2) and by explicit enumeration of (q1, q2) pairs (brute force, tiny meshes only).

Triangles: bins i <= j <= k whose centres close, c_k <= c_i + c_j (the paper says "all closed
triangles" without fixing the rule; the bin-centre rule is the reading used here).  The number of
closed triplets N_T is reported for every triangle.

Compressed TripoSH estimator B_l0l (Eq. new_bispec) for l2 = 0, L = l.  With H_{l0l} =
(-1)^l/sqrt(2l+1), (l 0 l; m 0 -m) = (-1)^{l-m}/sqrt(2l+1), N_{l0l} = (2l+1)^2 and the Racah
relation y_l^{-m*} = (-1)^m y_l^m, the m-sum collapses by the addition theorem (Eq. add_theorem):
  B_l0l(i,j) = (2l+1)/(I33 N_i N_j) sum_{q1 in b_i, q2 in b_j} X_0(q1) X_0(q2) X_l(-q1-q2)
where X_l carries its line of sight at the k3 endpoint.  ``compressed_explicit`` evaluates the
definition with the explicit (m1, M) sum and Wigner 3j symbols instead; the two are compared in
the tests (this pins the collapse).  In real space the collapsed form is
(2l+1)/(I33 N_i N_j n^3) sum_x F_i(x) F_j(x) G^(l)(x), G^(l)(x) = sum_{all q} X_l(q) e^{i q.x}.

Pinned by tests/test_oracle_bispec.py: the real-space closure sum against the explicit enumeration
of closed (q1, q2, q3) triplets and the compressed form against the (q1, q2) pair enumeration (brute
force, tiny meshes); the collapse against the explicit-3j definition; the compression identity (the
Scoccimarro estimator summed along k3 gives N_i N_j B_l0l); the triangle count for 19 bins (805) and
N_T against the thin-shell volume 8 pi^2 c1 c2 c3 dk^3 / k_f^6 (Sec. 5.2); the survey l = 2 forms
against the global line of sight for a distant observer.  ``odd_multipoles`` and
``cross_bispectrum`` state their own pins.
"""
from __future__ import annotations

import itertools
from math import pi

import numpy as np

from . import harmonics as H
from . import mesh as M


def bin_centres(kbins):
    kmin, dk, nb = kbins
    return np.array([kmin + (b + 0.5) * dk for b in range(nb)])


def triangles(kbins):
    """Closed triangles (i <= j <= k) by the bin-centre rule c_k <= c_i + c_j."""
    kmin, dk, nb = kbins
    c = [kmin + (b + 0.5) * dk for b in range(nb)]
    out = []
    for i in range(nb):
        for j in range(i, nb):
            for k in range(j, nb):
                if c[k] <= c[i] + c[j] + 1e-9 * dk:
                    out.append((i, j, k))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def pairs(kbins):
    nb = kbins[2]
    return np.array([(i, j) for i in range(nb) for j in range(i, nb)], dtype=np.int64).reshape(-1, 2)


def shell_fields(spec, X, kbins, ones=False):
    """F_b(x) = sum_{q in b} X(q) e^{i q.x} for every bin (real because X is Hermitian)."""
    kmin, dk, nb = kbins
    n = spec["n"]
    b, _ = M.bin_index(n, spec["box"], kmin, dk, nb)
    out = np.empty((nb, n, n, n))
    for ib in range(nb):
        mask = (b == ib)
        src = mask.astype(np.float64) if ones else np.where(mask, X, 0.0)
        out[ib] = np.real(np.fft.ifftn(src)) * n**3
    return out


def los_field(spec, X0, ell):
    """X_l(q) = L_l(qhat . los) X_0(q) for a global line of sight."""
    (kx, ky, kz), _ = M.kvectors(spec["n"], spec["box"])
    d = np.asarray(spec["los_dir"], dtype=np.float64)
    d = d / np.linalg.norm(d)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(kk > 0, (kx * d[0] + ky * d[1] + kz * d[2]) / np.where(kk > 0, kk, 1.0), 0.0)
    return H.legendre(ell, mu) * X0


def scoccimarro_fft(spec, X0, Xl, kbins, tri, i33, ells):
    """B_l for the listed triangles by shell-filtered inverse transforms.

    Xl: dict l -> X_l (line of sight on leg 1).  Returns (B dict, N_T, raw sums dict)."""
    n = spec["n"]
    f0 = shell_fields(spec, X0, kbins)
    ind = shell_fields(spec, None, kbins, ones=True)
    nt = np.array([np.sum(ind[i] * ind[j] * ind[k]) for i, j, k in tri]) / n**3
    B, raw = {}, {}
    for ell in ells:
        fl = f0 if ell == 0 else shell_fields(spec, Xl[ell], kbins)
        s = np.array([np.sum(fl[i] * f0[j] * f0[k]) for i, j, k in tri]) / n**3
        raw[ell] = s
        with np.errstate(invalid="ignore", divide="ignore"):
            B[ell] = np.where(nt > 0, (2 * ell + 1) * s / (i33 * np.where(nt > 0, nt, 1.0)), 0.0)
    return B, nt, raw


def _mode_lists(spec, kbins):
    kmin, dk, nb = kbins
    n = spec["n"]
    b, _ = M.bin_index(n, spec["box"], kmin, dk, nb)
    ii = M.int_freqs(n)
    lists = []
    for ib in range(nb):
        idx = np.argwhere(b == ib)
        lists.append(np.stack([ii[idx[:, 0]], ii[idx[:, 1]], ii[idx[:, 2]]], axis=1))
    return b, lists


def scoccimarro_brute(spec, X0, Xl_leg1, kbins, tri):
    """sum over explicit closed triplets of X_l(q1) X_0(q2) X_0(q3), and the triplet count."""
    n = spec["n"]
    b, lists = _mode_lists(spec, kbins)
    sums, counts = [], []
    for i, j, k in tri:
        q1 = lists[i]
        q2 = lists[j]
        q3 = -(q1[:, None, :] + q2[None, :, :])
        idx3 = q3 % n
        inb = b[idx3[..., 0], idx3[..., 1], idx3[..., 2]] == k
        # no aliasing: each component of q3 must stay inside (-n/2, n/2)
        inb &= np.all(np.abs(q3) < n // 2, axis=-1)
        i1 = q1 % n
        i2 = q2 % n
        v1 = Xl_leg1[i1[:, 0], i1[:, 1], i1[:, 2]]
        v2 = X0[i2[:, 0], i2[:, 1], i2[:, 2]]
        v3 = X0[idx3[..., 0], idx3[..., 1], idx3[..., 2]]
        prod = v1[:, None] * v2[None, :] * v3
        sums.append(np.sum(np.where(inb, prod, 0.0)))
        counts.append(int(np.sum(inb)))
    return np.array(sums), np.array(counts)


def compressed_fft(spec, X0, Xl_k3, kbins, prs, i33, ell):
    """B_l0l for the listed (i <= j) pairs via sum_x F_i F_j G^(l)."""
    n = spec["n"]
    f0 = shell_fields(spec, X0, kbins)
    g = np.real(np.fft.ifftn(Xl_k3)) * n**3
    _, cnt = M.bin_average(np.zeros((n, n, n)), M.bin_index(n, spec["box"], *kbins)[0], kbins[2])
    s = np.array([np.sum(f0[i] * f0[j] * g) for i, j in prs]) / n**3
    ni = cnt[prs[:, 0]]
    nj = cnt[prs[:, 1]]
    with np.errstate(invalid="ignore", divide="ignore"):
        val = np.where(ni * nj > 0, (2 * ell + 1) * s / (i33 * ni * nj), 0.0)
    return val, s, cnt


def compressed_explicit(spec, meshes, kbins, prs, i33, ell):
    """B_l0l from the definition (Eq. new_bispec) with the explicit (m1, M) sum:
    (H N / I) sum_{m1, M} (l 0 l; m1 0 M) <y_l^{m1*}(q3hat) X_0(q1) X_0(q2) dn_l^M(q3)/W(q3)>,
    dn_l^M(q) = sum_x F(x) y_l^{M*}(xhat) e^{-i q.x}, q3 = -q1-q2; brute force over (q1, q2)."""
    from .power import _xhat_dirs  # noqa: WPS433 (oracle-internal helper)

    n = spec["n"]
    shifts = (0.0, 0.5) if len(meshes) == 2 else (0.0,)
    win = M.window(n, spec["assign"])

    def transform(weight_fn):
        parts = [np.fft.fftn(mm * weight_fn(sh)) for mm, sh in zip(meshes, shifts)]
        s = parts[0] if len(parts) == 1 else 0.5 * (parts[0] + M.interlace_phase(n) * parts[1])
        return s / win

    X0 = transform(lambda sh: 1.0)
    dnlm = {mm: transform(lambda sh, mm=mm: np.conj(H.ylm_racah(ell, mm, _xhat_dirs(spec, sh))))
            for mm in range(-ell, ell + 1)}
    hnorm = H.wigner3j(ell, 0, ell, 0, 0, 0) * (2 * ell + 1) ** 2
    b, lists = _mode_lists(spec, kbins)
    ii = M.int_freqs(n)
    kf = 2.0 * pi / spec["box"]
    out = []
    for i, j in prs:
        q1, q2 = lists[i], lists[j]
        q3 = -(q1[:, None, :] + q2[None, :, :])
        idx3 = q3 % n
        i1, i2 = q1 % n, q2 % n
        x1 = X0[i1[:, 0], i1[:, 1], i1[:, 2]]
        x2 = X0[i2[:, 0], i2[:, 1], i2[:, 2]]
        acc = np.zeros(q3.shape[:2], dtype=np.complex128)
        for m1 in range(-ell, ell + 1):
            w3 = H.wigner3j(ell, 0, ell, m1, 0, -m1)
            if w3 == 0.0:
                continue
            y = np.conj(H.ylm_racah(ell, m1, kf * q3.astype(np.float64)))
            d = dnlm[-m1][idx3[..., 0], idx3[..., 1], idx3[..., 2]]
            acc += w3 * y * d
        tot = np.sum(x1[:, None] * x2[None, :] * acc)
        out.append(hnorm * tot / (i33 * len(q1) * len(q2)))
    del ii
    return np.array(out)


def bispectrum(spec, data, randoms, kbins, scoc_ells=(0, 2), tripo_ells=(0, 2), shot=True):
    """Full oracle measurement: B_l, N_T, compressed B_l0l, shot noise (analytic; shot="fft" adds
    the FFT-method shot noise as ``shot_B_fft`` / ``shot_BB_fft``, global line of sight only).
    spec["los"] = "global": X_l = L_l(qhat . los) X_0; otherwise (survey geometry, line of sight to
    each grid point from spec["observer"]) X_l is the Yamamoto field F_l of Eq. hand."""
    from . import power as P
    from . import shot as S

    sc = P.catalog_scalars(data, randoms, spec["box"])
    meshes = P.fkp_meshes(spec, data, randoms, sc)
    ells = sorted(set(scoc_ells) | set(tripo_ells) | {0})
    endpoint = spec.get("los", "endpoint") != "global"
    if endpoint:
        # survey geometry with the line of sight to each grid point: X_l is the Yamamoto field
        fields, _ = P.fields_plain(spec, meshes, ells)
        X0 = fields[0]
        Xl = {ell: fields[ell] for ell in ells}
    else:
        fields, _ = P.fields_plain(spec, meshes, [0])
        X0 = fields[0]
        Xl = {ell: los_field(spec, X0, ell) for ell in ells}
    tri = triangles(kbins)
    prs = pairs(kbins)
    B, nt, raw = scoccimarro_fft(spec, X0, Xl, kbins, tri, sc["I33"], scoc_ells)
    BB = {}
    for ell in tripo_ells:
        BB[ell], _, cnt = compressed_fft(spec, X0, Xl[ell], kbins, prs, sc["I33"], ell)
    res = dict(tri=tri, pairs=prs, B=B, NT=nt, BB=BB, raw=raw, scalars=sc)
    if shot:
        nmeshes = P.fkp_meshes(spec, data, randoms, sc, weight_power=2)
        nf, _ = P.fields_plain(spec, nmeshes, ells if endpoint else [0])
        survey = None
        if endpoint:
            survey = {ell: dict(Xl=Xl[ell], Nl=nf[ell], moments=S.ylm_moments(spec, data, randoms, sc["alpha"], ell))
                      for ell in ells}
        res["shot_B"], res["shot_BB"], res["shot_parts"] = S.analytic_shot_noise(
            spec, X0, nf[0], kbins, tri, prs, sc, scoc_ells, tripo_ells, survey)
        if shot == "fft":
            res["shot_B_fft"] = S.fft_method_shot_noise(spec, X0, nf[0], kbins, tri, sc["I33"], sc["S3"],
                                                        scoc_ells)
            res["shot_BB_fft"] = S.compressed_fft_method_shot(spec, X0, nf[0], kbins, prs, sc["I33"], sc["S3"],
                                                              tripo_ells)
    return res


def odd_multipoles(spec, data, randoms, kbins, ells=(1, 3)):
    """Odd Scoccimarro multipoles B_1, B_3 (raw), l on leg 1: X_l is anti-Hermitian for odd l, so its
    shell fields are imaginary, i A_b(x), and the closure sum is i sum_x A_i F_j F_k; B_l reports the
    imaginary part, (2l+1)/(I33 N_T) sum_x A_i F_j F_k / n^3 (reading, as for the odd P_l of Sec. 2.1).
    X_l is the Yamamoto field F_l of Eq. hand (line of sight to each grid point) in survey geometry,
    L_l(qhat . los) X_0 with a global line of sight.  Pinned by: the enumeration of the closed
    triples (global line of sight, tiny mesh) and the global-line-of-sight limit of a distant
    observer (tests)."""
    from . import power as P

    sc = P.catalog_scalars(data, randoms, spec["box"])
    meshes = P.fkp_meshes(spec, data, randoms, sc)
    endpoint = spec.get("los", "endpoint") != "global"
    if endpoint:
        fields, _ = P.fields_plain(spec, meshes, sorted(set(ells) | {0}))
        X0, Xl = fields[0], {ell: fields[ell] for ell in ells}
    else:
        X0 = P.fields_plain(spec, meshes, [0])[0][0]
        Xl = {ell: los_field(spec, X0, ell) for ell in ells}
    n = spec["n"]
    b, _ = M.bin_index(n, spec["box"], *kbins)
    tri = triangles(kbins)
    f0 = shell_fields(spec, X0, kbins)
    ind = shell_fields(spec, None, kbins, ones=True)
    nt = np.array([np.sum(ind[i] * ind[j] * ind[k]) for i, j, k in tri]) / n**3
    out = {}
    for ell in ells:
        a = np.empty((kbins[2], n, n, n))
        for ib in range(kbins[2]):
            a[ib] = np.imag(np.fft.ifftn(np.where(b == ib, Xl[ell], 0.0))) * n**3
        s = np.array([np.sum(a[i] * f0[j] * f0[k]) for i, j, k in tri]) / n**3
        with np.errstate(invalid="ignore", divide="ignore"):
            out[ell] = np.where(nt > 0, (2 * ell + 1) * s / (sc["I33"] * np.where(nt > 0, nt, 1.0)), 0.0)
    return dict(tri=tri, B=out, NT=nt, X0=X0, Xl=Xl, I33=sc["I33"])


def cross_bispectrum(spec, tracers, kbins, scoc_ells=(0, 2), tripo_ells=(0,)):
    """Multi-tracer bispectra, global line of sight, raw estimates: tracer t_1 on leg 1 (k1, which
    carries the line of sight of B_l), t_2 on leg 2, t_3 on leg 3, ``tracers`` = three (data,
    randoms) pairs (randoms None for a periodic box).
      B_l^{123}(i,j,k)  = (2l+1)/(I33^{123} N_T) sum_closed L_l(mu1) X^1(q1) X^2(q2) X^3(q3)
      B_l0l^{123}(i,j)  = (2l+1)/(I33^{123} N_i N_j) sum_{q1 in b_i, q2 in b_j} X^1(q1) X^2(q2)
                          L_l(mu3) X^3(q3),  q3 = -q1 - q2
    Readings (the paper's toolkit lists auto and cross bispectra without printing the cross form):
    I33^{123} = (I33^1 I33^2 I33^3)^(1/3), exact when the three selections n w have the same shape;
    no shot noise is subtracted (pairs of legs on the same tracer would carry one).  Pinned by:
    three equal tracers give the auto estimator; a copy of tracer A translated by whole cells on
    leg 3 multiplies each closed triple by the phase exp(-i q3.d) (explicit enumeration, tests)."""
    from . import power as P

    fields, i33 = [], 1.0
    for data, rnd in tracers:
        sc = P.catalog_scalars(data, rnd, spec["box"])
        meshes = P.fkp_meshes(spec, data, rnd, sc)
        fields.append(P.fields_plain(spec, meshes, [0])[0][0])
        i33 *= sc["I33"]
    i33 = i33 ** (1.0 / 3.0)
    n = spec["n"]
    tri = triangles(kbins)
    prs = pairs(kbins)
    ind = shell_fields(spec, None, kbins, ones=True)
    nt = np.array([np.sum(ind[i] * ind[j] * ind[k]) for i, j, k in tri]) / n**3
    f2 = shell_fields(spec, fields[1], kbins)
    f3 = shell_fields(spec, fields[2], kbins)
    B = {}
    for ell in scoc_ells:
        f1 = shell_fields(spec, los_field(spec, fields[0], ell), kbins)
        s = np.array([np.sum(f1[i] * f2[j] * f3[k]) for i, j, k in tri]) / n**3
        with np.errstate(invalid="ignore", divide="ignore"):
            B[ell] = np.where(nt > 0, (2 * ell + 1) * s / (i33 * np.where(nt > 0, nt, 1.0)), 0.0)
    f1 = shell_fields(spec, fields[0], kbins)
    _, cnt = M.bin_average(np.zeros((n, n, n)), M.bin_index(n, spec["box"], *kbins)[0], kbins[2])
    BB = {}
    for ell in tripo_ells:
        g = np.real(np.fft.ifftn(los_field(spec, fields[2], ell))) * n**3
        s = np.array([np.sum(f1[i] * f2[j] * g) for i, j in prs]) / n**3
        ni, nj = cnt[prs[:, 0]], cnt[prs[:, 1]]
        with np.errstate(invalid="ignore", divide="ignore"):
            BB[ell] = np.where(ni * nj > 0, (2 * ell + 1) * s / (i33 * ni * nj), 0.0)
    return dict(tri=tri, pairs=prs, B=B, BB=BB, NT=nt, I33=i33, fields=fields)


def all_pairs_product(nb):
    return list(itertools.product(range(nb), range(nb)))
