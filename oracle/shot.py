"""Analytic bispectrum shot noise (oracle; test infrastructure only).  Global line of sight.

Notation: X_0 = compensated interlaced FKP spectrum; N_0(q) = compensated interlaced spectrum of
the w^2 N-field (Sec. 5.2, Eq. generic_noise definitions); F_l^w(q) = L_l(qhat . los) N_0(q);
S = three-point self term (sum_g w^3 - alpha^3 sum_r w^3).  Shell averages <.>_k are over the
modes of a k-bin.  Self-pair term S_l(k) = S <L_l(qhat . los)>_k (the C_shot/W^2 factor of Sec. 5.4
is taken as 1 for interlaced meshes; reading).

* H_l(k) = <Re X_0 F_l^{w*}>_k - S_l(k)            (Eq. H_ell)
* Q_l(k) = <Re X_l N_0^*>_k - S_l(k), X_l = L_l X_0  (Eq. Q_ell, by the addition theorem)

Scoccimarro, l on leg 1 (Sec. 5.4.1, built from Lemma 1's ring average Eq. I_l0l):
  N^(l)(i,j,k) = (2l+1)/I33 [ delta_l0 S + Q_l(k_i) + L_l(c12) H_l(k_j) + L_l(c13) H_l(k_k) ]
with the cosines between legs from bin centres, c12 = (c_k^2 - c_i^2 - c_j^2)/(2 c_i c_j),
c13 = (c_j^2 - c_i^2 - c_k^2)/(2 c_i c_k) (reading: the paper does not say which k is used).

Compressed B_l0l (Sec. 5.4.3, boxed result), t = c_i/c_j:
  N(i,j) = (2l+1)/I33 [ delta_l0 S + (-1)^l g_l(t) H_l(k_i) + (-1)^l g_l(1/t) H_l(k_j)
                        + sum_m w_m Q_l(k_m) / sum_m w_m ]
over shells m of width dk centred at (m+1/2) dk with centre in [|c_i - c_j| + dk/2, c_i + c_j - dk/2]
and weight w_m = N_mode(m)/c_m.  Readings: the printed i=j=k term omits the 1/I that the Sugiyama
form carries (kept here); the printed i=j!=k term divides a mode-averaged Q by sum N_mode/k3,
which is not dimensionally consistent, so the mode count is applied to the averaged Q as the
V_ring V_dot ~ 1/k3 derivation of Sec. 5.4.2 requires.

These are thin-shell approximations (Sec. 5.3), so no exact identity pins them.  The tests check
them statistically against Poisson catalogues (the subtracted monopole averages to zero and the raw
monopole averages to the full shot noise), check the g_l factors separately, and compare them with
the exact FFT-method sums below on the same catalogue (a few per cent of the monopole shot-noise
scale, the thin-shell error the paper reports).

FFT method (Sec. 5.4.2, the exact reference the paper evaluates with extra inverse transforms
instead of the thin-shell integrals), Scoccimarro B_l with l on leg 1 and a global line of sight.
Over the closed triplets q1 in b_i, q2 in b_j, q3 in b_k, q1 + q2 + q3 = 0:
  T23 = sum L_l(mu1) X_0(q1) N_0^*(q1)     (legs 2, 3 from one object)
  T12 = sum L_l(mu1) X_0(q3) N_0^*(q3)     (legs 1, 2 from one object)
  T13 = sum L_l(mu1) X_0(q2) N_0^*(q2)     (legs 1, 3 from one object)
  N_T^(l) = sum L_l(mu1)
  N^(l)_fft(i,j,k) = (2l+1)/(I33 N_T) Re[T23 + T12 + T13 - 2 S N_T^(l)]
Each two-object term contains the three-of-one-object part S N_T^(l) once; the pure term adds it
back once, hence the -2.  ``fft_method_shot_noise`` enumerates the triplets (the definition written
out; tiny meshes).  Pinned by the exact identity it must satisfy: for uncompensated fields of at
most two objects every closed triplet draws two legs from one object, so the raw estimator equals
N_fft; with three objects the difference is the sum over distinct triples (tests).

The same construction for the compressed B_l0l (l on the k3 leg, q3 = -q1 - q2 over all modes):
  Ta = sum L_l(mu3) X_0(q3) N_0^*(q3),  Tb = sum L_l(mu3) X_0(q2) N_0^*(q2),
  Tc = sum L_l(mu3) X_0(q1) N_0^*(q1),  Td = sum L_l(mu3)      over q1 in b_i, q2 in b_j,
  N_fft(i,j) = (2l+1)/(I33 N_i N_j) Re[Ta + Tb + Tc - 2 S Td]
(``compressed_fft_method_shot``), pinned by the same two- and three-object identities.
"""
from __future__ import annotations

import numpy as np

from . import harmonics as H
from . import mesh as M


def _mu(spec):
    (kx, ky, kz), _ = M.kvectors(spec["n"], spec["box"])
    d = np.asarray(spec["los_dir"], dtype=np.float64)
    d = d / np.linalg.norm(d)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(kk > 0, (kx * d[0] + ky * d[1] + kz * d[2]) / np.where(kk > 0, kk, 1.0), 0.0)


def shell_terms(spec, X0, N0, kbins, ell, s3, survey=None):
    """(H_l, Q_l, N_mode) on the given bins.

    Global line of sight: X_l = L_l(mu) X_0 and F_l^w = L_l(mu) N_0, so H_l = Q_l with the self term
    S <L_l(mu)>.  Survey geometry (``survey`` = dict(Xl, Nl, moments)): Q_l = <Re X_l N_0^*> - S_l,
    H_l = <Re X_0 N_l^*> - S_l with X_l, N_l the Yamamoto fields of the FKP and N-fields, and the
    self term S_l(k) = sum_p c_p <L_l(qhat . xhat_p)>_k = 4 pi/(2l+1) sum_m <Y_lm(qhat)>_k C_lm^*,
    C_lm = sum_p c_p Y_lm(xhat_p), c_p = w^3 (data), -alpha^3 w^3 (randoms), xhat_p the direction of
    object p from the observer (reading: the objects' own directions)."""
    b, _ = M.bin_index(spec["n"], spec["box"], *kbins)
    nb = kbins[2]
    if survey is None:
        lmu = H.legendre(ell, _mu(spec))
        cross, cnt = M.bin_average(lmu * np.real(X0 * np.conj(N0)), b, nb)
        lavg, _ = M.bin_average(lmu, b, nb)
        hval = cross - s3 * lavg
        return hval, hval.copy(), cnt
    (kx, ky, kz), _ = M.kvectors(spec["n"], spec["box"])
    kh = np.stack(np.broadcast_arrays(kx, ky, kz), axis=-1)
    self_t = np.zeros(nb)
    for m in range(-ell, ell + 1):
        y = H.ylm(ell, m, kh)
        yr, _ = M.bin_average(np.real(y), b, nb)
        yi, _ = M.bin_average(np.imag(y), b, nb)
        cm = survey["moments"][m]
        self_t += 4.0 * np.pi / (2 * ell + 1) * np.real((yr + 1j * yi) * np.conj(cm))
    q, cnt = M.bin_average(np.real(survey["Xl"] * np.conj(N0)), b, nb)
    h, _ = M.bin_average(np.real(X0 * np.conj(survey["Nl"])), b, nb)
    return h - self_t, q - self_t, cnt


def ylm_moments(spec, data, randoms, alpha, ell):
    """C_lm = sum_g w^3 Y_lm(xhat_g) - alpha^3 sum_r w^3 Y_lm(xhat_r) for m = -l .. l, xhat the
    direction from the observer."""
    obs = np.asarray(spec.get("observer", (0.0, 0.0, 0.0)), dtype=np.float64)
    out = {}
    for m in range(-ell, ell + 1):
        v = np.sum(np.asarray(data.w, np.float64) ** 3 * H.ylm(ell, m, np.asarray(data.pos, np.float64) - obs))
        if randoms is not None:
            v -= alpha ** 3 * np.sum(np.asarray(randoms.w, np.float64) ** 3
                                     * H.ylm(ell, m, np.asarray(randoms.pos, np.float64) - obs))
        out[m] = v
    return out


def qgrid(kbins):
    """Shells [m dk, (m+1) dk) covering 0 .. 2 k_max for the compressed i=j!=k term."""
    kmin, dk, nb = kbins
    kmax = kmin + nb * dk
    nq = int(np.ceil(2.0 * kmax / dk)) + 1
    return (0.0, dk, nq)


def analytic_shot_noise(spec, X0, N0, kbins, tri, prs, sc, scoc_ells, tripo_ells, survey=None):
    """survey: None (global line of sight) or dict ell -> dict(Xl, Nl, moments) (see shell_terms)."""
    kmin, dk, nb = kbins
    c = np.array([kmin + (b + 0.5) * dk for b in range(nb)])
    i33, s3 = sc["I33"], sc["S3"]
    qb = qgrid(kbins)
    cq = np.array([(m + 0.5) * dk for m in range(qb[2])])
    shot_B, shot_BB, parts = {}, {}, {}
    for ell in sorted(set(scoc_ells) | set(tripo_ells)):
        sv = None if survey is None else survey[ell]
        hl, ql, _ = shell_terms(spec, X0, N0, kbins, ell, s3, sv)
        hq, qq, nq = shell_terms(spec, X0, N0, qb, ell, s3, sv)
        parts[ell] = dict(H=hl, Q=ql, Qq=qq, Nq=nq)
        if ell in scoc_ells:
            out = np.empty(len(tri))
            for t, (i, j, k) in enumerate(tri):
                c12 = (c[k] ** 2 - c[i] ** 2 - c[j] ** 2) / (2.0 * c[i] * c[j])
                c13 = (c[j] ** 2 - c[i] ** 2 - c[k] ** 2) / (2.0 * c[i] * c[k])
                v = (s3 if ell == 0 else 0.0) + ql[i]
                v += float(H.legendre(ell, c12)) * hl[j] + float(H.legendre(ell, c13)) * hl[k]
                out[t] = (2 * ell + 1) / i33 * v
            shot_B[ell] = out
        if ell in tripo_ells:
            out = np.empty(len(prs))
            sgn = (-1.0) ** ell
            for t, (i, j) in enumerate(prs):
                v = (s3 if ell == 0 else 0.0)
                v += sgn * H.g_ell(ell, c[i] / c[j]) * hl[i]
                v += sgn * H.g_ell(ell, c[j] / c[i]) * hl[j]
                lo = abs(c[i] - c[j]) + 0.5 * dk
                hi = c[i] + c[j] - 0.5 * dk
                sel = (cq >= lo - 1e-9 * dk) & (cq <= hi + 1e-9 * dk) & (nq > 0)
                wts = nq[sel] / cq[sel]
                v += np.sum(wts * qq[sel]) / np.sum(wts) if wts.size else 0.0
                out[t] = (2 * ell + 1) / i33 * v
            shot_BB[ell] = out
    return shot_B, shot_BB, parts


def triplet_shot_terms(spec, X0, N0, kbins, tri, ell):
    """Per triangle (i, j, k): explicit sums over the closed triplets of the FFT-method terms.

    Returns dict of arrays nt (triplet count), ntl (sum of L_l(mu1)), t23, t12, t13 (complex)."""
    from .bispec import _mode_lists

    n = spec["n"]
    kf = 2.0 * np.pi / spec["box"]
    d = np.asarray(spec["los_dir"], dtype=np.float64)
    d = d / np.linalg.norm(d)
    b, lists = _mode_lists(spec, kbins)
    out = {k: [] for k in ("nt", "ntl", "t23", "t12", "t13")}
    for i, j, k in tri:
        q1 = lists[i]
        q2 = lists[j]
        q3 = -(q1[:, None, :] + q2[None, :, :])
        idx3 = q3 % n
        inb = b[idx3[..., 0], idx3[..., 1], idx3[..., 2]] == k
        inb &= np.all(np.abs(q3) < n // 2, axis=-1)
        i1 = q1 % n
        i2 = q2 % n
        kk1 = np.sqrt(np.sum((kf * q1) ** 2, axis=1))
        mu1 = (kf * q1) @ d / kk1
        l1 = H.legendre(ell, mu1)[:, None] * np.ones(q3.shape[:2])
        xn1 = (X0 * np.conj(N0))[i1[:, 0], i1[:, 1], i1[:, 2]][:, None]
        xn2 = (X0 * np.conj(N0))[i2[:, 0], i2[:, 1], i2[:, 2]][None, :]
        xn3 = (X0 * np.conj(N0))[idx3[..., 0], idx3[..., 1], idx3[..., 2]]
        out["nt"].append(int(np.sum(inb)))
        out["ntl"].append(np.sum(np.where(inb, l1, 0.0)))
        out["t23"].append(np.sum(np.where(inb, l1 * xn1, 0.0)))
        out["t12"].append(np.sum(np.where(inb, l1 * xn3, 0.0)))
        out["t13"].append(np.sum(np.where(inb, l1 * xn2, 0.0)))
    return {k: np.array(v) for k, v in out.items()}


def fft_method_shot_noise(spec, X0, N0, kbins, tri, i33, s3, ells):
    """N^(l)_fft for every triangle and each l in ells (global line of sight)."""
    res = {}
    for ell in ells:
        t = triplet_shot_terms(spec, X0, N0, kbins, tri, ell)
        tot = np.real(t["t23"] + t["t12"] + t["t13"]) - 2.0 * s3 * t["ntl"]
        with np.errstate(invalid="ignore", divide="ignore"):
            res[ell] = np.where(t["nt"] > 0, (2 * ell + 1) * tot / (i33 * np.where(t["nt"] > 0, t["nt"], 1)), 0.0)
    return res


def compressed_fft_method_shot(spec, X0, N0, kbins, prs, i33, s3, ells):
    """N_fft(i, j) of the compressed B_l0l for every pair and each l in ells, by enumerating the
    (q1, q2) pairs with q3 = -q1 - q2 taken on the grid as the estimator does."""
    from .bispec import _mode_lists

    n = spec["n"]
    b, lists = _mode_lists(spec, kbins)
    cnt = np.array([len(x) for x in lists], dtype=np.float64)
    xn = X0 * np.conj(N0)
    res = {}
    for ell in ells:
        lmu = H.legendre(ell, _mu(spec))
        out = []
        for i, j in prs:
            q1, q2 = lists[i], lists[j]
            q3 = (-(q1[:, None, :] + q2[None, :, :])) % n
            i1, i2 = q1 % n, q2 % n
            l3 = lmu[q3[..., 0], q3[..., 1], q3[..., 2]]
            ta = np.sum(l3 * xn[q3[..., 0], q3[..., 1], q3[..., 2]])
            tb = np.sum(l3 * xn[i2[:, 0], i2[:, 1], i2[:, 2]][None, :])
            tc = np.sum(l3 * xn[i1[:, 0], i1[:, 1], i1[:, 2]][:, None])
            td = np.sum(l3)
            den = i33 * cnt[i] * cnt[j]
            out.append((2 * ell + 1) * np.real(ta + tb + tc - 2.0 * s3 * td) / den if den > 0 else 0.0)
        res[ell] = np.array(out)
    return res
