"""Pins for oracle.bispec / oracle.shot."""
from math import pi
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import bispec as B
from oracle import mesh as M
from oracle import power as P
from synthetic import make_periodic_catalog, make_survey_catalogs


def _periodic_spec(n, box, assign=3, interlace=1):
    return dict(n=n, box=box, origin=(0.0, 0.0, 0.0), assign=assign, interlace=interlace,
                los="global", los_dir=(0.0, 0.0, 1.0), periodic=1)


@pytest.fixture(scope="module")
def tiny_periodic():
    cat = make_periodic_catalog(4000, 300.0, 16, seed=11)
    spec = _periodic_spec(24, 300.0)
    sc = P.catalog_scalars(cat, None, 300.0)
    meshes = P.fkp_meshes(spec, cat, None, sc)
    fields, _ = P.fields_plain(spec, meshes, [0])
    return spec, cat, sc, fields[0]


def test_triangle_count_for_19_bins():
    """19 bins of 0.01 from 0.01 with the centre closure rule give 805 of 1330 ordered triples."""
    tri = B.triangles((0.01, 0.01, 19))
    assert len(tri) == 805
    assert np.all(tri[:, 0] <= tri[:, 1]) and np.all(tri[:, 1] <= tri[:, 2])


def test_fft_closure_equals_brute_force(tiny_periodic):
    spec, cat, sc, X0 = tiny_periodic
    kb = (0.02, 0.02, 5)  # k_max = 0.12 < k_N/2 = 0.126: no aliasing of the closure
    tri = B.triangles(kb)
    X2 = B.los_field(spec, X0, 2)
    Bfft, nt, raw = B.scoccimarro_fft(spec, X0, {2: X2}, kb, tri, sc["I33"], (0, 2))
    s0, c0 = B.scoccimarro_brute(spec, X0, X0, kb, tri)
    s2, _ = B.scoccimarro_brute(spec, X0, X2, kb, tri)
    np.testing.assert_allclose(nt, c0, rtol=1e-12, atol=1e-9)
    scale = np.max(np.abs(s0))
    np.testing.assert_allclose(raw[0], np.real(s0), atol=1e-12 * scale)
    np.testing.assert_allclose(raw[2], np.real(s2), atol=1e-12 * scale)
    assert np.max(np.abs(np.imag(s0))) < 1e-9 * scale
    ok = c0 > 0
    np.testing.assert_allclose(Bfft[0][ok], np.real(s0[ok]) / (sc["I33"] * c0[ok]), rtol=1e-10)


def test_compressed_fft_equals_pair_enumeration(tiny_periodic):
    spec, cat, sc, X0 = tiny_periodic
    kb = (0.02, 0.03, 3)
    prs = B.pairs(kb)
    X2 = B.los_field(spec, X0, 2)
    _, s, cnt = B.compressed_fft(spec, X0, X2, kb, prs, sc["I33"], 2)
    n = spec["n"]
    _, lists = B._mode_lists(spec, kb)
    for t, (i, j) in enumerate(prs):
        q1, q2 = lists[i], lists[j]
        q3 = (-(q1[:, None, :] + q2[None, :, :])) % n
        i1, i2 = q1 % n, q2 % n
        v = (X0[i1[:, 0], i1[:, 1], i1[:, 2]][:, None] * X0[i2[:, 0], i2[:, 1], i2[:, 2]][None, :]
             * X2[q3[..., 0], q3[..., 1], q3[..., 2]])
        assert abs(np.sum(v) - s[t]) < 1e-11 * np.sum(np.abs(v))
        assert cnt[i] == len(q1) and cnt[j] == len(q2)


def test_compression_identity(tiny_periodic):
    """sum_k N_T(i,j,k) B^(leg 3)(i,j,k) over k3 bins covering [0, k_i + k_j] = N_i N_j B_l0l(i,j)
    (pre-shot), Sec. 4: the compressed estimator is the Scoccimarro one summed along k3."""
    spec, cat, sc, X0 = tiny_periodic
    dk = 0.02
    kb = (0.0, dk, 12)
    X2 = B.los_field(spec, X0, 2)
    f0 = B.shell_fields(spec, X0, kb)
    f2 = B.shell_fields(spec, X2, kb)
    n = spec["n"]
    _, _, cnt = B.compressed_fft(spec, X0, X2, kb, np.array([[1, 2]]), sc["I33"], 2)
    for (i, j) in [(1, 1), (1, 2), (2, 3)]:
        lhs = sum(np.sum(f0[i] * f0[j] * f2[k]) for k in range(kb[2])) / n**3
        val, s, _ = B.compressed_fft(spec, X0, X2, kb, np.array([[i, j]]), sc["I33"], 2)
        assert abs(lhs - s[0]) < 1e-10 * (abs(lhs) + abs(s[0]) + 1e-30)
        assert val[0] == pytest.approx(5 * s[0] / (sc["I33"] * cnt[i] * cnt[j]), rel=1e-12)


def test_compressed_collapse_matches_explicit_3j():
    """The collapsed B_l0l (Fourier-space Yamamoto F_l at the k3 leg) equals the definition with the
    explicit (m1, M) sum and Wigner 3j symbols, endpoint line of sight (survey geometry)."""
    g, r, origin = make_survey_catalogs(1500, 12000, 600.0, 900.0, 12, seed=21, fkp_p0=1e4)
    spec = dict(n=20, box=600.0, origin=tuple(origin), assign=2, interlace=0, los="endpoint",
                observer=(0.0, 0.0, 0.0))
    sc = P.catalog_scalars(g, r)
    meshes = P.fkp_meshes(spec, g, r, sc)
    fields, _ = P.fields_plain(spec, meshes, [0, 2])
    kb = (0.011, 0.0135, 3)  # k_max = 0.0515 < k_N/2 = 0.052
    prs = B.pairs(kb)
    val, _, _ = B.compressed_fft(spec, fields[0], fields[2], kb, prs, sc["I33"], 2)
    exp = B.compressed_explicit(spec, meshes, kb, prs, sc["I33"], 2)
    assert np.max(np.abs(np.imag(exp))) < 1e-9 * np.max(np.abs(val))
    np.testing.assert_allclose(np.real(exp), val, rtol=1e-9, atol=1e-12 * np.max(np.abs(val)))


def test_triangle_count_thin_shell_limit():
    """N_T -> V_T / k_f^6 = 8 pi^2 c1 c2 c3 dk^3 / k_f^6 (Sec. 5.2, Appendix I) for triangles away
    from the closure boundary and the smallest shells (k_max < k_N/2: no aliasing)."""
    n, box = 64, 1000.0
    kf = 2 * pi / box
    spec = _periodic_spec(n, box, 2, 0)
    kb = (4 * kf, 2 * kf, 6)
    tri = B.triangles(kb)
    ind = B.shell_fields(spec, None, kb, ones=True)
    c = B.bin_centres(kb)
    ratios = []
    for i, j, k in tri:
        if c[i] + c[j] - c[k] >= 1.5 * kb[1] and i >= 2:
            nt = np.sum(ind[i] * ind[j] * ind[k]) / n**3
            vt = 8 * pi**2 * c[i] * c[j] * c[k] * kb[1] ** 3 / kf**6
            ratios.append(nt / vt)
    ratios = np.array(ratios)
    assert ratios.size >= 10
    assert np.all(np.abs(ratios - 1) < 0.06)


def test_global_line_of_sight_enters_by_direction_only():
    """los_dir is a direction: (1, 2, 2) and (1/3, 2/3, 2/3) give the same B_0, B_2, B_000, B_202 and
    analytic shot noise (B_2 is far from zero here, so the comparison is not empty)."""
    cat = make_periodic_catalog(4000, 300.0, 16, seed=12)
    kb = (0.02, 0.02, 5)
    base = _periodic_spec(24, 300.0)
    a = B.bispectrum(dict(base, los_dir=(1.0, 2.0, 2.0)), cat, None, kb, (0, 2), (0, 2))
    b = B.bispectrum(dict(base, los_dir=(1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)), cat, None, kb, (0, 2), (0, 2))
    scale = np.max(np.abs(a["B"][0]))
    assert np.max(np.abs(a["B"][2])) > 1e-2 * scale
    for key in ("B", "BB", "shot_B", "shot_BB"):
        for ell in (0, 2):
            np.testing.assert_allclose(a[key][ell], b[key][ell], rtol=1e-10, atol=1e-10 * scale)


@pytest.mark.slow
def test_poisson_shot_noise_is_subtracted():
    """Uniform Poisson catalogues (no clustering): the raw monopole B_0 averages to the analytic
    shot noise, and B_l - N^(l), B_l0l - N_l0l average to zero within the sample scatter (Sec. 5.1:
    B_shot = sum P/n + 1/n^2)."""
    n, box, npart, nseed = 32, 400.0, 6000, 12
    kb = (0.03, 0.03, 3)  # k_max = 0.12 < k_N/2 = 0.126
    rows = {k: [] for k in ("B0", "N0", "B2", "N2", "BB0", "NB0", "BB2", "NB2")}
    for seed in range(nseed):
        rng = np.random.default_rng(4000 + seed)
        pos = rng.random((npart, 3)) * box
        cat = SimpleNamespace(pos=pos, w=np.ones(npart), nbar=np.full(npart, npart / box**3))
        spec = _periodic_spec(n, box)
        res = B.bispectrum(spec, cat, None, kb, (0, 2), (0, 2), shot=True)
        rows["B0"].append(res["B"][0])
        rows["N0"].append(res["shot_B"][0])
        rows["B2"].append(res["B"][2])
        rows["N2"].append(res["shot_B"][2])
        rows["BB0"].append(res["BB"][0])
        rows["NB0"].append(res["shot_BB"][0])
        rows["BB2"].append(res["BB"][2])
        rows["NB2"].append(res["shot_BB"][2])
    r = {k: np.array(v) for k, v in rows.items()}
    level = (box**3 / npart) ** 2
    for sig, noi in (("B0", "N0"), ("B2", "N2"), ("BB0", "NB0"), ("BB2", "NB2")):
        d = r[sig] - r[noi]
        se = d.std(axis=0, ddof=1) / np.sqrt(nseed)
        assert np.all(np.abs(d.mean(axis=0)) < 4 * se + 0.02 * level), sig
    assert np.all(np.abs(r["N0"].mean(axis=0) / level - 1) < 0.1)


# --- FFT-method (exact triplet) shot noise ------------------------------------------------------

def _object_fields(spec, pos, w):
    """Uncompensated transforms of a few point objects: X(q) = sum_p w_p e^{-i q.x_p} and the
    N-field sum_p w_p^2 e^{-i q.x_p}, on the integer grid of spec."""
    (kx, ky, kz), _ = M.kvectors(spec["n"], spec["box"])
    X = np.zeros((spec["n"],) * 3, dtype=np.complex128)
    N = np.zeros_like(X)
    for p, wp in zip(pos, w):
        e = np.exp(-1j * (kx * p[0] + ky * p[1] + kz * p[2]))
        X += wp * e
        N += wp * wp * e
    return X, N


def _distinct_triple_part(spec, pos, w, kbins, tri, ell):
    """(2l+1)/N_T sum over closed triplets of L_l(mu1) sum_{a, b, c distinct} w_a w_b w_c
    e^{-i(q1.x_a + q2.x_b + q3.x_c)}, by explicit loops over modes (independent of the oracle)."""
    from oracle import harmonics as Hm

    n, box = spec["n"], spec["box"]
    kf = 2 * pi / box
    b, _ = M.bin_index(n, box, *kbins)
    ii = M.int_freqs(n)
    modes = [[] for _ in range(kbins[2])]
    for a in range(n):
        for c in range(n):
            for e in range(n):
                if b[a, c, e] >= 0:
                    modes[b[a, c, e]].append((ii[a], ii[c], ii[e]))
    out = []
    for i, j, k in tri:
        tot, cnt = 0.0, 0
        for q1 in modes[i]:
            l1 = float(Hm.legendre(ell, q1[2] / np.sqrt(q1[0] ** 2 + q1[1] ** 2 + q1[2] ** 2)))
            for q2 in modes[j]:
                q3 = (-q1[0] - q2[0], -q1[1] - q2[1], -q1[2] - q2[2])
                if max(abs(q3[0]), abs(q3[1]), abs(q3[2])) >= n // 2:
                    continue
                if b[q3[0] % n, q3[1] % n, q3[2] % n] != k:
                    continue
                cnt += 1
                s = 0.0
                for xa in range(len(w)):
                    for xb in range(len(w)):
                        for xc in range(len(w)):
                            if len({xa, xb, xc}) < 3:
                                continue
                            ph = sum(kf * (q1[d] * pos[xa][d] + q2[d] * pos[xb][d] + q3[d] * pos[xc][d])
                                     for d in range(3))
                            s += w[xa] * w[xb] * w[xc] * np.cos(ph)
                tot += l1 * s
        out.append((2 * ell + 1) * tot / cnt if cnt else 0.0)
    return np.array(out)


@pytest.mark.parametrize("ell", [0, 2])
def test_fft_shot_equals_raw_estimator_for_two_objects(ell):
    """With at most two objects every closed triplet takes two legs from one object, so the raw
    estimator (no window, I33 = 1) equals the FFT-method shot noise exactly."""
    from oracle import shot as S

    spec = _periodic_spec(12, 100.0)
    kf = 2 * pi / 100.0
    kb = (0.5 * kf, 1.0 * kf, 3)
    tri = B.triangles(kb)
    pos = [(13.7, 42.1, 77.3), (61.2, 5.9, 30.4)]
    w = [0.8, 1.7]
    X, N = _object_fields(spec, pos, w)
    Xl = B.los_field(spec, X, ell)
    sums, counts = B.scoccimarro_brute(spec, X, Xl, kb, tri)
    raw = (2 * ell + 1) * np.real(sums) / counts
    s3 = sum(x ** 3 for x in w)
    sn = S.fft_method_shot_noise(spec, X, N, kb, tri, 1.0, s3, [ell])[ell]
    scale = np.max(np.abs(raw))
    assert scale > 0
    np.testing.assert_allclose(sn, raw, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("ell", [0, 2])
def test_fft_shot_leaves_the_distinct_triples(ell):
    """With three objects, raw estimator minus FFT-method shot noise is the sum over triples of
    three distinct objects (evaluated here by explicit loops)."""
    from oracle import shot as S

    spec = _periodic_spec(10, 100.0)
    kf = 2 * pi / 100.0
    kb = (0.5 * kf, 1.0 * kf, 3)
    tri = B.triangles(kb)
    pos = [(13.7, 42.1, 77.3), (61.2, 5.9, 30.4), (88.8, 70.2, 12.6)]
    w = [0.8, 1.7, 1.1]
    X, N = _object_fields(spec, pos, w)
    Xl = B.los_field(spec, X, ell)
    sums, counts = B.scoccimarro_brute(spec, X, Xl, kb, tri)
    raw = (2 * ell + 1) * np.real(sums) / counts
    s3 = sum(x ** 3 for x in w)
    sn = S.fft_method_shot_noise(spec, X, N, kb, tri, 1.0, s3, [ell])[ell]
    distinct = _distinct_triple_part(spec, pos, w, kb, tri, ell)
    scale = np.max(np.abs(raw))
    np.testing.assert_allclose(raw - sn, distinct, rtol=0, atol=1e-11 * scale)


def _distinct_pair_part(spec, pos, w, kbins, prs, ell):
    """(2l+1)/(N_i N_j) sum over q1 in b_i, q2 in b_j (q3 = -q1-q2 on the grid) of L_l(mu3)
    sum_{a, b, c distinct} w_a w_b w_c e^{-i(q1.x_a + q2.x_b + q3.x_c)}, by explicit loops."""
    from oracle import harmonics as Hm

    n, box = spec["n"], spec["box"]
    kf = 2 * pi / box
    b, _ = M.bin_index(n, box, *kbins)
    ii = M.int_freqs(n)
    modes = [[] for _ in range(kbins[2])]
    for a in range(n):
        for c in range(n):
            for e in range(n):
                if b[a, c, e] >= 0:
                    modes[b[a, c, e]].append((ii[a], ii[c], ii[e]))
    out = []
    for i, j in prs:
        tot = 0.0
        for q1 in modes[i]:
            for q2 in modes[j]:
                q3 = tuple(int(ii[(-q1[d] - q2[d]) % n]) for d in range(3))
                r = np.sqrt(sum(x * x for x in q3))
                l3 = float(Hm.legendre(ell, q3[2] / r if r > 0 else 0.0))
                s = 0.0
                for xa in range(len(w)):
                    for xb in range(len(w)):
                        for xc in range(len(w)):
                            if len({xa, xb, xc}) < 3:
                                continue
                            ph = sum(kf * (q1[d] * pos[xa][d] + q2[d] * pos[xb][d] + q3[d] * pos[xc][d])
                                     for d in range(3))
                            s += w[xa] * w[xb] * w[xc] * np.cos(ph)
                tot += l3 * s
        out.append((2 * ell + 1) * tot / (len(modes[i]) * len(modes[j])))
    return np.array(out)


@pytest.mark.parametrize("ell", [0, 2])
@pytest.mark.parametrize("nobj", [2, 3])
def test_compressed_fft_shot_object_identities(ell, nobj):
    """Compressed B_l0l: with two objects the raw estimator equals the FFT-method shot noise; with
    three, the difference is the distinct-triple sum (explicit loops)."""
    from oracle import shot as S

    spec = _periodic_spec(16, 100.0)   # k_max = 3.5 k_f < n k_f / 4: q1 + q2 stays off the Nyquist planes
    kf = 2 * pi / 100.0
    kb = (0.5 * kf, 1.0 * kf, 3)
    prs = B.pairs(kb)
    pos = [(13.7, 42.1, 77.3), (61.2, 5.9, 30.4), (88.8, 70.2, 12.6)][:nobj]
    w = [0.8, 1.7, 1.1][:nobj]
    X, N = _object_fields(spec, pos, w)
    Xl = B.los_field(spec, X, ell)
    raw, _, _ = B.compressed_fft(spec, X, Xl, kb, prs, 1.0, ell)
    s3 = sum(x ** 3 for x in w)
    sn = S.compressed_fft_method_shot(spec, X, N, kb, prs, 1.0, s3, [ell])[ell]
    scale = np.max(np.abs(raw))
    want = 0.0 if nobj == 2 else _distinct_pair_part(spec, pos, w, kb, prs, ell)
    np.testing.assert_allclose(raw - sn, want, rtol=0, atol=1e-11 * scale)


def test_survey_l2_tends_to_global_los_for_a_distant_observer():
    """Survey geometry (Yamamoto X_2 with the line of sight to each grid point, the self term from
    the objects' own directions) equals the global-LOS form in the limit of a distant observer,
    where every direction is the box's (1,1,1)/sqrt(3): B_2, B_202 and their analytic shot noise."""
    box, dist = 600.0, 1.0e8
    g, r, origin = make_survey_catalogs(3000, 30000, box, dist, 12, seed=23, fkp_p0=1e4, dtype=np.float64)
    kb = (0.011, 0.0135, 3)
    common = dict(n=20, box=box, origin=tuple(origin), assign=3, interlace=1)
    surv = B.bispectrum(dict(common, los="endpoint", observer=(0.0, 0.0, 0.0)), g, r, kb, (0, 2), (0, 2))
    d = np.ones(3) / np.sqrt(3.0)
    glob = B.bispectrum(dict(common, los="global", los_dir=tuple(d)), g, r, kb, (0, 2), (0, 2))
    st = np.abs(glob["B"][0]) + np.abs(glob["shot_B"][0])
    sp = np.abs(glob["BB"][0]) + np.abs(glob["shot_BB"][0])
    for key, scale in (("B", st), ("shot_B", st), ("BB", sp), ("shot_BB", sp)):
        for ell in (0, 2):
            err = np.abs(surv[key][ell] - glob[key][ell]) / scale
            assert np.max(err) < 1e-5, (key, ell, np.max(err))
    # and a nearby observer changes B_2 (the line of sight varies across the box)
    g2, r2, origin2 = make_survey_catalogs(3000, 30000, box, 900.0, 12, seed=23, fkp_p0=1e4, dtype=np.float64)
    near = B.bispectrum(dict(common, origin=tuple(origin2), los="endpoint", observer=(0.0, 0.0, 0.0)), g2, r2,
                        kb, (2,), (), shot=False)
    nearg = B.bispectrum(dict(common, origin=tuple(origin2), los="global", los_dir=tuple(d)), g2, r2, kb, (2,), (),
                         shot=False)
    assert np.max(np.abs(near["B"][2] - nearg["B"][2])) > 1e-3 * np.max(np.abs(nearg["B"][2]))


def test_analytic_shot_noise_tracks_the_fft_method():
    """The thin-shell analytic shot noise of B_l and B_l0l (Sec. 5.4.1, 5.4.3) against the exact
    FFT-method sums (Sec. 5.4.2) on the same catalogue: within a few per cent of the monopole
    shot-noise scale (median), larger only on the few triangles of thin low-k bins."""
    spec = _periodic_spec(32, 300.0)
    cat = make_periodic_catalog(20000, 300.0, 32, seed=5)
    res = B.bispectrum(spec, cat, None, (0.02, 0.02, 5), (0, 2), (0, 2), shot="fft")
    for key, fkey, med, mx in (("shot_B", "shot_B_fft", 0.03, 0.2), ("shot_BB", "shot_BB_fft", 0.02, 0.1)):
        scale = np.abs(res[fkey][0])
        for ell in (0, 2):
            rel = np.abs(res[key][ell] - res[fkey][ell]) / scale
            assert np.median(rel) < med and np.max(rel) < mx, (key, ell, np.median(rel), np.max(rel))


def test_cross_bispectrum_identities():
    """Multi-tracer B_l and B_l0l (raw): three equal tracers give the auto estimator; with a copy
    translated by whole cells d on leg 3 every closed triple carries exp(-i q3.d) (enumerated)."""
    n, box = 16, 300.0
    spec = _periodic_spec(n, box)
    kb = (0.02, 0.02, 3)
    cat = make_periodic_catalog(4000, box, 16, seed=11)
    auto = B.bispectrum(spec, cat, None, kb, (0, 2), (0, 2), shot=False)
    same = B.cross_bispectrum(spec, [(cat, None)] * 3, kb, (0, 2), (0, 2))
    for key in ("B", "BB"):
        for ell in (0, 2):
            np.testing.assert_allclose(same[key][ell], auto[key][ell], rtol=1e-11,
                                       atol=1e-12 * np.max(np.abs(auto[key][0])))
    h = box / n
    d = np.array([3, 1, 2])
    from oracle import harmonics as Hm
    from synthetic import Catalog

    moved = Catalog(np.mod(cat.pos.astype(np.float64) + d * h, box), cat.w, cat.nbar)
    cross = B.cross_bispectrum(spec, [(cat, None), (cat, None), (moved, None)], kb, (0, 2), ())
    X = same["fields"][0]
    b, lists = B._mode_lists(spec, kb)
    for ell in (0, 2):
        want = []
        for (i, j, k), nt in zip(cross["tri"], cross["NT"]):
            q1, q2 = lists[i], lists[j]
            q3 = -(q1[:, None, :] + q2[None, :, :])
            inb = (b[q3[..., 0] % n, q3[..., 1] % n, q3[..., 2] % n] == k) & np.all(np.abs(q3) < n // 2, axis=-1)
            i1, i2, i3 = q1 % n, q2 % n, q3 % n
            mu1 = q1[:, 2] / np.linalg.norm(q1, axis=1)
            v = (Hm.legendre(ell, mu1) * X[i1[:, 0], i1[:, 1], i1[:, 2]])[:, None] * X[i2[:, 0], i2[:, 1], i2[:, 2]][None, :]
            v = v * X[i3[..., 0], i3[..., 1], i3[..., 2]] * np.exp(-1j * (q3 @ d) * 2 * pi / n)
            want.append((2 * ell + 1) * np.real(np.sum(np.where(inb, v, 0.0))) / (cross["I33"] * nt) if nt > 0 else 0.0)
        scale = np.max(np.abs(auto["B"][0]))
        assert np.max(np.abs(cross["B"][ell] - np.array(want))) < 1e-10 * scale, ell


def test_odd_multipoles_enumeration_and_distant_observer():
    """B_1, B_3 (imaginary part of the closure sum with the odd field on leg 1): equal to the
    explicit enumeration of the closed triples with a global line of sight, and, in survey geometry,
    to the global-line-of-sight form when the observer is far away (a nearby one changes B_1)."""
    from oracle import harmonics as Hm

    n, box = 16, 300.0
    kb = (0.02, 0.02, 3)
    cat = make_periodic_catalog(4000, box, 16, seed=11)
    spec = dict(_periodic_spec(n, box), los_dir=(1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0))
    res = B.odd_multipoles(spec, cat, None, kb)
    X = res["X0"]
    b, lists = B._mode_lists(spec, kb)
    d = np.asarray(spec["los_dir"])
    for ell in (1, 3):
        want = []
        for (i, j, k), nt in zip(res["tri"], res["NT"]):
            q1, q2 = lists[i], lists[j]
            q3 = -(q1[:, None, :] + q2[None, :, :])
            inb = (b[q3[..., 0] % n, q3[..., 1] % n, q3[..., 2] % n] == k) & np.all(np.abs(q3) < n // 2, axis=-1)
            i1, i2, i3 = q1 % n, q2 % n, q3 % n
            mu1 = (q1 @ d) / np.linalg.norm(q1, axis=1)
            v = (Hm.legendre(ell, mu1) * X[i1[:, 0], i1[:, 1], i1[:, 2]])[:, None] * X[i2[:, 0], i2[:, 1], i2[:, 2]][None, :]
            v = v * X[i3[..., 0], i3[..., 1], i3[..., 2]]
            want.append((2 * ell + 1) * np.imag(np.sum(np.where(inb, v, 0.0))) / (res["I33"] * nt) if nt > 0 else 0.0)
        scale = np.max(np.abs(res["B"][ell]))
        assert scale > 0 and np.max(np.abs(res["B"][ell] - np.array(want))) < 1e-10 * scale, ell
    # survey geometry: distant observer -> global line of sight along the box direction
    boxs, kbs = 600.0, (0.011, 0.0135, 3)
    dd = np.ones(3) / np.sqrt(3.0)
    out = {}
    for dist in (1.0e8, 900.0):
        g, r, origin = make_survey_catalogs(3000, 30000, boxs, dist, 12, seed=23, fkp_p0=1e4, dtype=np.float64)
        common = dict(n=20, box=boxs, origin=tuple(origin), assign=3, interlace=1, periodic=0)
        ep = B.odd_multipoles(dict(common, los="endpoint", observer=(0.0, 0.0, 0.0)), g, r, kbs)
        gl = B.odd_multipoles(dict(common, los="global", los_dir=tuple(dd)), g, r, kbs)
        out[dist] = (ep, gl)
    ep, gl = out[1.0e8]
    for ell in (1, 3):
        sc = np.max(np.abs(gl["B"][ell]))
        assert np.max(np.abs(ep["B"][ell] - gl["B"][ell])) < 1e-4 * sc, ell
    ep, gl = out[900.0]
    assert np.max(np.abs(ep["B"][1] - gl["B"][1])) > 1e-2 * np.max(np.abs(gl["B"][1]))
