"""Pins for oracle.sugiyama (the TripoSH B_{l1 l2 L} of Eq. sugi_estimator)."""
import numpy as np
import pytest

from oracle import bispec as B
from oracle import harmonics as H
from oracle import mesh as M
from oracle import power as P
from oracle import sugiyama as S
from synthetic import Catalog, make_periodic_catalog

KB = (0.02, 0.02, 3)   # k_max = 0.08 < k_N/2 = 0.084 at n = 16, L = 300
MULTIPOLES = [(0, 0, 0), (1, 1, 0), (1, 1, 2), (2, 0, 2), (0, 2, 2), (2, 2, 0), (2, 2, 2), (2, 2, 4)]
TILT = (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)


def _spec(n, los_dir=(0.0, 0.0, 1.0)):
    return dict(n=n, box=300.0, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global",
                los_dir=los_dir, periodic=1)


@pytest.fixture(scope="module")
def cat():
    return make_periodic_catalog(4000, 300.0, 16, seed=11)


def _setup(cat, los_dir, n=16):
    spec = _spec(n, los_dir)
    sc = P.catalog_scalars(cat, None, 300.0)
    return spec, sc, P.fkp_meshes(spec, cat, None, sc)


def _scale(res):
    return np.max(np.abs(res[(0, 0, 0)]))


def test_valid_multipoles():
    assert S.valid_multipole(2, 0, 2) and S.valid_multipole(1, 1, 2) and S.valid_multipole(2, 2, 4)
    assert not S.valid_multipole(1, 0, 0) and not S.valid_multipole(2, 0, 0) and not S.valid_multipole(2, 2, 1)


@pytest.mark.parametrize("los_dir", [(0.0, 0.0, 1.0), TILT])
def test_fft_against_mode_pair_enumeration(cat, los_dir):
    """sum_x F F G equals the explicit (q1, q2) sum (the Kronecker delta of the closure) exactly."""
    spec, sc, meshes = _setup(cat, los_dir)
    res = S.sugiyama_fft(spec, meshes, KB, MULTIPOLES, sc["I33"])
    prs = [(0, 0), (0, 2), (2, 1), (1, 2), (2, 2)]
    for mp in [(0, 0, 0), (1, 1, 2), (2, 0, 2), (0, 2, 2), (2, 2, 2), (2, 2, 4)]:
        brute = S.sugiyama_brute(spec, meshes, KB, mp, sc["I33"], prs)
        got = np.array([res[mp][i, j] for i, j in prs])
        assert np.max(np.abs(got - brute)) < 1e-11 * _scale(res), mp


@pytest.mark.parametrize("los_dir", [(0.0, 0.0, 1.0), TILT])
def test_ll0_against_legendre_form(cat, los_dir):
    """B_{l l 0}: the m-sum with 3j symbols collapses to the Legendre polynomial of the angle between
    q1 and q2 (addition theorem), independent of the line of sight."""
    spec, sc, meshes = _setup(cat, los_dir)
    res = S.sugiyama_fft(spec, meshes, KB, [(0, 0, 0), (1, 1, 0), (2, 2, 0)], sc["I33"])
    prs = [(i, j) for i in range(3) for j in range(3)]
    for ell in (0, 1, 2):
        leg = S.legendre_ll0(spec, meshes, KB, ell, sc["I33"], prs)
        got = np.array([res[(ell, ell, 0)][i, j] for i, j in prs])
        assert np.max(np.abs(got - leg)) < 1e-11 * _scale(res), ell


def test_monopole_equals_compressed_monopole(cat):
    """Sec. 6: the compressed estimator's B_000 coincides with Sugiyama's B_000."""
    spec, sc, meshes = _setup(cat, (0.0, 0.0, 1.0))
    res = S.sugiyama_fft(spec, meshes, KB, [(0, 0, 0)], sc["I33"])
    X0 = P.fields_plain(spec, meshes, [0])[0][0]
    prs = B.pairs(KB)
    comp, _, _ = B.compressed_fft(spec, X0, X0, KB, prs, sc["I33"], 0)
    got = np.array([res[(0, 0, 0)][i, j] for i, j in prs])
    np.testing.assert_allclose(np.real(got), comp, rtol=1e-11, atol=1e-13 * np.max(np.abs(comp)))


@pytest.mark.parametrize("los_dir", [(0.0, 0.0, 1.0), TILT])
def test_halved_sum_and_reality(cat, los_dir):
    """Eq. sym_sugi: the paired sub-configurations are complex conjugates, so the boxed half-sum
    (eta = 2, real part) equals the full sum, which is real."""
    spec, sc, meshes = _setup(cat, los_dir)
    mps = [(1, 1, 2), (2, 0, 2), (2, 2, 2), (2, 2, 4)]
    full = S.sugiyama_fft(spec, meshes, KB, mps + [(0, 0, 0)], sc["I33"])
    half = S.sugiyama_halved(spec, meshes, KB, mps, sc["I33"])
    for mp in mps:
        assert np.max(np.abs(np.imag(full[mp]))) < 1e-12 * _scale(full), mp
        assert np.max(np.abs(np.real(full[mp]) - half[mp])) < 1e-12 * _scale(full), mp


def test_cyclic_axis_permutation(cat):
    """A cyclic permutation of the axes is a rotation: applied to the catalogue and the line of
    sight together it leaves every B_{l1 l2 L} unchanged (the tilted line of sight makes every
    G_L^M with M != 0 contribute)."""
    spec, sc, meshes = _setup(cat, TILT)
    res = S.sugiyama_fft(spec, meshes, KB, MULTIPOLES, sc["I33"])
    rot = Catalog(np.ascontiguousarray(cat.pos[:, [1, 2, 0]]), cat.w, cat.nbar)
    spec_r, sc_r, meshes_r = _setup(rot, (TILT[1], TILT[2], TILT[0]))
    res_r = S.sugiyama_fft(spec_r, meshes_r, KB, MULTIPOLES, sc_r["I33"])
    for mp in MULTIPOLES:
        assert np.max(np.abs(res[mp] - res_r[mp])) < 1e-11 * _scale(res), mp
    # and the multipoles with l > 0 do depend on the line of sight
    spec_z, sc_z, meshes_z = _setup(cat, (0.0, 0.0, 1.0))
    res_z = S.sugiyama_fft(spec_z, meshes_z, KB, [(0, 0, 0), (2, 0, 2)], sc_z["I33"])
    assert np.max(np.abs(res_z[(2, 0, 2)] - res[(2, 0, 2)])) > 1e-3 * _scale(res)


def test_l0l_reduces_to_legendre_shell_along_z(cat):
    """Line of sight along z: only M = 0 survives and B_l0l = (2l+1)/(I33 N_i N_j n^3)
    sum_x F_l(x; k_i) F_0(x; k_j) G(x), with F_l the shell of L_l(mu) X and G the full-range X."""
    spec, sc, meshes = _setup(cat, (0.0, 0.0, 1.0))
    res = S.sugiyama_fft(spec, meshes, KB, [(0, 0, 0), (2, 0, 2)], sc["I33"])
    n = spec["n"]
    X0 = P.fields_plain(spec, meshes, [0])[0][0]
    f0 = B.shell_fields(spec, X0, KB)
    f2 = B.shell_fields(spec, B.los_field(spec, X0, 2), KB)
    g = np.real(np.fft.ifftn(X0)) * n**3
    cnt = S.mode_counts(spec, KB)
    for i in range(3):
        for j in range(3):
            want = 5.0 * np.sum(f2[i] * f0[j] * g) / (n**3 * sc["I33"] * cnt[i] * cnt[j])
            assert abs(res[(2, 0, 2)][i, j] - want) < 1e-11 * _scale(res)


def test_wigner_coefficients_of_the_l0l_collapse():
    """H N (l 0 l; 0 0 0) = 2l + 1: the normalisation the reduction above relies on."""
    for ell in range(5):
        hN = H.wigner3j(ell, 0, ell, 0, 0, 0) * (2 * ell + 1) ** 2
        assert abs(hN * H.wigner3j(ell, 0, ell, 0, 0, 0) - (2 * ell + 1)) < 1e-12


def _ring_quadrature(l1, l2, L, k1, k2, k3, u3, ng=2048):
    """Mean over the ring of k1 around k3 (k1 + k2 + k3 = 0) of
    sum_m (l1 l2 L; m -m 0) y_l1^{m*}(k1hat) y_l2^{-m*}(k2hat), by direct quadrature."""
    u3 = u3 / np.linalg.norm(u3)
    c13 = (k2 * k2 - k1 * k1 - k3 * k3) / (2 * k1 * k3)
    a = np.array([1.0, 0.0, 0.0]) if abs(u3[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = a - a.dot(u3) * u3
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u3, e1)
    g = np.arange(ng) * 2 * np.pi / ng
    kv1 = k1 * (c13 * u3[None, :] + np.sqrt(1 - c13 * c13) * (np.cos(g)[:, None] * e1 + np.sin(g)[:, None] * e2))
    kv2 = -kv1 - k3 * u3[None, :]
    tot = 0.0 + 0.0j
    for m in range(-min(l1, l2), min(l1, l2) + 1):
        w = H.wigner3j(l1, l2, L, m, -m, 0)
        tot += w * np.mean(np.conj(H.ylm_racah(l1, m, kv1)) * np.conj(H.ylm_racah(l2, -m, kv2)))
    return tot


@pytest.mark.parametrize("mp", [(0, 0, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2), (3, 1, 2), (4, 2, 2), (1, 3, 4),
                                (2, 4, 6), (4, 4, 8)])
def test_lemma1_closed_form_against_ring_quadrature(mp):
    """The ring average of the m-sum around k3 equals q_{l1 l2 L}(k1, k2, k3) L_L(mu3) (Lemma 1 with
    the Racah-normalised associated Legendre functions)."""
    rng = np.random.default_rng(7)
    done = 0
    while done < 4:
        k1, k2, k3 = rng.uniform(0.04, 0.12, 3)
        if not abs(k1 - k2) < k3 < k1 + k2:
            continue
        u3 = rng.normal(size=3)
        ring = _ring_quadrature(*mp, k1, k2, k3, u3)
        pred = S.q_ring(*mp, k1, k2, k3) * H.legendre(mp[2], u3[2] / np.linalg.norm(u3))
        assert abs(ring.imag) < 1e-12 and abs(ring.real - pred) < 1e-12, (mp, ring, pred)
        done += 1


def test_monopole_shot_noise_equals_the_compressed_one(cat):
    """B_000: the TripoSH analytic shot noise (S + H_0(k1) + H_0(k2) + <Q_0>)/I33 equals the
    compressed estimator's analytic B_000 shot noise (g_0 = 1)."""
    from oracle import shot as SH

    spec, sc, meshes = _setup(cat, (0.0, 0.0, 1.0))
    nmeshes = P.fkp_meshes(spec, cat, None, sc, weight_power=2)
    X0 = P.fields_plain(spec, meshes, [0])[0][0]
    N0 = P.fields_plain(spec, nmeshes, [0])[0][0]
    sn = S.analytic_shot_noise(spec, X0, N0, KB, [(0, 0, 0), (2, 0, 2)], sc)
    prs = B.pairs(KB)
    _, bb, _ = SH.analytic_shot_noise(spec, X0, N0, KB, B.triangles(KB), prs, sc, (0,), (0,))
    got = np.array([sn[(0, 0, 0)][i, j] for i, j in prs])
    np.testing.assert_allclose(got, bb[0], rtol=1e-12)
    # symmetric in (k1, k2) for l1 = l2
    np.testing.assert_allclose(sn[(0, 0, 0)], sn[(0, 0, 0)].T, rtol=1e-12)


@pytest.mark.parametrize("los_dir", [(0.0, 0.0, 1.0), TILT])
def test_fft_method_shot_equals_raw_for_two_objects(los_dir):
    """Two point objects, uncompensated fields: every closed triple draws two legs from one object,
    so the raw estimator equals the FFT-method shot noise (all three pair terms and the -2 S)."""
    spec = _spec(16, los_dir)
    (kx, ky, kz), _ = M.kvectors(16, 300.0)
    pos, w = [(13.7, 142.1, 277.3), (161.2, 5.9, 30.4)], [0.8, 1.7]
    X = np.zeros((16,) * 3, dtype=np.complex128)
    N = np.zeros_like(X)
    for p, wp in zip(pos, w):
        e = np.exp(-1j * (kx * p[0] + ky * p[1] + kz * p[2]))
        X += wp * e
        N += wp * wp * e
    d = np.asarray(los_dir) / np.linalg.norm(los_dir)
    mps = [(0, 0, 0), (2, 0, 2), (0, 2, 2), (1, 1, 2), (2, 2, 2), (2, 2, 4)]
    dn = {(L, Mm): np.conj(H.ylm_racah(L, Mm, d)) * X for L in (0, 2, 4) for Mm in range(-L, L + 1)}
    raw = S.sugiyama_from_spectra(spec, X, dn, KB, mps, 1.0)
    sn = S.fft_method_shot_noise(spec, X, N, KB, mps, 1.0, sum(x ** 3 for x in w))
    scale = np.max(np.abs(raw[(0, 0, 0)]))
    for mp in mps:
        assert np.max(np.abs(np.real(raw[mp]) - sn[mp])) < 1e-11 * scale, mp


def test_analytic_shot_noise_tracks_the_fft_method():
    """The thin-shell analytic shot noise (Lemma 1 with Racah-normalised functions, mode-count
    weighted k3 average) stays within a few per cent of the exact FFT-method shot noise, relative to
    the B_000 shot-noise scale (Sec. 5.5 makes the same comparison); the printed unweighted form
    would be off by the mode counts."""
    spec = _spec(32)
    cat = make_periodic_catalog(20000, 300.0, 32, seed=5)
    sc = P.catalog_scalars(cat, None, 300.0)
    X0, _ = S.spectra(spec, P.fkp_meshes(spec, cat, None, sc), [])
    N0, _ = S.spectra(spec, P.fkp_meshes(spec, cat, None, sc, weight_power=2), [])
    kb = (0.05, 0.01, 8)
    mps = [(0, 0, 0), (2, 0, 2), (1, 1, 0), (2, 2, 0), (1, 1, 2)]
    an = S.analytic_shot_noise(spec, X0, N0, kb, mps, sc)
    ff = S.fft_method_shot_noise(spec, X0, N0, kb, mps, sc["I33"], sc["S3"])
    scale = np.abs(ff[(0, 0, 0)])
    for mp in mps:
        rel = np.abs(an[mp] - ff[mp]) / scale
        assert np.median(rel) < 0.03 and np.max(rel) < 0.12, (mp, np.median(rel), np.max(rel))


def test_endpoint_line_of_sight_tends_to_global_for_a_distant_observer():
    """Survey geometry (G_L^M from y_L^M-weighted transforms with the line of sight to each grid
    point) equals the global-line-of-sight estimator when the observer is so far away that every
    direction is the same; a nearby observer changes B_202."""
    from synthetic import make_survey_catalogs

    box, kb = 600.0, (0.011, 0.0135, 3)
    mps = [(0, 0, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)]
    d = np.ones(3) / np.sqrt(3.0)
    res = {}
    for dist in (1.0e8, 900.0):
        g, r, origin = make_survey_catalogs(3000, 30000, box, dist, 12, seed=23, fkp_p0=1e4, dtype=np.float64)
        common = dict(n=20, box=box, origin=tuple(origin), assign=3, interlace=1, periodic=0)
        ep = S.bispectrum_sugiyama(dict(common, los="endpoint", observer=(0.0, 0.0, 0.0)), g, r, kb, mps)
        gl = S.bispectrum_sugiyama(dict(common, los="global", los_dir=tuple(d)), g, r, kb, mps)
        res[dist] = (ep, gl)
    ep, gl = res[1.0e8]
    scale = np.max(np.abs(gl["B"][(0, 0, 0)]))
    for mp in mps:
        assert np.max(np.abs(ep["B"][mp] - gl["B"][mp])) < 5e-5 * scale, mp   # directions vary by box/dist ~ 6e-6
    ep, gl = res[900.0]
    assert np.max(np.abs(ep["B"][(2, 0, 2)] - gl["B"][(2, 0, 2)])) > 1e-3 * np.max(np.abs(gl["B"][(2, 0, 2)]))
