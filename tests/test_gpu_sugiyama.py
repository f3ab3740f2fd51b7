"""GPU parity: npc_bispectrum_sugiyama (TripoSH B_{l1 l2 L}, through the C ABI) against the FP64
oracle, which sums every (m1, m2, M) sub-configuration in the catalogue's own frame."""
import numpy as np
import pytest

from helpers import ensure_built, golden_module, stored_or_live
from oracle import power as P
from oracle import sugiyama as OS
from synthetic import make_periodic_catalog

pytestmark = pytest.mark.gpu

LOW = [(0, 0, 0), (1, 1, 0), (1, 1, 2), (2, 0, 2), (0, 2, 2), (2, 2, 0), (2, 2, 2), (2, 2, 4)]
HIGH = [(0, 0, 0), (3, 1, 2), (1, 3, 4), (3, 3, 0), (4, 0, 4), (4, 2, 2), (2, 4, 6), (4, 4, 8), (3, 3, 6)]
TILT = (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)


@pytest.fixture(scope="module")
def api():
    ensure_built()
    from paper_2605_04864_gb300 import api as A

    return A


def _spec(n, box, los_dir, periodic=1, origin=(0.0, 0.0, 0.0)):
    return dict(n=n, box=box, origin=origin, assign=3, interlace=1, los="global", los_dir=los_dir,
                periodic=periodic)


def _oracle(spec, cat, randoms, kb, mps):
    sc = P.catalog_scalars(cat, randoms, spec["box"])
    meshes = P.fkp_meshes(spec, cat, randoms, sc)
    return OS.sugiyama_fft(spec, meshes, kb, mps, sc["I33"]), OS.mode_counts(spec, kb)


def _check(res, orc, cnt, mps, tol):
    """Error relative to the B_000 scale of the same bin pair.  For l1 + l2 odd (odd L, line of sight
    to each grid point) the sum is imaginary and the library reports its imaginary part."""
    np.testing.assert_array_equal(res["nmodes"], cnt)
    scale = np.abs(np.real(orc[(0, 0, 0)]))
    for mp in mps:
        got = res["B"][mp]
        want = np.imag(orc[mp]) if (mp[0] + mp[1]) % 2 else np.real(orc[mp])
        e = np.abs(got - want) / np.maximum(np.abs(want), scale)
        assert np.max(e) < tol, (mp, np.max(e))


@pytest.mark.parametrize("mps", [LOW, HIGH], ids=["l<=2", "l<=4"])
@pytest.mark.parametrize("los_dir", [(0.0, 0.0, 1.0), TILT], ids=["z", "tilted"])
def test_fp64_periodic(api, mps, los_dir):
    cat = make_periodic_catalog(20000, 300.0, 32, seed=81)
    kb = (0.02, 0.02, 5)   # k_max = 0.12 < k_N/2 = 0.168
    res = api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=mps, los_dir=los_dir,
                                  precision="fp64")
    orc, cnt = _oracle(_spec(32, 300.0, los_dir), cat, None, kb, mps)
    _check(res, orc, cnt, mps, 1e-10)


@pytest.mark.parametrize("n", [64, 48])
def test_mixed_periodic(api, n):
    """Float32 shell fields and 3xTF32 tensor-core products; a radix-3 mesh as well."""
    box = 600.0 if n == 64 else 450.0
    cat = make_periodic_catalog(60000, box, 32, seed=83)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 6)   # k_max = 11 k_f < k_N/2 = n k_f / 4
    mps = [(0, 0, 0), (1, 1, 2), (2, 0, 2), (2, 2, 2)]
    res = api.bispectrum_sugiyama(cat, n=n, box=box, kbins=kb, multipoles=mps, los_dir=TILT, precision="mixed")
    orc, cnt = _oracle(_spec(n, box, TILT), cat, None, kb, mps)
    _check(res, orc, cnt, mps, 1e-4)


def test_survey_geometry_global_line_of_sight(api):
    """FKP field with randoms and a global line of sight."""
    from synthetic import make_survey_catalogs

    box = 600.0
    g, r, origin = make_survey_catalogs(20000, 200000, box, 900.0, 32, seed=85, fkp_p0=1e4)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 4)   # k_max = 8 k_f = k_N/2 at 32^3
    mps = [(0, 0, 0), (2, 0, 2), (1, 1, 2)]
    res = api.bispectrum_sugiyama(g, n=32, box=box, kbins=kb, multipoles=mps, los_dir=TILT, precision="fp64",
                                  origin=origin, randoms=r)
    orc, cnt = _oracle(_spec(32, box, TILT, periodic=0, origin=tuple(origin)), g, r, kb, mps)
    _check(res, orc, cnt, mps, 1e-10)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_analytic_shot_noise(api, prec, tol):
    """Sec. 5.4 analytic shot noise (S, H_L on k1 and k2, Lemma 1's ring average over the k3 shells)
    against the oracle; the estimate is the raw sum minus it."""
    cat = make_periodic_catalog(20000, 300.0, 32, seed=93)
    kb = (0.02, 0.02, 5)
    mps = [(0, 0, 0), (2, 0, 2), (0, 2, 2), (1, 1, 2), (2, 2, 2), (3, 1, 2), (4, 2, 2), (4, 4, 8)]
    res = api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=mps, shot=True, los_dir=TILT,
                                  precision=prec)
    spec = _spec(32, 300.0, TILT)
    orc = OS.bispectrum_sugiyama(spec, cat, None, kb, mps, shot=True)
    scale = np.abs(orc["B"][(0, 0, 0)]) + np.abs(orc["shot"][(0, 0, 0)])
    for mp in mps:
        e = np.abs(res["shot"][mp] - orc["shot"][mp]) / np.maximum(np.abs(orc["shot"][mp]), scale)
        assert np.max(e) < tol, ("shot", mp, np.max(e))
        e = np.abs(res["B"][mp] + res["shot"][mp] - orc["B"][mp]) / np.maximum(np.abs(orc["B"][mp]), scale)
        assert np.max(e) < tol, ("raw", mp, np.max(e))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_fft_method_shot_noise(api, prec, tol):
    """Sec. 5.4.2 FFT-method (exact) shot noise against the oracle's mode-pair enumeration, with a
    tilted line of sight (every sub-configuration of the oracle contributes)."""
    cat = make_periodic_catalog(20000, 300.0, 32, seed=97)
    kb = (0.02, 0.02, 5)
    mps = [(0, 0, 0), (2, 0, 2), (0, 2, 2), (1, 1, 2), (2, 2, 2), (3, 1, 2), (2, 2, 4)]
    res = api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=mps, shot="fft", los_dir=TILT,
                                  precision=prec)
    orc = OS.bispectrum_sugiyama(_spec(32, 300.0, TILT), cat, None, kb, mps, shot="fft")
    scale = np.abs(orc["B"][(0, 0, 0)]) + np.abs(orc["shot"][(0, 0, 0)])
    for mp in mps:
        e = np.abs(res["shot"][mp] - orc["shot"][mp]) / np.maximum(np.abs(orc["shot"][mp]), scale)
        assert np.max(e) < tol, ("shot", mp, np.max(e))
        e = np.abs(res["B"][mp] + res["shot"][mp] - orc["B"][mp]) / np.maximum(np.abs(orc["B"][mp]), scale)
        assert np.max(e) < tol, ("raw", mp, np.max(e))


def test_monopole_matches_the_compressed_estimator(api):
    """B_000 of the two estimators coincide (Sec. 6): the library's two paths agree."""
    cat = make_periodic_catalog(20000, 300.0, 32, seed=87)
    kb = (0.02, 0.02, 5)
    sug = api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=[(0, 0, 0)], shot=True,
                                  precision="fp64")
    comp = api.bispectrum(cat, n=32, box=300.0, kbins=kb, scoc_ells=(0,), tripo_ells=(0,), shot=True,
                          precision="fp64")
    prs = [(i, j) for i in range(5) for j in range(i, 5)]
    for key, ckey in (("B", "BB"), ("shot", "shot_BB")):
        got = np.array([sug[key][(0, 0, 0)][i, j] for i, j in prs])
        np.testing.assert_allclose(got, comp[ckey][0], rtol=1e-10, atol=1e-12 * np.max(np.abs(got)))


def test_rejects(api):
    cat = make_periodic_catalog(2000, 300.0, 16, seed=89)
    kb = (0.02, 0.02, 5)
    with pytest.raises(RuntimeError):   # odd l1 + l2 + L
        api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=[(1, 0, 0)])
    with pytest.raises(RuntimeError):   # odd L (odd-parity multipole)
        api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=[(1, 0, 1)])
    with pytest.raises(RuntimeError):   # l above 4
        api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=[(5, 5, 0)])
    with pytest.raises(RuntimeError):   # no such shot-noise mode
        api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=kb, multipoles=[(0, 0, 0)], shot=3)
    with pytest.raises(RuntimeError):   # aliasing closure
        api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=(0.02, 0.02, 8), multipoles=[(0, 0, 0)])
    from synthetic import make_survey_catalogs

    g, r, origin = make_survey_catalogs(2000, 20000, 600.0, 900.0, 16, seed=91, fkp_p0=1e4)
    with pytest.raises(RuntimeError):   # line of sight to each grid point: L above 4
        api.bispectrum_sugiyama(g, n=32, box=600.0, kbins=(0.02, 0.01, 3), multipoles=[(4, 2, 6)], origin=origin,
                                randoms=r, los_dir=None)
    with pytest.raises(RuntimeError):   # line of sight to each grid point: odd l1 + l2 + L
        api.bispectrum_sugiyama(g, n=32, box=600.0, kbins=(0.02, 0.01, 3), multipoles=[(1, 0, 0)], origin=origin,
                                randoms=r, los_dir=None)


def test_max_bins_and_empty_bins(api):
    """24 bins (the maximum; the staged fields then need two m tiles per warp) of half a fundamental
    frequency from k = 0, so the first bins hold no modes and must report zero."""
    box = 450.0
    kf = 2 * np.pi / box
    cat = make_periodic_catalog(40000, box, 32, seed=95)
    kb = (0.0, 0.5 * kf, 24)   # k_max = 12 k_f = k_N/2 at 48^3
    mps = [(0, 0, 0), (2, 0, 2), (1, 1, 2)]
    res = api.bispectrum_sugiyama(cat, n=48, box=box, kbins=kb, multipoles=mps, shot=True, precision="mixed")
    spec = _spec(48, box, (0.0, 0.0, 1.0))
    orc = OS.bispectrum_sugiyama(spec, cat, None, kb, mps, shot=True)
    cnt = orc["counts"]
    assert cnt[0] == 0 and cnt[1] == 0   # |q| < k_f holds only the excluded DC mode
    np.testing.assert_array_equal(res["nmodes"], cnt)
    empty = (cnt[:, None] * cnt[None, :]) == 0
    scale = np.abs(orc["B"][(0, 0, 0)]) + np.abs(orc["shot"][(0, 0, 0)])
    for mp in mps:
        assert np.all(res["B"][mp][empty] == 0) and np.all(res["shot"][mp][empty] == 0), mp
        full = ~empty
        e = np.abs(res["B"][mp] + res["shot"][mp] - orc["B"][mp])[full] / np.maximum(np.abs(orc["B"][mp]), scale)[full]
        assert np.max(e) < 1e-4, ("raw", mp, np.max(e))
        e = np.abs(res["shot"][mp] - orc["shot"][mp])[full] / np.maximum(np.abs(orc["shot"][mp]), scale)[full]
        assert np.max(e) < 1e-4, ("shot", mp, np.max(e))


def test_cached_triangle_counts_survive_a_larger_call(api):
    """N_T is cached per geometry; a TripoSH call with more bins grows the shared workspaces, after
    which the smaller bispectrum must still report the same counts (a reallocated workspace drops
    its cached contents)."""
    cat = make_periodic_catalog(20000, 300.0, 32, seed=99)
    kb = (0.02, 0.02, 5)
    first = api.bispectrum(cat, n=32, box=300.0, kbins=kb, scoc_ells=(0,), tripo_ells=(0,), precision="fp64")
    kf = 2 * np.pi / 300.0
    api.bispectrum_sugiyama(cat, n=32, box=300.0, kbins=(0.0, 0.3 * kf, 24), multipoles=[(0, 0, 0)],
                            precision="fp64")
    again = api.bispectrum(cat, n=32, box=300.0, kbins=kb, scoc_ells=(0,), tripo_ells=(0,), precision="fp64")
    np.testing.assert_array_equal(again["NT"], first["NT"])
    np.testing.assert_array_equal(again["B"][0], first["B"][0])


ENDPOINT = [(0, 0, 0), (2, 0, 2), (0, 2, 2), (1, 1, 0), (1, 1, 2), (2, 2, 2), (1, 0, 1), (2, 1, 1), (2, 1, 3)]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_survey_endpoint_line_of_sight(api, prec, tol):
    """Survey geometry with the line of sight to each grid point: G_L^M for every M from the
    y_L^M-weighted transforms, F_l^m in the catalogue frame and the full m1 + m2 + M = 0 sum,
    including odd L (l1 + l2 + L even), against the oracle's sum over every sub-configuration."""
    from synthetic import make_survey_catalogs

    box = 600.0
    g, r, origin = make_survey_catalogs(20000, 200000, box, 800.0, 32, seed=87, fkp_p0=1e4)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 4)
    spec = dict(n=32, box=box, origin=tuple(origin), assign=3, interlace=1, los="endpoint",
                observer=(0.0, 0.0, 0.0), periodic=0)
    res = api.bispectrum_sugiyama(g, n=32, box=box, kbins=kb, multipoles=ENDPOINT, los_dir=None, precision=prec,
                                  origin=origin, randoms=r)
    orc, cnt = _oracle(spec, g, r, kb, ENDPOINT)
    _check(res, orc, cnt, ENDPOINT, tol)
    # the odd-L multipoles measured are not all zero
    scale = np.abs(np.real(orc[(0, 0, 0)]))
    assert np.max(np.abs(np.imag(orc[(1, 0, 1)])) / scale) > 1e-4


def test_endpoint_rejects_shot_noise(api):
    from paper_2605_04864_gb300 import binding as B
    from synthetic import make_survey_catalogs

    g, r, origin = make_survey_catalogs(2000, 20000, 600.0, 900.0, 16, seed=89)
    with pytest.raises(B.NpcError) as ei:
        api.bispectrum_sugiyama(g, n=32, box=600.0, kbins=(0.03, 0.02, 3), multipoles=[(0, 0, 0)], los_dir=None,
                                origin=origin, randoms=r, shot=True)
    assert ei.value.status == 4


@pytest.mark.slow
def test_full_size_256_sample(api):
    """The 256^3 bispectrum workload (1e6 particles, 19 bins, line of sight z): TripoSH B_000 and
    B_202 on all 361 (k1, k2) pairs against the oracle's every-sub-configuration sum (stored by
    tests/golden/make_full_size.py, re-evaluated here if this machine generates different input
    bytes); tolerance 1e-4 of the B_000 scale of the pair."""
    from synthetic import fingerprint

    gm = golden_module()
    w, cat, spec = gm.bispec_inputs()

    def live():
        res, cnt = gm.sugiyama_oracle(w, cat, spec)
        return {"nmodes": cnt, "B_raw": {"".join(str(v) for v in mp): res[mp] for mp in gm.SUGIYAMA_MULTIPOLES}}

    orc, _ = stored_or_live(gm.SUGIYAMA_FILE, fingerprint(cat), live)
    kb = (w["kmin"], w["dk"], w["nbins"])
    mps = list(gm.SUGIYAMA_MULTIPOLES)
    res = api.bispectrum_sugiyama(cat, n=256, box=w["box"], kbins=kb, multipoles=mps, precision="mixed")
    np.testing.assert_array_equal(res["nmodes"], np.asarray(orc["nmodes"]))
    scale = np.abs(np.asarray(orc["B_raw"]["000"]))
    for mp in mps:
        want = np.asarray(orc["B_raw"]["".join(str(v) for v in mp)])
        e = np.abs(res["B"][mp] - want) / np.maximum(np.abs(want), scale)
        assert np.max(e) < 1e-4, (mp, np.max(e))
