"""GPU parity: npc_bispectrum (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

from helpers import ensure_built, golden_module, stored_or_live
from oracle import bispec as OB
from synthetic import make_periodic_catalog, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    ensure_built()
    from paper_2605_04864_gb300 import api as A

    return A


def _spec(n, box, assign=3, interlace=1):
    return dict(n=n, box=box, origin=(0.0, 0.0, 0.0), assign=assign, interlace=interlace, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=1)


def _check(res, orc, tol):
    """Error relative to the monopole + shot-noise scale of the same triangle / pair."""
    np.testing.assert_array_equal(res["tri"], orc["tri"])
    np.testing.assert_allclose(res["NT"], orc["NT"], rtol=max(tol, 1e-9) * 10, atol=1e-6)
    # the oracle reports raw estimates and the analytic shot noise separately; the library
    # reports the subtracted estimate and the shot noise
    scale_t = np.abs(orc["B"][0]) + np.abs(orc["shot_B"][0])
    for l in orc["B"]:
        raw_g = res["B"][l] + res["shot_B"][l]
        raw_o = orc["B"][l]
        e = np.abs(raw_g - raw_o) / np.maximum(np.abs(raw_o), scale_t)
        assert np.max(e) < tol, ("B", l, np.max(e))
        e = np.abs(res["shot_B"][l] - orc["shot_B"][l]) / np.maximum(np.abs(orc["shot_B"][l]), scale_t)
        assert np.max(e) < tol, ("shot_B", l, np.max(e))
    scale_p = np.abs(orc["BB"][0]) + np.abs(orc["shot_BB"][0])
    for l in orc["BB"]:
        raw_g = res["BB"][l] + res["shot_BB"][l]
        raw_o = orc["BB"][l]
        e = np.abs(raw_g - raw_o) / np.maximum(np.abs(raw_o), scale_p)
        assert np.max(e) < tol, ("BB", l, np.max(e))
        e = np.abs(res["shot_BB"][l] - orc["shot_BB"][l]) / np.maximum(np.abs(orc["shot_BB"][l]), scale_p)
        assert np.max(e) < tol, ("shot_BB", l, np.max(e))


@pytest.mark.parametrize("assign,interlace", [(3, 1), (2, 0)])
def test_fp64_small_periodic(api, assign, interlace):
    cat = make_periodic_catalog(20000, 300.0, 32, seed=41)
    kb = (0.02, 0.02, 5)   # k_max = 0.12 < k_N/2 = 0.168
    res = api.bispectrum(cat, n=32, box=300.0, kbins=kb, assign=assign, interlace=interlace, precision="fp64")
    orc = OB.bispectrum(_spec(32, 300.0, assign, interlace), cat, None, kb, (0, 2), (0, 2), shot=True)
    _check(res, orc, 1e-10)


@pytest.mark.parametrize("n,prec,tol", [(48, "fp64", 1e-10), (96, "mixed", 1e-4)])
def test_radix3_meshes(api, n, prec, tol):
    """Meshes of 3 * 2^k cells through the whole bispectrum path (forward, shell inverses, triple
    products, shot noise)."""
    box = 300.0 * n / 32
    cat = make_periodic_catalog(30000, box, 32, seed=43 + n)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 5)   # k_max = 9.5 k_f < k_N/2 = n k_f/4
    res = api.bispectrum(cat, n=n, box=box, kbins=kb, precision=prec)
    orc = OB.bispectrum(_spec(n, box), cat, None, kb, (0, 2), (0, 2), shot=True)
    _check(res, orc, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_survey_monopoles(api, prec, tol):
    """Survey geometry (FKP field with randoms, no line of sight needed): B_0 and B_000 with their
    analytic shot noise, which then carry the randoms' alpha^3 self term."""
    from synthetic import make_survey_catalogs

    box = 600.0
    g, r, origin = make_survey_catalogs(20000, 200000, box, 900.0, 32, seed=71, fkp_p0=1e4)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 4)   # k_max = 8 k_f = k_N/2 at 32^3
    res = api.bispectrum(g, n=32, box=box, kbins=(kb[0], kb[1], 3), scoc_ells=(0,), tripo_ells=(0,),
                         precision=prec, origin=origin, randoms=r)
    spec = dict(n=32, box=box, origin=tuple(origin), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=0)
    orc = OB.bispectrum(spec, g, r, (kb[0], kb[1], 3), (0,), (0,), shot=True)
    _check(res, orc, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_fft_method_shot_noise_periodic(api, prec, tol):
    """shot = "fft": the exact two-object triplet sums (B_0, B_2) against the oracle's explicit
    enumeration; the raw estimates and the compressed estimator's analytic shot noise are unchanged."""
    cat = make_periodic_catalog(20000, 300.0, 32, seed=47)
    kb = (0.02, 0.02, 5)
    res = api.bispectrum(cat, n=32, box=300.0, kbins=kb, precision=prec, shot="fft")
    orc = OB.bispectrum(_spec(32, 300.0), cat, None, kb, (0, 2), (0, 2), shot="fft")
    scale_t = np.abs(orc["B"][0]) + np.abs(orc["shot_B_fft"][0])
    for l in (0, 2):
        raw_g = res["B"][l] + res["shot_B"][l]
        e = np.abs(raw_g - orc["B"][l]) / np.maximum(np.abs(orc["B"][l]), scale_t)
        assert np.max(e) < tol, ("B", l, np.max(e))
        e = np.abs(res["shot_B"][l] - orc["shot_B_fft"][l]) / np.maximum(np.abs(orc["shot_B_fft"][l]), scale_t)
        assert np.max(e) < tol, ("shot_B_fft", l, np.max(e))
    scale_p = np.abs(orc["BB"][0]) + np.abs(orc["shot_BB_fft"][0])
    for l in (0, 2):
        e = np.abs(res["shot_BB"][l] - orc["shot_BB_fft"][l]) / np.maximum(np.abs(orc["shot_BB_fft"][l]), scale_p)
        assert np.max(e) < tol, ("shot_BB_fft", l, np.max(e))
    # the exact and thin-shell forms estimate the same noise: close for the monopole, not equal
    d = np.abs(orc["shot_B_fft"][0] - orc["shot_B"][0]) / np.abs(orc["shot_B"][0])
    assert 0 < np.max(d) < 0.2


def test_fft_method_shot_noise_survey_monopole(api):
    """Survey geometry: the FFT-method shot noise of B_0 with randoms (alpha-weighted N-field)."""
    from synthetic import make_survey_catalogs

    box = 600.0
    g, r, origin = make_survey_catalogs(20000, 200000, box, 900.0, 32, seed=73, fkp_p0=1e4)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 3)
    res = api.bispectrum(g, n=32, box=box, kbins=kb, scoc_ells=(0,), tripo_ells=(0,), precision="fp64",
                         origin=origin, randoms=r, shot="fft")
    spec = dict(n=32, box=box, origin=tuple(origin), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=0)
    orc = OB.bispectrum(spec, g, r, kb, (0,), (0,), shot="fft")
    scale = np.abs(orc["B"][0]) + np.abs(orc["shot_B_fft"][0])
    e = np.abs(res["shot_B"][0] - orc["shot_B_fft"][0]) / np.maximum(np.abs(orc["shot_B_fft"][0]), scale)
    assert np.max(e) < 1e-10
    scale = np.abs(orc["BB"][0]) + np.abs(orc["shot_BB_fft"][0])
    e = np.abs(res["shot_BB"][0] - orc["shot_BB_fft"][0]) / np.maximum(np.abs(orc["shot_BB_fft"][0]), scale)
    assert np.max(e) < 1e-10


@pytest.mark.parametrize("assign,interlace,prec,tol", [(3, 1, "fp64", 1e-10), (2, 0, "fp64", 1e-10),
                                                      (3, 1, "mixed", 1e-4)])
def test_survey_l2_endpoint_line_of_sight(api, assign, interlace, prec, tol):
    """Survey geometry with the line of sight to each grid point: Yamamoto X_2 (Y_2m-weighted
    transforms), B_0, B_2, B_000, B_202 and their analytic shot noise with the survey self term."""
    from synthetic import make_survey_catalogs

    box = 600.0
    g, r, origin = make_survey_catalogs(20000, 200000, box, 900.0, 32, seed=75, fkp_p0=1e4)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 4)   # k_max = 8 k_f = k_N/2 at 32^3
    res = api.bispectrum(g, n=32, box=box, kbins=kb, assign=assign, interlace=interlace, precision=prec,
                         origin=origin, randoms=r, los_dir=None, observer=(0.0, 0.0, 0.0))
    spec = dict(n=32, box=box, origin=tuple(origin), assign=assign, interlace=interlace, los="endpoint",
                observer=(0.0, 0.0, 0.0), periodic=0)
    orc = OB.bispectrum(spec, g, r, kb, (0, 2), (0, 2), shot=True)
    _check(res, orc, tol)


def _check_odd(res, orc, ells, tol):
    """Odd multipoles (raw, imaginary part) against the oracle, relative to the raw monopole scale of
    the same triangle; their reported shot noise is zero."""
    np.testing.assert_array_equal(res["tri"], orc["tri"])
    scale = np.abs(res["B"][0] + res["shot_B"][0])
    for l in ells:
        e = np.abs(res["B"][l] - orc["B"][l]) / np.maximum(np.abs(orc["B"][l]), scale)
        assert np.max(e) < tol, (l, np.max(e))
        assert np.all(res["shot_B"][l] == 0)
    assert max(np.max(np.abs(orc["B"][l]) / scale) for l in ells) > 1e-4   # the odd parts are not all zero


@pytest.mark.parametrize("assign,interlace,prec,tol", [(3, 1, "fp64", 1e-10), (2, 0, "fp64", 1e-10),
                                                      (3, 1, "mixed", 1e-4)])
def test_survey_odd_multipoles_endpoint_line_of_sight(api, assign, interlace, prec, tol):
    """Survey geometry with the line of sight to each grid point: B_1 and B_3 (Yamamoto X_1, X_3 from
    the Y_1m- and Y_3m-weighted transforms, imaginary part of the closure sum), requested together
    with B_0, B_2 and the compressed multipoles, against the oracle's odd multipoles."""
    from synthetic import make_survey_catalogs

    box = 600.0
    g, r, origin = make_survey_catalogs(20000, 200000, box, 700.0, 32, seed=79, fkp_p0=1e4)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 4)
    res = api.bispectrum(g, n=32, box=box, kbins=kb, assign=assign, interlace=interlace, precision=prec,
                         origin=origin, randoms=r, los_dir=None, observer=(0.0, 0.0, 0.0),
                         scoc_ells=(0, 1, 2, 3), tripo_ells=(0, 2))
    spec = dict(n=32, box=box, origin=tuple(origin), assign=assign, interlace=interlace, los="endpoint",
                observer=(0.0, 0.0, 0.0), periodic=0)
    orc = OB.odd_multipoles(spec, g, r, kb, (1, 3))
    _check_odd(res, orc, (1, 3), tol)
    even = OB.bispectrum(spec, g, r, kb, (0, 2), (0, 2), shot=True)
    _check(dict(res, B={l: res["B"][l] for l in (0, 2)}, shot_B={l: res["shot_B"][l] for l in (0, 2)}), even, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_odd_multipoles_global_line_of_sight(api, prec, tol):
    """B_1 alone and B_1, B_3 with B_0, survey geometry with a tilted global line of sight
    (X_l = L_l(qhat . los) X_0), against the oracle."""
    from synthetic import make_survey_catalogs

    box = 600.0
    los = (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)
    g, r, origin = make_survey_catalogs(20000, 200000, box, 800.0, 32, seed=83, fkp_p0=1e4)
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 4)
    spec = dict(n=32, box=box, origin=tuple(origin), assign=3, interlace=1, los="global", los_dir=los, periodic=0)
    orc = OB.odd_multipoles(spec, g, r, kb, (1, 3))
    res = api.bispectrum(g, n=32, box=box, kbins=kb, precision=prec, origin=origin, randoms=r, los_dir=los,
                         scoc_ells=(0, 1, 3), tripo_ells=(), shot=True)
    _check_odd(res, orc, (1, 3), tol)
    one = api.bispectrum(g, n=32, box=box, kbins=kb, precision=prec, origin=origin, randoms=r, los_dir=los,
                         scoc_ells=(0, 1), tripo_ells=(), shot=False)
    scale = np.abs(res["B"][0] + res["shot_B"][0])
    assert np.max(np.abs(one["B"][1] - orc["B"][1]) / np.maximum(np.abs(orc["B"][1]), scale)) < tol


def test_mixed_19_bins_805_triangles_128(api):
    """The 19-bin / 805-triangle layout of the 256^3 workload on a 128^3 mesh of the same box
    (k_max = 0.2 = k_N/2), float32 transforms: <= 1e-4."""
    w = workload("bispec_256")
    cat = make_periodic_catalog(w["n_gal"] // 8, w["box"], 128, seed=w["seed"])
    kb = (w["kmin"], w["dk"], w["nbins"])
    res = api.bispectrum(cat, n=128, box=w["box"], kbins=kb, precision="mixed")
    assert res["tri"].shape == (805, 3)
    orc = OB.bispectrum(_spec(128, w["box"]), cat, None, kb, (0, 2), (0, 2), shot=True)
    _check(res, orc, 1e-4)


def test_subsets_and_repeat(api):
    cat = make_periodic_catalog(30000, 400.0, 32, seed=5)
    kb = (0.015, 0.025, 4)
    a = api.bispectrum(cat, n=64, box=400.0, kbins=kb, scoc_ells=(0,), tripo_ells=(2,), shot=False, precision="fp64")
    b = api.bispectrum(cat, n=64, box=400.0, kbins=kb, scoc_ells=(0,), tripo_ells=(2,), shot=False, precision="fp64")
    np.testing.assert_array_equal(a["B"][0], b["B"][0])
    orc = OB.bispectrum(_spec(64, 400.0), cat, None, kb, (0,), (2,), shot=False)
    scale = np.abs(orc["B"][0])
    assert np.max(np.abs(a["B"][0] - orc["B"][0]) / scale.max()) < 1e-10
    assert np.max(np.abs(a["BB"][2] - orc["BB"][2]) / np.abs(orc["BB"][2]).max()) < 1e-10
    assert np.all(a["shot_B"][0] == 0)


def test_bispectrum_rejects(api):
    from paper_2605_04864_gb300 import binding as B

    cat = make_periodic_catalog(1000, 300.0, 16, seed=2)
    with pytest.raises(B.NpcError) as ei:        # k_max beyond k_N/2
        api.bispectrum(cat, n=32, box=300.0, kbins=(0.02, 0.05, 5))
    assert ei.value.status == 4
    with pytest.raises(B.NpcError) as ei:        # multipole beyond l = 3
        api.bispectrum(cat, n=32, box=300.0, kbins=(0.02, 0.02, 4), scoc_ells=(4,))
    assert ei.value.status == 1
    with pytest.raises(B.NpcError) as ei:        # compressed odd multipole
        api.bispectrum(cat, n=32, box=300.0, kbins=(0.02, 0.02, 4), tripo_ells=(1,))
    assert ei.value.status == 1
    from synthetic import make_survey_catalogs

    g, r, origin = make_survey_catalogs(2000, 20000, 600.0, 900.0, 16, seed=77)
    with pytest.raises(B.NpcError) as ei:        # FFT-method l = 2 shot noise with the endpoint line of sight
        api.bispectrum(g, n=32, box=600.0, kbins=(0.03, 0.02, 3), origin=origin, randoms=r, los_dir=None,
                       shot="fft")
    assert ei.value.status == 4


def test_tensor_core_paths_agree(api):
    """The tcgen05 triple products (f16 hi + lo split after exact power-of-two scales, TMEM
    accumulators) against the warp-level mma.sync path (tf32 hi + lo) on the same shell fields:
    both carry about 21 bits per product, so they agree far inside the 1e-4 bispectrum tolerance;
    N_T (integer counts) is identical.  The statistics show which path ran: the tcgen05 path issues
    two f16 products per k step (hi and lo rows against interleaved hi and lo columns), mma.sync three
    tf32 products."""
    cat = make_periodic_catalog(60000, 600.0, 32, seed=45)
    kf = 2 * np.pi / 600.0
    kb = (2 * kf, 1.5 * kf, 7)
    path = api.get_option("tcgen05_triple")
    try:
        api.set_option("tcgen05_triple", 1)
        api.bispectrum(cat, n=64, box=600.0, kbins=kb, precision="mixed")   # N_T counted and cached here
        a = api.bispectrum(cat, n=64, box=600.0, kbins=kb, precision="mixed")
        st_a = api.last_stats()
        api.set_option("tcgen05_triple", 0)
        b = api.bispectrum(cat, n=64, box=600.0, kbins=kb, precision="mixed")
        st_b = api.last_stats()
    finally:
        api.set_option("tcgen05_triple", path)
    assert st_a["contraction_launches"] >= 1 and st_a["contraction_flops"] == st_b["contraction_flops"]
    # 7 bins: 56 rows x 9 columns of B_0, B_2, B_000, B_202; the tcgen05 plan puts the 14 single
    # fields F_0,i, F_2,i on the N side (N = 32) against the 28 products F_0,j F_0,k and the 14
    # products F_0,j G (one 128-row tile)
    assert st_a["contraction_issued_flops"] != st_b["contraction_issued_flops"]
    np.testing.assert_array_equal(a["NT"], b["NT"])
    scale = np.abs(b["B"][0] + b["shot_B"][0]) + np.abs(b["shot_B"][0])
    for l in (0, 2):
        assert np.max(np.abs(a["B"][l] - b["B"][l]) / scale) < 1e-5, l
    sp = np.abs(b["BB"][0] + b["shot_BB"][0]) + np.abs(b["shot_BB"][0])
    for l in (0, 2):
        assert np.max(np.abs(a["BB"][l] - b["BB"][l]) / sp) < 1e-5, l


def test_bounded_wait_timeout_is_reported_and_the_context_recovers(api):
    """A wait bound far below the work's latency makes the triple-product kernel's waits give up:
    the call returns NPC_ERR_TIMEOUT (no fault, no hang), and with the default bound the next call
    on the same context gives the same result as before."""
    from paper_2605_04864_gb300 import binding as B

    cat = make_periodic_catalog(30000, 400.0, 32, seed=47)
    kb = (0.02, 0.02, 6)
    path = api.get_option("tcgen05_triple")
    api.set_option("tcgen05_triple", 1)   # the bounded waits are the tensor-core kernel's
    try:
        ref = api.bispectrum(cat, n=64, box=400.0, kbins=kb, precision="mixed")
        try:
            api.set_wait_limit(1)
            with pytest.raises(B.NpcError) as ei:
                api.bispectrum(cat, n=64, box=400.0, kbins=kb, precision="mixed")
            assert ei.value.status == 5
        finally:
            api.set_wait_limit(0)
        api.device_status()
        again = api.bispectrum(cat, n=64, box=400.0, kbins=kb, precision="mixed")
    finally:
        api.set_option("tcgen05_triple", path)
    for l in (0, 2):
        np.testing.assert_array_equal(again["B"][l], ref["B"][l])
    np.testing.assert_array_equal(again["NT"], ref["NT"])


@pytest.mark.slow
def test_full_size_256_all_triangles(api):
    """The bench workload in full (256^3, 1e6 particles, 19 bins): all 805 closed triangles of B_0,
    B_2 and N_T and all 190 pairs of B_000, B_202, with their analytic shot noise, against the
    oracle (stored by tests/golden/make_full_size.py, re-evaluated here if this machine generates
    different input bytes).  Float32 shell fields: the rounded triangle count can miss the exact
    integer by about 1e-5 of itself for the largest shells; B within 1e-4 of the monopole scale."""
    from synthetic import fingerprint

    gm = golden_module()
    w, cat, spec = gm.bispec_inputs()

    def live():
        o = gm.bispec_oracle(w, cat, spec)
        return {"tri": o["tri"], "pairs": o["pairs"], "NT": o["NT"],
                "B_raw": {str(l): v for l, v in o["B"].items()}, "shot_B": {str(l): v for l, v in o["shot_B"].items()},
                "BB_raw": {str(l): v for l, v in o["BB"].items()},
                "shot_BB": {str(l): v for l, v in o["shot_BB"].items()}}

    orc, _ = stored_or_live(gm.BISPEC_FILE, fingerprint(cat), live)
    kb = (w["kmin"], w["dk"], w["nbins"])
    res = api.bispectrum(cat, n=256, box=w["box"], kbins=kb, precision="mixed")
    np.testing.assert_array_equal(res["tri"], np.asarray(orc["tri"]))
    assert res["tri"].shape == (805, 3)
    np.testing.assert_allclose(res["NT"], np.asarray(orc["NT"]), rtol=5e-5, atol=1e-6)
    b0 = np.asarray(orc["B_raw"]["0"])
    scale_t = np.abs(b0) + np.abs(np.asarray(orc["shot_B"]["0"]))
    for l in (0, 2):
        raw_o = np.asarray(orc["B_raw"][str(l)])
        e = np.abs(res["B"][l] + res["shot_B"][l] - raw_o) / np.maximum(np.abs(raw_o), scale_t)
        assert np.max(e) < 1e-4, ("B", l, np.max(e))
        sh = np.asarray(orc["shot_B"][str(l)])
        e = np.abs(res["shot_B"][l] - sh) / np.maximum(np.abs(sh), scale_t)
        assert np.max(e) < 1e-4, ("shot_B", l, np.max(e))
    scale_p = np.abs(np.asarray(orc["BB_raw"]["0"])) + np.abs(np.asarray(orc["shot_BB"]["0"]))
    for l in (0, 2):
        raw_o = np.asarray(orc["BB_raw"][str(l)])
        e = np.abs(res["BB"][l] + res["shot_BB"][l] - raw_o) / np.maximum(np.abs(raw_o), scale_p)
        assert np.max(e) < 1e-4, ("BB", l, np.max(e))
        sh = np.asarray(orc["shot_BB"][str(l)])
        e = np.abs(res["shot_BB"][l] - sh) / np.maximum(np.abs(sh), scale_p)
        assert np.max(e) < 1e-4, ("shot_BB", l, np.max(e))


def _shape_case(api, case):
    """One bispectrum call of the launch shape `case`; returns the result dictionary."""
    from synthetic import make_survey_catalogs

    box = 600.0
    kf = 2 * np.pi / box
    if case == "periodic_24_bins":   # the most bins: 348 product rows, two row groups over the CTAs
        cat = make_periodic_catalog(200000, box, 48, seed=61)
        return api.bispectrum(cat, n=192, box=box, kbins=(2 * kf, 1.5 * kf, 24), precision="mixed")
    if case == "fft_method_shot":    # the shot-noise products of the FFT method (shot = 2)
        cat = make_periodic_catalog(60000, box, 32, seed=62)
        return api.bispectrum(cat, n=64, box=box, kbins=(2 * kf, 1.5 * kf, 7), shot=2, precision="mixed")
    if case == "survey_odd":         # four row families: F_0, F_2, F_1, F_3 on the first leg
        g, r, origin = make_survey_catalogs(20000, 200000, box, 700.0, 32, seed=63, fkp_p0=1e4)
        return api.bispectrum(g, n=32, box=box, kbins=(2 * kf, 1.5 * kf, 4), origin=origin, randoms=r, los_dir=None,
                              scoc_ells=(0, 1, 2, 3), tripo_ells=(0, 2), precision="mixed")
    # three tracers of one density field (one seed, different numbers of objects: a cross
    # bispectrum with signal), every product of two different catalogues' fields
    cats = [make_periodic_catalog(nn, box, 32, seed=64) for nn in (30000, 20000, 40000)]
    return api.cross_bispectrum([(c, None) for c in cats], n=64, box=box, kbins=(2 * kf, 1.5 * kf, 7),
                                scoc_ells=(0, 2), tripo_ells=(0, 2), precision="mixed")


@pytest.mark.parametrize("case", ["periodic_24_bins", "fft_method_shot", "survey_odd", "cross_three_tracers"])
def test_tensor_core_paths_agree_over_launch_shapes(api, case):
    """The tcgen05 plan (which two fields form the product rows, row tiles per CTA and row groups,
    stages in flight) against the mma.sync path on launch shapes beyond the plain 7-bin case: the
    largest bin count, the FFT-method shot-noise products, four row families of odd multipoles and
    three different tracers.  Each form carries its own float32 accumulation error (1e-5 to 3e-5 of
    the monopole scale against the FP64 oracle on a 128^3 shell grid), so they agree within half the
    1e-4 tolerance; the statistics show that the tcgen05 path ran."""
    path = api.get_option("tcgen05_triple")
    try:
        api.set_option("tcgen05_triple", 1)
        _shape_case(api, case)   # N_T counted and cached on the first call of a geometry
        a = _shape_case(api, case)
        st_a = api.last_stats()
        api.set_option("tcgen05_triple", 0)
        b = _shape_case(api, case)
        st_b = api.last_stats()
    finally:
        api.set_option("tcgen05_triple", path)
    assert st_a["contraction_flops"] == st_b["contraction_flops"] > 0
    assert st_a["contraction_issued_flops"] != st_b["contraction_issued_flops"]
    np.testing.assert_array_equal(a["tri"], b["tri"])
    if "NT" in b:
        np.testing.assert_allclose(a["NT"], b["NT"], rtol=1e-6)
    for key, skey in (("B", "shot_B"), ("BB", "shot_BB")):
        if key not in b:
            continue
        shot = b.get(skey, {})
        scale = np.abs(b[key][0] + shot.get(0, 0.0)) + np.abs(shot.get(0, 0.0))
        # triangles without a closed triplet (N_T = 0: possible with bins of half a fundamental
        # mode) are undefined on both paths
        ok = np.isfinite(scale) & (scale > 0)
        for l in b[key]:
            np.testing.assert_array_equal(np.isfinite(a[key][l]), np.isfinite(b[key][l]))
            err = np.max(np.abs(a[key][l] - b[key][l])[ok] / scale[ok])
            assert err < 5e-5, (key, l, err)
            if l in shot:
                err = np.max(np.abs(a[skey][l] - shot[l])[ok] / scale[ok])
                assert err < 5e-5, (skey, l, err)
    assert ok.sum() > 0.9 * ok.size
