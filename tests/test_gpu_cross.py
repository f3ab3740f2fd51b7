"""GPU parity: npc_cross_power_multipoles and npc_cross_bispectrum (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

from helpers import ensure_built, p_error
from oracle import power as P
from synthetic import make_periodic_catalog, make_survey_catalogs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    ensure_built()
    from paper_2605_04864_gb300 import api as A

    return A


def _two_tracers(seed):
    """Two survey tracers of one density field (same generator seed): different densities, FKP
    weights and randoms, so the cross spectrum carries the common clustering."""
    ga, ra, origin = make_survey_catalogs(6000, 60000, 800.0, 1300.0, 24, seed=seed, fkp_p0=1e4)
    gb, rb, _ = make_survey_catalogs(3000, 45000, 800.0, 1300.0, 24, seed=seed, fkp_p0=2e4)
    return ga, ra, gb, rb, origin


def _scale(orc):
    """|P_0^AB| plus the geometric mean of the tracers' shot levels: the size of F_0^A F_l^B*."""
    return np.abs(orc["P"][0]) + np.sqrt(orc["scalars_a"]["N0"] * orc["scalars_b"]["N0"])


@pytest.mark.parametrize("n,assign,interlace,prec,tol", [(32, 2, 0, "fp64", 1e-12), (48, 3, 1, "fp64", 1e-12),
                                                         (64, 3, 1, "mixed", 1e-5)])
def test_survey_cross_against_oracle(api, n, assign, interlace, prec, tol):
    ga, ra, gb, rb, origin = _two_tracers(101 + n)
    kb = (0.0, 0.02, 5)
    res = api.cross_power_multipoles(ga, ra, gb, rb, n=n, box=800.0, origin=origin, assign=assign,
                                     interlace=interlace, kbins=kb, ells=(0, 2, 4), precision=prec)
    spec = dict(n=n, box=800.0, origin=tuple(origin), assign=assign, interlace=interlace, los="endpoint",
                observer=(0.0, 0.0, 0.0))
    orc = P.cross_power_multipoles(spec, ga, ra, gb, rb, kb, (0, 2, 4))
    np.testing.assert_array_equal(res["nmodes"], orc["nmodes"])
    scale = _scale(orc)
    for l in (0, 2, 4):
        e = p_error(res["P"][l], orc["P"][l], scale)
        assert np.max(e) < tol, (l, np.max(e))
    sc = res["scalars"]
    assert sc["I22_ab"] == pytest.approx(orc["I22"], rel=1e-12)
    assert sc["alpha_a"] == pytest.approx(orc["scalars_a"]["alpha"], rel=1e-12)
    assert sc["alpha_b"] == pytest.approx(orc["scalars_b"]["alpha"], rel=1e-12)


def test_periodic_global_los_cross_is_symmetric(api):
    a = make_periodic_catalog(20000, 500.0, 32, seed=111)
    b = make_periodic_catalog(12000, 500.0, 32, seed=111)   # same density field, other objects
    kb = (0.0, 0.02, 8)
    kw = dict(n=64, box=500.0, kbins=kb, ells=(0, 2, 4), precision="fp64", los_dir=(0.0, 0.0, 1.0))
    ab = api.cross_power_multipoles(a, None, b, None, **kw)
    ba = api.cross_power_multipoles(b, None, a, None, **kw)
    spec = dict(n=64, box=500.0, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=1)
    orc = P.cross_power_multipoles(spec, a, None, b, None, kb, (0, 2, 4))
    scale = _scale(orc)
    for l in (0, 2, 4):
        assert np.max(p_error(ab["P"][l], orc["P"][l], scale)) < 1e-12
        assert np.max(p_error(ba["P"][l], orc["P"][l], scale)) < 1e-12


def test_cross_with_itself_matches_auto(api):
    """Mixed precision: the cross spectrum of a tracer with itself is its auto spectrum plus N_0."""
    g, r, origin = make_survey_catalogs(20000, 200000, 1000.0, 1500.0, 32, seed=121, fkp_p0=1e4)
    kb = (0.0, 0.01, 12)
    kw = dict(n=96, box=1000.0, origin=origin, kbins=kb, ells=(0, 2, 4), precision="mixed")
    cross = api.cross_power_multipoles(g, r, g, r, **kw)
    auto = api.power_multipoles(g, r, **kw)
    n0 = auto["scalars"]["N0"]
    scale = np.abs(auto["P"][0]) + n0
    for l in (0, 2, 4):
        want = auto["P"][l] + (n0 if l == 0 else 0.0) * (auto["nmodes"] > 0)
        assert np.max(p_error(cross["P"][l], want, scale)) < 1e-5, l


def test_cross_rejects(api):
    a = make_periodic_catalog(1000, 500.0, 16, seed=131)
    g, r, origin = make_survey_catalogs(1000, 10000, 500.0, 900.0, 16, seed=132, fkp_p0=None)
    with pytest.raises(RuntimeError):
        api.cross_power_multipoles(a, None, g, r, n=32, box=500.0, kbins=(0.0, 0.02, 4))   # one randoms only
    with pytest.raises(RuntimeError):
        api.cross_power_multipoles(a, None, a, None, n=32, box=500.0, kbins=(0.0, 0.02, 4), ells=(5,))


def test_odd_cross_of_a_shifted_copy(api):
    """Cross multipoles of a tracer and its copy moved two cells along the line of sight: the odd
    P_1, P_3 (imaginary part) and the even ones against the oracle, periodic, global LOS."""
    from types import SimpleNamespace

    box, n = 500.0, 32
    a = make_periodic_catalog(30000, box, 32, seed=141, dtype=np.float64)
    b = SimpleNamespace(pos=a.pos.copy(), w=a.w, nbar=a.nbar)
    b.pos[:, 2] = np.mod(b.pos[:, 2] + 2 * box / n, box)
    kb = (0.0, 0.02, 8)
    res = api.cross_power_multipoles(a, None, b, None, n=n, box=box, kbins=kb, ells=(0, 1, 2, 3, 4),
                                     precision="fp64", los_dir=(0.0, 0.0, 1.0))
    spec = dict(n=n, box=box, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=1)
    orc = P.cross_power_multipoles(spec, a, None, b, None, kb, (0, 1, 2, 3, 4))
    scale = _scale(orc)
    for l in (0, 1, 2, 3, 4):
        assert np.max(p_error(res["P"][l], orc["P"][l], scale)) < 1e-12, l
    assert np.max(np.abs(orc["P"][1]) / scale) > 1e-3


def _check_cross_b(res, orc, scoc, tripo, tol):
    np.testing.assert_array_equal(res["tri"], orc["tri"])
    scale = np.abs(orc["B"][0])
    for l in scoc:
        e = np.abs(res["B"][l] - orc["B"][l]) / np.maximum(np.abs(orc["B"][l]), scale)
        assert np.max(e) < tol, ("B", l, np.max(e))
        assert np.all(res["shot_B"][l] == 0)
    sp = np.abs(orc["BB"][0]) if 0 in orc["BB"] else None
    for l in tripo:
        ref = np.abs(orc["BB"][l]) if sp is None else np.maximum(np.abs(orc["BB"][l]), sp)
        e = np.abs(res["BB"][l] - orc["BB"][l]) / ref
        assert np.max(e) < tol, ("BB", l, np.max(e))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_cross_bispectrum_three_periodic_tracers(api, prec, tol):
    """Three different periodic catalogues, tracer t on leg t, global line of sight along z:
    B_0^{123}, B_2^{123} (l on leg 1) and B_000^{123}, B_202^{123} (l on leg 3) against the oracle."""
    from oracle import bispec as OB

    cats = [make_periodic_catalog(n, 300.0, 32, seed=s) for n, s in ((20000, 51), (15000, 52), (25000, 53))]
    kb = (0.02, 0.02, 5)
    spec = dict(n=32, box=300.0, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=1)
    orc = OB.cross_bispectrum(spec, [(c, None) for c in cats], kb, (0, 2), (0, 2))
    res = api.cross_bispectrum([(c, None) for c in cats], n=32, box=300.0, kbins=kb, scoc_ells=(0, 2),
                               tripo_ells=(0, 2), precision=prec)
    _check_cross_b(res, orc, (0, 2), (0, 2), tol)
    np.testing.assert_allclose(res["NT"], orc["NT"], rtol=1e-9, atol=1e-6)


def test_cross_bispectrum_survey_and_equal_tracers(api):
    """Survey geometry with three (data, randoms) pairs and a tilted global line of sight against the
    oracle; and three copies of one catalogue give the auto bispectrum's raw B_0 and B_000."""
    from oracle import bispec as OB

    box = 600.0
    los = (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)
    tr = []
    for s in (61, 62, 63):
        g, r, origin = make_survey_catalogs(15000, 150000, box, 900.0, 32, seed=s, fkp_p0=1e4)
        tr.append((g, r))
    kf = 2 * np.pi / box
    kb = (2 * kf, 1.5 * kf, 4)
    spec = dict(n=32, box=box, origin=tuple(origin), assign=3, interlace=1, los="global", los_dir=los, periodic=0)
    orc = OB.cross_bispectrum(spec, tr, kb, (0, 2), (0,))
    res = api.cross_bispectrum(tr, n=32, box=box, kbins=kb, scoc_ells=(0, 2), tripo_ells=(0,), los_dir=los,
                               origin=origin, precision="fp64")
    _check_cross_b(res, orc, (0, 2), (0,), 1e-10)
    g, r = tr[0]
    same = api.cross_bispectrum([(g, r)] * 3, n=32, box=box, kbins=kb, scoc_ells=(0,), tripo_ells=(0,),
                                los_dir=los, origin=origin, precision="fp64")
    auto = api.bispectrum(g, n=32, box=box, kbins=kb, scoc_ells=(0,), tripo_ells=(0,), shot=False, origin=origin,
                          randoms=r, los_dir=los, precision="fp64")
    np.testing.assert_allclose(same["B"][0], auto["B"][0], rtol=1e-11, atol=0)
    np.testing.assert_allclose(same["BB"][0], auto["BB"][0], rtol=1e-11, atol=0)


def test_cross_bispectrum_rejects(api):
    from paper_2605_04864_gb300 import binding as B

    cats = [make_periodic_catalog(2000, 300.0, 16, seed=s) for s in (1, 2, 3)]
    with pytest.raises(B.NpcError) as ei:       # line of sight to each grid point
        api.cross_bispectrum([(c, None) for c in cats], n=32, box=300.0, kbins=(0.02, 0.02, 4), los_dir=None)
    assert ei.value.status == 4
    with pytest.raises(B.NpcError) as ei:       # odd multipole
        api.cross_bispectrum([(c, None) for c in cats], n=32, box=300.0, kbins=(0.02, 0.02, 4), scoc_ells=(1,))
    assert ei.value.status == 1
