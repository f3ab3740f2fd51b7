"""GPU parity: npc_cross_power_multipoles (through the C ABI) against the FP64 oracle."""
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
