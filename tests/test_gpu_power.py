"""GPU parity: npc_power_multipoles (through the C ABI) against the FP64 oracle."""
import ctypes as C
from types import SimpleNamespace

import numpy as np
import pytest

from helpers import ensure_built, golden_module, p_error, stored_or_live
from oracle import power as P
from synthetic import make_periodic_catalog, make_survey_catalogs, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    ensure_built()
    from paper_2605_04864_gb300 import api as A

    return A


def _oracle(g, r, origin, n, box, assign, interlace, kb, ells, modified=(), los_dir=None):
    spec = dict(n=n, box=box, origin=tuple(origin), assign=assign, interlace=interlace,
                los="global" if los_dir is not None else "endpoint", los_dir=los_dir,
                observer=(0.0, 0.0, 0.0))
    return P.power_multipoles(spec, g, r, kb, ells, modified, method="plain")


def _compare(res, orc, ells, modified, tol):
    scale = np.abs(orc["P"][0]) + orc["scalars"]["N0"] if 0 in orc["P"] else orc["scalars"]["N0"]
    np.testing.assert_array_equal(res["nmodes"], orc["nmodes"])
    np.testing.assert_allclose(res["k_eff"], orc["k_eff"], rtol=1e-6, atol=1e-12)
    worst = 0.0
    for l in ells:
        e = p_error(res["P"][l], orc["P"][l], scale)
        worst = max(worst, float(np.max(e)))
        assert np.max(e) < tol, (l, np.max(e))
    for l in modified:
        e = p_error(res["Pmod"][l], orc["Pmod"][l], scale)
        worst = max(worst, float(np.max(e)))
        assert np.max(e) < tol, ("b", l, np.max(e))
    for k in ("alpha", "I22", "N0"):
        assert res["scalars"][k] == pytest.approx(orc["scalars"][k], rel=1e-12)
    return worst


def test_fp64_plain_64_cic_survey(api):
    """Plain FP64 Yamamoto P_0,2,4: 64^3 CIC, no interlacing, survey geometry, unit weights."""
    w = workload("p024_fp64_64")
    g, r, origin = make_survey_catalogs(w["n_gal"], w["n_ran"], w["box"], w["distance"], w["n_gen"],
                                        seed=w["seed"], fkp_p0=None)
    kb = (w["kmin"], w["dk"], w["nbins"])
    res = api.power_multipoles(g, r, n=64, box=w["box"], origin=origin, assign=2, interlace=0, kbins=kb,
                               ells=(0, 2, 4), precision="fp64")
    orc = _oracle(g, r, origin, 64, w["box"], 2, 0, kb, (0, 2, 4))
    _compare(res, orc, (0, 2, 4), (), 1e-12)
    st = api.last_stats()
    assert st["n_transforms"] == 9 and st["n_r2c_equivalent"] == 15 and st["n_phases"] == 1


@pytest.mark.parametrize("n", [32, 64, 128])
def test_mixed_tsc_interlaced_modified(api, n):
    """P_0,2,4 + P_4b,6b,8b, TSC + interlacing, FKP weights, float32 transforms: <= 1e-5."""
    box = 800.0
    g, r, origin = make_survey_catalogs(40000, 400000, box, 1300.0, 32, seed=31 + n, fkp_p0=1e4)
    kn = np.pi * n / box
    kb = (0.0, 0.01, int(kn / 0.01))
    res = api.power_multipoles(g, r, n=n, box=box, origin=origin, assign=3, interlace=1, kbins=kb,
                               ells=(0, 2, 4), modified=(4, 6, 8), precision="mixed")
    orc = _oracle(g, r, origin, n, box, 3, 1, kb, (0, 2, 4), (4, 6, 8))
    _compare(res, orc, (0, 2, 4), (4, 6, 8), 1e-5)


@pytest.mark.parametrize("n,prec,tol", [(48, "fp64", 1e-12), (96, "mixed", 1e-5), (192, "mixed", 1e-5)])
def test_radix3_meshes(api, n, prec, tol):
    """Meshes of 3 * 2^k cells (48, 96, 192: transforms split into three power-of-two transforms
    and a radix-3 combination), survey geometry, TSC + interlacing, P_0,2,4 + P_4b,6b,8b."""
    box = 900.0
    g, r, origin = make_survey_catalogs(30000, 300000, box, 1400.0, 48, seed=300 + n, fkp_p0=1e4)
    kn = np.pi * n / box
    kb = (0.0, 0.01, int(kn / 0.01))
    res = api.power_multipoles(g, r, n=n, box=box, origin=origin, assign=3, interlace=1, kbins=kb,
                               ells=(0, 2, 4), modified=(4, 6, 8), precision=prec)
    orc = _oracle(g, r, origin, n, box, 3, 1, kb, (0, 2, 4), (4, 6, 8))
    _compare(res, orc, (0, 2, 4), (4, 6, 8), tol)


def test_fp64_ragged_bins_and_subsets(api):
    """Ragged bins (kmin offset, odd dk, partial coverage), a subset of multipoles, float64 input."""
    box = 700.0
    g, r, origin = make_survey_catalogs(9000, 60000, box, 1200.0, 16, seed=77, fkp_p0=5e3,
                                        dtype=np.float64)
    kb = (0.013, 0.017, 7)
    for ells, mods in [((2,), ()), ((0, 4), (4,)), ((4,), (8,))]:
        res = api.power_multipoles(g, r, n=32, box=box, origin=origin, assign=3, interlace=1, kbins=kb,
                                   ells=ells, modified=mods, precision="fp64")
        orc = _oracle(g, r, origin, 32, box, 3, 1, kb, tuple(sorted(set(ells) | {0})), mods)
        _compare(res, orc, ells, mods, 1e-12)


def test_global_los_survey_and_periodic(api):
    box = 500.0
    g, r, origin = make_survey_catalogs(6000, 50000, box, 900.0, 16, seed=5, fkp_p0=1e4)
    kb = (0.0, 0.02, 9)
    res = api.power_multipoles(g, r, n=32, box=box, origin=origin, assign=2, interlace=1, kbins=kb,
                               ells=(0, 2, 4), modified=(4,), precision="fp64", los_dir=(1.0, 1.0, 1.0))
    orc = _oracle(g, r, origin, 32, box, 2, 1, kb, (0, 2, 4), (4,), los_dir=(1.0, 1.0, 1.0))
    _compare(res, orc, (0, 2, 4), (4,), 1e-12)
    assert api.last_stats()["n_transforms"] == 1
    cat = make_periodic_catalog(20000, 300.0, 16, seed=8)
    res = api.power_multipoles(cat, None, n=64, box=300.0, origin=(0, 0, 0), assign=3, interlace=1,
                               kbins=(0.02, 0.02, 25), ells=(0, 2), precision="mixed", los_dir=(0, 0, 1))
    spec = dict(n=64, box=300.0, origin=(0, 0, 0), assign=3, interlace=1, los="global", los_dir=(0, 0, 1))
    orc = P.power_multipoles(spec, cat, None, (0.02, 0.02, 25), (0, 2))
    _compare(res, orc, (0, 2), (), 1e-5)


def test_tiny_mesh_16(api):
    g, r, origin = make_survey_catalogs(2000, 20000, 400.0, 700.0, 8, seed=3, fkp_p0=1e4)
    kb = (0.0, 0.015, 8)
    res = api.power_multipoles(g, r, n=16, box=400.0, origin=origin, assign=3, interlace=1, kbins=kb,
                               ells=(0, 2, 4), modified=(4, 6, 8), precision="fp64")
    orc = _oracle(g, r, origin, 16, 400.0, 3, 1, kb, (0, 2, 4), (4, 6, 8))
    _compare(res, orc, (0, 2, 4), (4, 6, 8), 1e-12)


def test_particles_on_box_edges_and_outside(api):
    """Positions at the box faces and slightly outside wrap periodically on both sides."""
    rng = np.random.default_rng(9)
    box = 200.0
    pos = rng.random((3000, 3)) * box
    pos[:200, 0] = 0.0
    pos[200:400, 1] = np.nextafter(box, 0)
    pos[400:500, 2] = box + 3.0
    pos[500:600, 0] = -2.5
    g = SimpleNamespace(pos=pos, w=np.ones(3000), nbar=np.full(3000, 3000 / box**3))
    rr = rng.random((20000, 3)) * box
    r = SimpleNamespace(pos=rr, w=np.ones(20000), nbar=np.full(20000, 3000 / box**3))
    kb = (0.0, 0.03, 8)
    res = api.power_multipoles(g, r, n=32, box=box, origin=(0, 0, 0), assign=3, interlace=1, kbins=kb,
                               ells=(0, 2), precision="fp64", observer=(-500.0, -400.0, -300.0))
    spec = dict(n=32, box=box, origin=(0, 0, 0), assign=3, interlace=1, los="endpoint",
                observer=(-500.0, -400.0, -300.0))
    orc = P.power_multipoles(spec, g, r, kb, (0, 2))
    _compare(res, orc, (0, 2), (), 1e-12)


@pytest.mark.parametrize("assign", [2, 3])
def test_float_positions_on_cell_faces_mixed(api, assign):
    """Float positions on cell faces, cell centres and the box faces (where the float-pair fraction is
    within 1e-6 of an assignment decision and the float64 form decides), and a few float ulps off them
    (where the float-pair form decides alone), paint as the oracle does in mixed precision."""
    rng = np.random.default_rng(23 + assign)
    box, n = 200.0, 32
    h = box / n
    for origin in [(0.0, 0.0, 0.0), (-18.75, 12.5, 3.125), (0.1, -0.3, 7.7)]:
        o = np.array(origin)
        pos = o + rng.random((20000, 3)) * box
        pos[:12000] = o + rng.integers(-2, 2 * n + 2, size=(12000, 3)) * (h / 2)
        pos[8000:9000, 0] = o[0]
        pos[9000:10000, 1] = o[1] + box
        pos = pos.astype(np.float32)
        away = np.where(rng.random((2000, 3)) < 0.5, -np.inf, np.inf).astype(np.float32)
        pos[10000:12000] = np.nextafter(pos[10000:12000], away)
        nb = np.float32(20000 / box**3)
        cat = SimpleNamespace(pos=pos, w=np.ones(20000, np.float32), nbar=np.full(20000, nb, np.float32))
        kb = (0.0, 0.03, 8)
        res = api.power_multipoles(cat, None, n=n, box=box, origin=origin, assign=assign, interlace=1,
                                   kbins=kb, ells=(0, 2), precision="mixed", los_dir=(0, 0, 1))
        spec = dict(n=n, box=box, origin=origin, assign=assign, interlace=1, los="global", los_dir=(0, 0, 1))
        orc = P.power_multipoles(spec, cat, None, kb, (0, 2))
        _compare(res, orc, (0, 2), (), 1e-5)


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-5), ("fp64", 1e-11)])
def test_most_objects_in_one_cell(api, prec, tol):
    """A degenerate catalogue: 250,000 of 300,000 objects at one point, so one brick holds almost the
    whole catalogue (the largest per-brick count the painter's fixed-point scale has to absorb) and the
    field is nearly a spike; P_0, P_2 as the oracle has them.  FP64 tolerance: the brick's taps are
    rounded to multiples of 2^-e with 2^(61-e) > count x max w (count = 250,780 here, e = 43), and the
    250,000 identical taps all round the same way, so each of the 27 cells of a phase may be off by
    count x 2^-44 = 1.4e-8; divided by the compensation W > 0.5 in these bins and compared with
    |F| = 2.5e5 that is at most 3e-12 of F, 6e-12 of P (1.7e-12 measured), hence 1e-11."""
    rng = np.random.default_rng(61)
    box, n = 200.0, 32
    pos = rng.random((300000, 3)) * box
    pos[:250000] = (37.3, 101.9, 150.2)
    dt = np.float32 if prec == "mixed" else np.float64
    cat = SimpleNamespace(pos=pos.astype(dt), w=np.ones(300000, dt), nbar=np.full(300000, 300000 / box**3, dt))
    kb = (0.0, 0.03, 8)
    res = api.power_multipoles(cat, None, n=n, box=box, origin=(0.0, 0.0, 0.0), assign=3, interlace=1,
                               kbins=kb, ells=(0, 2), precision=prec, los_dir=(0, 0, 1))
    spec = dict(n=n, box=box, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global", los_dir=(0, 0, 1))
    orc = P.power_multipoles(spec, cat, None, kb, (0, 2))
    _compare(res, orc, (0, 2), (), tol)


def test_determinism_and_device_inputs(api):
    torch = pytest.importorskip("torch")
    g, r, origin = make_survey_catalogs(30000, 300000, 800.0, 1300.0, 32, seed=12, fkp_p0=1e4)
    kb = (0.0, 0.01, 20)
    a = api.power_multipoles(g, r, n=64, box=800.0, origin=origin, kbins=kb, ells=(0, 2, 4), modified=(4,))
    b = api.power_multipoles(g, r, n=64, box=800.0, origin=origin, kbins=kb, ells=(0, 2, 4), modified=(4,))
    for l in (0, 2, 4):
        np.testing.assert_array_equal(a["P"][l], b["P"][l])
    dev = lambda c: SimpleNamespace(pos=torch.from_numpy(c.pos).cuda(), w=torch.from_numpy(c.w).cuda(),
                                    nbar=torch.from_numpy(c.nbar).cuda())
    length = api.B.npc_power_out_len(C.byref(api.B.npc_kbins(*kb)), 0b10101, 1 << 4)
    out = torch.zeros(length, dtype=torch.float64, device="cuda")
    api.power_multipoles(dev(g), dev(r), n=64, box=800.0, origin=origin, kbins=kb, ells=(0, 2, 4),
                         modified=(4,), out=out)
    torch.cuda.synchronize()
    got = api.unpack_power(out.cpu().numpy(), kb[2], (0, 2, 4), (4,))
    for l in (0, 2, 4):
        np.testing.assert_array_equal(got["P"][l], a["P"][l])


def test_invalid_arguments_rejected(api):
    from paper_2605_04864_gb300 import binding as B

    g, r, origin = make_survey_catalogs(1000, 5000, 300.0, 600.0, 8, seed=1)
    kb = (0.0, 0.02, 5)
    for kw, code in [(dict(n=24), 1), (dict(n=2048), 1), (dict(assign=1), 1), (dict(interlace=2), 1),
                     (dict(kbins=(0.0, -0.01, 5)), 1), (dict(kbins=(0.0, 0.01, 0)), 1)]:
        args = dict(n=32, box=300.0, origin=origin, assign=3, interlace=1, kbins=kb, ells=(0,))
        args.update(kw)
        with pytest.raises(B.NpcError) as ei:
            api.power_multipoles(g, r, **args)
        assert ei.value.status == code, kw
    with pytest.raises(B.NpcError) as ei:
        api.power_multipoles(g, r, n=512, box=300.0, origin=origin, kbins=kb, ells=(0,), precision="fp64")
    assert ei.value.status == 4
    empty = SimpleNamespace(pos=np.zeros((0, 3), np.float32), w=np.zeros(0, np.float32),
                            nbar=np.zeros(0, np.float32))
    with pytest.raises(B.NpcError) as ei:
        api.power_multipoles(empty, r, n=32, box=300.0, origin=origin, kbins=kb, ells=(0,))
    assert ei.value.status == 6
    with pytest.raises(B.NpcError) as ei:
        api.power_multipoles(g, r, n=32, box=300.0, origin=origin, kbins=kb, ells=(0,), periodic=1)
    assert ei.value.status == 1
    # a catalogue and its randoms share one brick sort with 32-bit offsets: together they must hold
    # fewer than 2^31 objects.  The declared counts are rejected before any array is read (the
    # arrays behind them are the small ones above).
    keep = api._Keep()
    spec = api.make_spec(32, 300.0, origin, 3, 1, 0)
    kbs = B.npc_kbins(*kb)
    buf = np.zeros(64)
    ctx = api.context(0)
    for nd, nr in [((1 << 31) - 1, 1), (1 << 30, 1 << 30)]:
        d, rr = api.make_catalog(g, keep), api.make_catalog(r, keep)
        d.n, rr.n = nd, nr
        st = B.npc_power_multipoles(ctx, C.byref(spec), C.byref(d), C.byref(rr), C.byref(kbs), 1, 0,
                                    B.NPC_PREC_MIXED, buf.ctypes.data_as(C.c_void_p), 0)
        assert st == 4, (nd, nr, st)
        ga, ra = api.make_catalog(g, keep), api.make_catalog(r, keep)
        st = B.npc_cross_power_multipoles(ctx, C.byref(spec), C.byref(ga), C.byref(ra), C.byref(d), C.byref(rr),
                                          C.byref(kbs), 1, B.NPC_PREC_MIXED, buf.ctypes.data_as(C.c_void_p), 0)
        assert st == 4, ("cross", nd, nr, st)
    res = api.power_multipoles(g, r, n=32, box=300.0, origin=origin, kbins=kb, ells=(0,))
    assert np.all(np.isfinite(res["P"][0]))


@pytest.mark.slow
def test_full_size_512_all_multipoles(api):
    """The bench workload in full (512^3, 2e6 galaxies + 2e7 randoms, TSC interlaced, FKP weights,
    80 bins): every P_0, P_2, P_4, P_4b, P_6b, P_8b bin against the oracle's half-spectrum form,
    whose values are stored by tests/golden/make_full_size.py (re-evaluated here if this machine
    generates different input bytes); N_modes exactly, tolerance 1e-5 in the monopole-scale metric."""
    from synthetic import fingerprint

    gm = golden_module()
    w, g, r, spec = gm.power_inputs()

    def live():
        res = gm.power_oracle(w, g, r, spec)
        return {"k_eff": res["k_eff"], "nmodes": res["nmodes"], "P": {str(l): v for l, v in res["P"].items()},
                "Pmod": {str(l): v for l, v in res["Pmod"].items()},
                "scalars": {k: res["scalars"][k] for k in ("alpha", "I22", "N0")}}

    orc, _ = stored_or_live(gm.POWER_FILE, fingerprint(g, r), live)
    kb = (w["kmin"], w["dk"], w["nbins"])
    res = api.power_multipoles(g, r, n=512, box=w["box"], origin=spec["origin"], assign=3, interlace=1, kbins=kb,
                               ells=(0, 2, 4), modified=(4, 6, 8), precision="mixed")
    np.testing.assert_array_equal(res["nmodes"], np.asarray(orc["nmodes"]))
    np.testing.assert_allclose(res["k_eff"], np.asarray(orc["k_eff"]), rtol=1e-6, atol=1e-12)
    for k in ("alpha", "I22", "N0"):
        assert res["scalars"][k] == pytest.approx(orc["scalars"][k], rel=1e-12)
    scale = np.abs(np.asarray(orc["P"]["0"])) + orc["scalars"]["N0"]
    for l in (0, 2, 4):
        e = p_error(res["P"][l], np.asarray(orc["P"][str(l)]), scale)
        assert np.max(e) < 1e-5, (l, np.max(e))
    for l in (4, 6, 8):
        e = p_error(res["Pmod"][l], np.asarray(orc["Pmod"][str(l)]), scale)
        assert np.max(e) < 1e-5, ("b", l, np.max(e))


@pytest.mark.parametrize("prec,tol,n", [("fp64", 1e-12, 32), ("mixed", 1e-5, 64)])
def test_odd_multipoles_survey(api, prec, tol, n):
    """Odd P_1, P_3 (imaginary part, Sec. 2.1) with the endpoint line of sight, together with the
    even ones and the modified multipoles (ten sums per bin)."""
    g, r, origin = make_survey_catalogs(20000, 200000, 1000.0, 1200.0, 24, seed=61, fkp_p0=1e4)
    kb = (0.0, 0.015, 8)
    res = api.power_multipoles(g, r, n=n, box=1000.0, origin=origin, kbins=kb, ells=(0, 1, 2, 3, 4),
                               modified=(4, 6, 8), precision=prec)
    orc = _oracle(g, r, origin, n, 1000.0, 3, 1, kb, (0, 1, 2, 3, 4), (4, 6, 8))
    _compare(res, orc, (0, 1, 2, 3, 4), (4, 6, 8), tol)
    scale = np.abs(orc["P"][0]) + orc["scalars"]["N0"]
    assert np.max(np.abs(orc["P"][1]) / scale) > 1e-6   # the odd terms measured are not all zero


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_two_index_multipoles(api, prec, tol):
    """P_22, P_42, P_44 of Eq. Pllp reported next to the modified multipoles, alone and together."""
    g, r, origin = make_survey_catalogs(20000, 200000, 800.0, 1300.0, 24, seed=63, fkp_p0=1e4)
    kb = (0.0, 0.015, 8)
    orc = _oracle(g, r, origin, 32, 800.0, 3, 1, kb, (0, 2, 4), (4, 6, 8))
    scale = np.abs(orc["P"][0]) + orc["scalars"]["N0"]
    res = api.power_multipoles(g, r, n=32, box=800.0, origin=origin, kbins=kb, ells=(0, 2), modified=(6,),
                               two_index=((2, 2), (4, 2), (4, 4)), precision=prec)
    for p in ((2, 2), (4, 2), (4, 4)):
        assert np.max(p_error(res["Pll"][p], orc["Pll"][p], scale)) < tol, p
    assert np.max(p_error(res["Pmod"][6], orc["Pmod"][6], scale)) < tol
    only = api.power_multipoles(g, r, n=32, box=800.0, origin=origin, kbins=kb, ells=(0,), two_index=((4, 4),),
                                precision=prec)
    assert np.max(p_error(only["Pll"][(4, 4)], orc["Pll"][(4, 4)], scale)) < tol
