"""Pins for oracle.power / oracle.mesh against closed forms, brute force and the paper's identities."""
from fractions import Fraction
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import harmonics as H
from oracle import mesh as M
from oracle import power as P
from synthetic import make_survey_catalogs


def _survey_spec(n, box, origin, assign=2, interlace=0):
    return dict(n=n, box=box, origin=tuple(origin), assign=assign, interlace=interlace,
                los="endpoint", observer=(0.0, 0.0, 0.0))


@pytest.fixture(scope="module")
def small_survey():
    g, r, origin = make_survey_catalogs(3000, 30000, 1000.0, 1500.0, 16, seed=5, fkp_p0=1e4)
    return g, r, origin


@pytest.mark.parametrize("interlace,assign", [(0, 2), (1, 3)])
def test_symmetric_equals_hand17(small_survey, interlace, assign):
    """Eqs. pk_final / new_F_ell (l+1 transforms) equal Eq. hand (2l+1 transforms) on the grid."""
    g, r, origin = small_survey
    spec = _survey_spec(24, 1000.0, origin, assign, interlace)
    kb = (0.0, 0.02, 4)
    a = P.power_multipoles(spec, g, r, kb, (0, 2, 4), (4, 6, 8), method="plain")
    b = P.power_multipoles(spec, g, r, kb, (0, 2, 4), (4, 6, 8), method="symmetric")
    for ell in (0, 2, 4):
        scale = np.abs(a["P"][0]) + a["scalars"]["N0"]
        assert np.max(np.abs(a["P"][ell] - b["P"][ell]) / scale) < 1e-13
    for lb in (4, 6, 8):
        scale = np.abs(a["P"][0]) + a["scalars"]["N0"]
        assert np.max(np.abs(a["Pmod"][lb] - b["Pmod"][lb]) / scale) < 1e-12
    # Table 1: 15 (Hand+17) vs 9 (this work) transforms for l_max = 4
    assert a["n_transforms_per_phase"] == 15
    assert b["n_transforms_per_phase"] == 9


def test_transform_counts_table1():
    """Table 1 closed forms, l_max = 4 and 8, from the oracle's loops."""
    spec = dict(n=4, box=100.0, origin=(0, 0, 0), assign=2, los="global", los_dir=(0, 0, 1))
    mesh = [np.zeros((4, 4, 4))]
    for lmax, hand, ours, modified in [(4, 15, 9, 4), (8, 45, 25, 9)]:
        ells = list(range(0, lmax + 1, 2))
        _, n1 = P.fields_plain(spec, mesh, ells)
        _, n2 = P.fields_symmetric(spec, mesh, ells)
        _, n3 = P.fields_symmetric(spec, mesh, list(range(0, lmax // 2 + 1, 2)))
        assert (n1, n2, n3) == (hand, ours, modified)
        assert hand == (lmax + 1) * (lmax + 2) // 2
        assert ours == (lmax + 2) ** 2 // 4
        assert modified == (lmax + 4) ** 2 // 16


def test_inversion_gives_hermitian_F(small_survey):
    """F_l from G_l by space inversion equals the Hand+17 F_l away from Nyquist planes."""
    g, r, origin = small_survey
    spec = _survey_spec(16, 1000.0, origin, 2, 0)
    sc = P.catalog_scalars(g, r)
    meshes = P.fkp_meshes(spec, g, r, sc)
    fp, _ = P.fields_plain(spec, meshes, [2, 4])
    gs, _ = P.fields_symmetric(spec, meshes, [2, 4])
    _, (ix, iy, iz) = M.kvectors(16, 1000.0)
    ok = (ix != -8) & (iy != -8) & (iz != -8)
    ok = np.broadcast_to(ok, (16, 16, 16))
    for ell in (2, 4):
        fi = P.f_from_g(gs[ell], ell)
        assert np.max(np.abs(fi - fp[ell])[ok]) < 1e-10 * np.max(np.abs(fp[ell]))
        herm = np.conj(P.space_invert(fi))
        assert np.max(np.abs(fi - herm)[ok]) < 1e-10 * np.max(np.abs(fi))


def test_gaussian_fixed_amplitude_gives_input_power():
    """A field with |delta(k)| fixed to the input power: P_0 and P_2 equal the binned input exactly."""
    n, box, beta = 32, 500.0, 0.8
    rng = np.random.default_rng(3)
    wk = np.fft.fftn(rng.standard_normal((n, n, n)))
    (kx, ky, kz), _ = M.kvectors(n, box)
    kk = np.sqrt(kx**2 + ky**2 + kz**2)
    mu = np.where(kk > 0, kz / np.where(kk > 0, kk, 1), 0)
    pin = np.where(kk > 0, 1e4 * np.exp(-kk / 0.3), 0.0) * (1 + beta * mu**2) ** 2
    vol, nc = box**3, n**3
    delta_k = wk / np.abs(wk) * nc * np.sqrt(pin / vol)
    delta_x = np.real(np.fft.ifftn(delta_k))
    nbar = 1e-3
    field = nbar * (vol / nc) * delta_x
    spec = dict(n=n, box=box, origin=(0, 0, 0), assign=0, los="global", los_dir=(0, 0, 1))
    fields, _ = P.fields_plain(spec, [field], [0, 2])
    sc = dict(I22=nbar**2 * vol, N0=0.0)
    kb = (0.0, 0.02, 6)
    res = P.power_from_fields(spec, fields, kb, (0, 2), sc)
    b, _ = M.bin_index(n, box, *kb)
    p0, _ = M.bin_average(pin, b, kb[2])
    p2, _ = M.bin_average(5 * pin * H.legendre(2, mu), b, kb[2])
    np.testing.assert_allclose(res["P"][0], p0, rtol=1e-12)
    np.testing.assert_allclose(res["P"][2], p2, rtol=1e-10, atol=1e-12 * np.max(p0))


@pytest.mark.parametrize("assign", [2, 3])
def test_poisson_shot_noise_alias_sum(assign):
    """Uniform Poisson points: E|F(k)|^2 = N sum_n W^2(k + 2 k_N n) (Jing 2005, cited in Sec. 3.1).
    After compensation P_0 + N_0 = (V/N) <C(k)/W^2(k)>, C the closed-form alias sum."""
    n, box, npart, nseed = 16, 100.0, 4000, 24
    kb = (0.1, 0.3, 3)
    acc = 0.0
    for seed in range(nseed):
        rng = np.random.default_rng(100 + seed)
        pos = rng.random((npart, 3)) * box
        cat = SimpleNamespace(pos=pos, w=np.ones(npart), nbar=np.full(npart, npart / box**3))
        spec = dict(n=n, box=box, origin=(0, 0, 0), assign=assign, interlace=0, los="global",
                    los_dir=(0, 0, 1))
        res = P.power_multipoles(spec, cat, None, kb, (0,))
        acc = acc + res["P"][0] + res["scalars"]["N0"]
    acc /= nseed
    s = np.sin(np.pi * M.int_freqs(n) / n) ** 2
    if assign == 2:
        c1 = 1 - 2.0 / 3.0 * s
    else:
        c1 = 1 - s + 2.0 / 15.0 * s * s
    C = c1[:, None, None] * c1[None, :, None] * c1[None, None, :]
    W = M.window(n, assign)
    b, _ = M.bin_index(n, box, *kb)
    want, cnt = M.bin_average(C / W**2, b, kb[2])
    want *= box**3 / npart
    err = 3.0 / np.sqrt(cnt * nseed)
    assert np.all(np.abs(acc / want - 1) < err)


def test_interlacing_removes_alias_at_low_k():
    n, box, npart, nseed = 16, 100.0, 4000, 16
    kb = (0.05, 0.1, 2)
    acc = 0.0
    for seed in range(nseed):
        rng = np.random.default_rng(700 + seed)
        pos = rng.random((npart, 3)) * box
        cat = SimpleNamespace(pos=pos, w=np.ones(npart), nbar=np.full(npart, npart / box**3))
        spec = dict(n=n, box=box, origin=(0, 0, 0), assign=3, interlace=1, los="global",
                    los_dir=(0, 0, 1))
        res = P.power_multipoles(spec, cat, None, kb, (0,))
        acc = acc + (res["P"][0] + res["scalars"]["N0"]) / res["scalars"]["N0"]
    acc /= nseed
    assert np.all(np.abs(acc - 1) < 0.08)


def test_cic_at_grid_points_equals_direct_dft():
    """Particles exactly on grid points with CIC: mesh DFT equals the per-particle DFT exactly."""
    n, box = 8, 80.0
    rng = np.random.default_rng(1)
    idx = rng.integers(0, n, size=(50, 3))
    pos = idx * (box / n)
    w = rng.random(50)
    mesh = M.paint(M.grid_coords(pos, (0, 0, 0), box, n), w, n, 2)
    fk = np.fft.fftn(mesh)
    (kx, ky, kz), _ = M.kvectors(n, box)
    kv = np.stack(np.broadcast_arrays(kx, ky, kz), -1).reshape(-1, 3)
    direct = P.direct_dft(pos, w, kv, (0, 0, 0)).reshape(n, n, n)
    np.testing.assert_allclose(fk, direct, atol=1e-12)


@pytest.mark.parametrize("assign,interlace", [(2, 0), (3, 0), (3, 1)])
def test_compensated_mesh_dft_matches_direct_at_low_k(assign, interlace):
    n, box = 32, 320.0
    rng = np.random.default_rng(2)
    pos = rng.random((400, 3)) * box
    w = 0.5 + rng.random(400)
    cat = SimpleNamespace(pos=pos, w=w, nbar=np.ones(400))
    spec = dict(n=n, box=box, origin=(0, 0, 0), assign=assign, interlace=interlace,
                los="global", los_dir=(0, 0, 1))
    sc = dict(alpha=0.0)
    meshes = []
    for sh in ((0.0, 0.5) if interlace else (0.0,)):
        meshes.append(M.paint(M.grid_coords(pos, (0, 0, 0), box, n, sh), w, n, assign))
    s = P.ylm_transform(spec, meshes, 0, 0) * np.sqrt(4 * np.pi)
    (kx, ky, kz), (ix, iy, iz) = M.kvectors(n, box)
    sel = np.broadcast_to((np.abs(ix) <= 2) & (np.abs(iy) <= 2) & (np.abs(iz) <= 2), (n, n, n))
    kv = np.stack(np.broadcast_arrays(kx, ky, kz), -1)[sel]
    direct = P.direct_dft(pos, w, kv, (0, 0, 0))
    rel = np.abs(s[sel] - direct) / np.sqrt(np.sum(w**2))
    assert np.max(rel) < (0.25 if not interlace else 0.05)
    del sc


def test_modified_equal_direct_for_global_los(small_survey):
    """With one global line of sight F_l = L_l(mu) F_0 exactly, so by Eq. legendre P_lb = P_l."""
    g, r, origin = small_survey
    spec = dict(n=16, box=1000.0, origin=tuple(origin), assign=3, interlace=1, los="global",
                los_dir=(1.0, 1.0, 1.0))
    kb = (0.0, 0.02, 5)
    res = P.power_multipoles(spec, g, r, kb, (0, 2, 4, 6, 8), (4, 6, 8), method="plain")
    scale = np.abs(res["P"][0]) + res["scalars"]["N0"]
    for lb in (4, 6, 8):
        assert np.max(np.abs(res["Pmod"][lb] - res["P"][lb]) / scale) < 1e-12


def test_plb_coefficients_from_legendre_identities():
    """Eq. Plnew from Eq. legendre: coefficient of P_ab is c_ab (2l+1)/(2(a+b)+1), of P_b (a=0)
    is c_0b (2l+1)/(2b+1); the shot noise of every P_lb cancels exactly (N_22 = 9/5 N_0, N_44 = 17/9 N_0)."""
    leg = {
        4: {(2, 2): Fraction(35, 18), (0, 2): Fraction(-5, 9), (0, 0): Fraction(-7, 18)},
        6: {(4, 2): Fraction(11, 5), (0, 4): Fraction(-4, 7), (0, 2): Fraction(-22, 35)},
        8: {(4, 4): Fraction(1287, 490), (4, 2): Fraction(-286, 245), (0, 4): Fraction(-209, 1715),
            (0, 2): Fraction(-78, 1715), (0, 0): Fraction(-143, 490)},
    }
    for lb, terms in leg.items():
        for (a, b), c in terms.items():
            want = c * (2 * lb + 1) / (2 * (a + b) + 1)
            assert P.PLB_COEFFS[lb][(a, b)] == want
        shot = sum(c * (2 * lb + 1) / (2 * (a + b) + 1)
                   * (Fraction(2 * (a + b) + 1, 2 * a + 1) if a == b else 0)
                   for (a, b), c in terms.items())
        assert shot == 0
    assert P.n_shot_two_index(2, 2, 1.0) == pytest.approx(9 / 5)
    assert P.n_shot_two_index(4, 4, 1.0) == pytest.approx(17 / 9)


def test_catalog_scalars_uniform():
    rng = np.random.default_rng(0)
    g = SimpleNamespace(pos=rng.random((1000, 3)), w=np.ones(1000), nbar=np.full(1000, 2.0))
    r = SimpleNamespace(pos=rng.random((5000, 3)), w=np.ones(5000), nbar=np.full(5000, 2.0))
    sc = P.catalog_scalars(g, r)
    assert sc["alpha"] == pytest.approx(0.2)
    assert sc["I22"] == pytest.approx(0.2 * 5000 * 2.0)
    assert sc["N0"] == pytest.approx((1000 + 0.04 * 5000) / 2000.0)
    per = P.catalog_scalars(g, None, box=10.0)
    assert per["I22"] == pytest.approx(1000**2 / 1000.0)
    assert per["N0"] == pytest.approx(1.0)


@pytest.mark.parametrize("c", [1.0, 0.37])
def test_catalog_scalars_are_the_density_integrals(c):
    """I22 and I33 are the integrals of (nbar w)^2 and (nbar w)^3 over the volume (Secs. 2.1, 2.2):
    for a uniform survey of volume V (nbar = N_g / V on every random) with constant weight c they are
    nbar^2 c^2 V and nbar^3 c^3 V, the values the periodic-box forms give for the same data, and the
    three-point self term is N_g c^3 (1 - alpha^2)."""
    rng = np.random.default_rng(3)
    ng, nr, box = 2000, 30000, 50.0
    vol = box**3
    nb = ng / vol
    g = SimpleNamespace(pos=rng.random((ng, 3)) * box, w=np.full(ng, c), nbar=np.full(ng, nb))
    r = SimpleNamespace(pos=rng.random((nr, 3)) * box, w=np.full(nr, c), nbar=np.full(nr, nb))
    sur = P.catalog_scalars(g, r)
    per = P.catalog_scalars(g, None, box=box)
    alpha = ng / nr
    assert sur["I22"] == pytest.approx(nb**2 * c**2 * vol, rel=1e-12)
    assert sur["I33"] == pytest.approx(nb**3 * c**3 * vol, rel=1e-12)
    assert per["I22"] == pytest.approx(nb**2 * c**2 * vol, rel=1e-12)
    assert per["I33"] == pytest.approx(nb**3 * c**3 * vol, rel=1e-12)
    assert sur["S3"] == pytest.approx(ng * c**3 * (1 - alpha**2), rel=1e-12)


@pytest.mark.parametrize("interlace,assign", [(0, 2), (1, 3)])
def test_rfft_monopole_equals_full_grid(small_survey, interlace, assign):
    """The half-grid monopole used for full-size checks equals the full-grid Hand+17 P_0."""
    g, r, origin = small_survey
    spec = _survey_spec(24, 1000.0, origin, assign, interlace)
    kb = (0.0, 0.015, 6)
    a = P.power_multipoles(spec, g, r, kb, (0,), method="plain")
    p0, cnt, sc = P.power_monopole_rfft(spec, g, r, kb)
    np.testing.assert_array_equal(cnt, a["nmodes"])
    np.testing.assert_allclose(p0, a["P"][0], rtol=1e-12, atol=1e-12 * sc["N0"])


@pytest.mark.parametrize("interlace,assign", [(0, 2), (1, 3)])
def test_cross_with_itself_is_auto_plus_shot(small_survey, interlace, assign):
    """The cross multipoles of a tracer with itself equal its auto multipoles with the shot noise
    N_0 added back to the monopole (same fields, I22^AA = I22^A)."""
    g, r, origin = small_survey
    spec = _survey_spec(20, 1000.0, origin, assign, interlace)
    kb = (0.0, 0.02, 4)
    auto = P.power_multipoles(spec, g, r, kb, (0, 2, 4))
    cross = P.cross_power_multipoles(spec, g, r, g, r, kb, (0, 2, 4))
    n0 = auto["scalars"]["N0"]
    scale = np.abs(auto["P"][0]) + n0
    for ell in (0, 2, 4):
        want = auto["P"][ell] + (n0 if ell == 0 else 0.0) * (auto["nmodes"] > 0)
        assert np.max(np.abs(cross["P"][ell] - want) / scale) < 1e-12


def test_cross_is_symmetric_for_a_global_line_of_sight():
    """With a fixed line of sight F_l = L_l(mu) F_0 for both tracers, so P_l^AB = P_l^BA."""
    from synthetic import make_periodic_catalog

    a = make_periodic_catalog(5000, 500.0, 16, seed=91)
    b = make_periodic_catalog(3000, 500.0, 16, seed=92)
    spec = dict(n=20, box=500.0, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=1)
    kb = (0.0, 0.03, 5)
    ab = P.cross_power_multipoles(spec, a, None, b, None, kb, (0, 2, 4))
    ba = P.cross_power_multipoles(spec, b, None, a, None, kb, (0, 2, 4))
    scale = np.max(np.abs(ab["P"][0]))
    for ell in (0, 2, 4):
        assert np.max(np.abs(ab["P"][ell] - ba["P"][ell])) < 1e-12 * scale
    # and it is not the auto spectrum of either
    assert np.max(np.abs(ab["P"][0] - P.power_multipoles(spec, a, None, kb, (0,))["P"][0])) > 1e-3 * scale


def test_odd_multipoles_symmetric_equals_hand17(small_survey):
    """Odd l (Sec. 2.1: the imaginary part): Im<F_0 G_l^*> from the l+1 transforms equals
    Im<F_0 F_l^*> of the Hand+17 sum over 2l+1 transforms."""
    g, r, origin = small_survey
    spec = _survey_spec(20, 1000.0, origin, 3, 1)
    kb = (0.0, 0.02, 4)
    a = P.power_multipoles(spec, g, r, kb, (0, 1, 3), method="plain")
    b = P.power_multipoles(spec, g, r, kb, (0, 1, 3), method="symmetric")
    scale = np.abs(a["P"][0]) + a["scalars"]["N0"]
    for ell in (1, 3):
        assert np.max(np.abs(a["P"][ell])) > 1e-6 * np.max(scale)   # wide-angle odd terms are not zero
        assert np.max(np.abs(a["P"][ell] - b["P"][ell]) / scale) < 1e-13


def test_odd_cross_multipoles_of_a_shifted_copy():
    """Tracer B = tracer A moved by two cells along the line of sight (periodic box): F^B = e^{-i k.d}
    F^A exactly, so P_l^AB = (2l+1)/I22 <|F^A|^2 L_l(mu) cos(k_z d)> (even l) and the same with
    sin(k_z d) (odd l), and the odd auto multipoles vanish."""
    from types import SimpleNamespace

    from synthetic import make_periodic_catalog

    box, n = 500.0, 20
    a = make_periodic_catalog(4000, box, 16, seed=93, dtype=np.float64)
    d = 2 * box / n
    b = SimpleNamespace(pos=a.pos.copy(), w=a.w, nbar=a.nbar)
    b.pos[:, 2] = np.mod(b.pos[:, 2] + d, box)
    spec = dict(n=n, box=box, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, los="global",
                los_dir=(0.0, 0.0, 1.0), periodic=1)
    kb = (0.0, 0.04, 4)
    ells = (0, 1, 2, 3, 4)
    cross = P.cross_power_multipoles(spec, a, None, b, None, kb, ells)
    sc = P.catalog_scalars(a, None, box)
    f0 = P.fields_plain(spec, P.fkp_meshes(spec, a, None, sc), [0])[0][0]
    bidx, _ = M.bin_index(n, box, *kb)
    (kx, ky, kz), _ = M.kvectors(n, box)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(kk > 0, kz / np.where(kk > 0, kk, 1.0), 0.0)
    scale = np.max(np.abs(cross["P"][0]))
    for ell in ells:
        ph = np.sin(kz * d) if ell % 2 else np.cos(kz * d)
        want, _ = M.bin_average(np.abs(f0) ** 2 * H.legendre(ell, mu) * ph, bidx, kb[2])
        want = (2 * ell + 1) / sc["I22"] * want
        assert np.max(np.abs(cross["P"][ell] - want)) < 1e-9 * scale, ell
    assert np.max(np.abs(cross["P"][1])) > 1e-3 * scale
    auto = P.power_multipoles(spec, a, None, kb, (0, 1, 3))
    for ell in (1, 3):
        assert np.max(np.abs(auto["P"][ell])) < 1e-12 * np.max(np.abs(auto["P"][0]))


@pytest.mark.parametrize("n,assign,interlace,los", [(24, 2, 0, "endpoint"), (32, 3, 1, "endpoint"),
                                                    (48, 3, 1, "endpoint"), (32, 3, 1, "global")])
def test_half_spectrum_form_equals_full_grid(small_survey, n, assign, interlace, los):
    """The half-spectrum (real-to-complex) evaluation of the symmetric form gives, for every
    multipole (even and odd l, the two-index P_ll' and the modified P_lb), the values of the
    full-grid Hand+17 sum over all 2l+1 values of m (Eq. hand), and the same mode counts and k_eff,
    in bins reaching the corners of the Fourier cube: meshes of 2^k and 3 * 2^k cells, CIC without
    and TSC with interlacing, both lines of sight."""
    g, r, origin = small_survey
    spec = _survey_spec(n, 1000.0, origin, assign, interlace)
    if los == "global":
        spec.update(los="global", los_dir=(1.0, 2.0, 2.0))
    # bins up to sqrt(3) k_N: every mode of the cube has a bin, so the Nyquist planes that both
    # forms leave out are compared too
    kb = (0.0, 0.01, int(np.sqrt(3.0) * np.pi * n / 1000.0 / 0.01) + 1)
    ells = (0, 1, 2, 3, 4)
    two = ((2, 2), (4, 2), (4, 4))
    a = P.power_multipoles(spec, g, r, kb, ells, (4, 6, 8), method="plain")
    b = P.power_multipoles_rfft(spec, g, r, kb, ells, (4, 6, 8), two_index=two)
    np.testing.assert_array_equal(a["nmodes"], b["nmodes"])
    np.testing.assert_allclose(a["k_eff"], b["k_eff"], rtol=1e-13, atol=0)
    scale = np.abs(a["P"][0]) + a["scalars"]["N0"]
    for ell in ells:
        assert np.max(np.abs(a["P"][ell] - b["P"][ell]) / scale) < 1e-12, ell
    for lb in (4, 6, 8):
        assert np.max(np.abs(a["Pmod"][lb] - b["Pmod"][lb]) / scale) < 1e-12, lb
    for key in two:
        assert np.max(np.abs(a["Pll"][key] - b["Pll"][key]) / scale) < 1e-12, key
    if los == "endpoint":
        assert np.max(np.abs(b["P"][1]) / scale) > 1e-8     # the odd terms compared are not all zero


def test_half_spectrum_stages_are_the_pipeline(small_survey):
    """The stage list runs the painting of each phase, one stage per phase and (l, m >= 0), then
    the binning: 2 + 2 * 9 + 1 stages for P_0,2,4 with interlacing (Table 1: 9 transforms per
    phase), and running them one by one gives the function's result."""
    g, r, origin = small_survey
    spec = _survey_spec(16, 1000.0, origin, 3, 1)
    kb = (0.0, 0.02, 2)
    run = P.HalfSpectrumPower(spec, g, r, kb, (0, 2, 4), (4,))
    st = run.stages()
    assert len(st) == 2 + 2 * 9 + 1
    for _, f in st:
        f()
    ref = P.power_multipoles_rfft(spec, g, r, kb, (0, 2, 4), (4,))
    for ell in (0, 2, 4):
        np.testing.assert_array_equal(run.result["P"][ell], ref["P"][ell])
