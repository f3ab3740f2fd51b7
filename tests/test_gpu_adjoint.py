"""GPU parity of the mesh-level estimators and their adjoints (through the C ABI and the torch
autograd front end) against the FP64 oracle and finite differences."""
import ctypes as C

import numpy as np
import pytest

from helpers import ensure_built
from oracle import adjoint as OA
from oracle import mesh as OM
from synthetic import make_periodic_catalog, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    ensure_built()
    from paper_2605_04864_gb300 import api as A
    from paper_2605_04864_gb300 import autograd as AG
    from paper_2605_04864_gb300 import binding as B

    return A, AG, B


def _oracle_mesh(n, box, n_gal, seed, assign=3):
    """Oracle-painted periodic lognormal mesh (mean removed), index order (x, y, z)."""
    cat = make_periodic_catalog(n_gal, box, max(n, 16), seed=seed, dtype=np.float64)
    s = OM.grid_coords(cat.pos, (0.0, 0.0, 0.0), box, n)
    m = OM.paint(s, cat.w, n, assign)
    return m - m.mean(), cat


def _dev(m_xyz, dtype):
    """(x, y, z) oracle array -> device mesh with index (z, y, x)."""
    return torch.tensor(np.ascontiguousarray(m_xyz.transpose(2, 1, 0)), dtype=dtype, device="cuda")


def _host(m_dev):
    return m_dev.double().cpu().numpy().transpose(2, 1, 0)


def _forward(mods, mesh, box, kb, ells, b0, i22, n0, i33, prec, assign=3):
    A, _, B = mods
    n = mesh.shape[0]
    spec = A.make_spec(n, box, (0, 0, 0), assign, 0, 1, (0.0, 0.0, 1.0))
    kbs = B.npc_kbins(*kb)
    emask = sum(1 << l for l in ells)
    length = B.npc_mesh_multipoles_len(C.byref(kbs), emask, int(b0))
    out = np.zeros(length)
    h = A.context(0)
    B.check(B.npc_mesh_multipoles(h, C.byref(spec), C.c_void_p(mesh.data_ptr()), C.byref(kbs), emask, int(b0),
                                  i22, n0, i33, A._prec(prec), out.ctypes.data_as(C.c_void_p), 0), h)
    nb = kb[2]
    res = {"k_eff": out[:nb], "nmodes": out[nb:2 * nb]}
    for e, l in enumerate(sorted(ells)):
        res[l] = out[(2 + e) * nb:(3 + e) * nb]
    if b0:
        res["B0"] = out[(2 + len(ells)) * nb:(3 + len(ells)) * nb]
        res["NT"] = out[(3 + len(ells)) * nb:(4 + len(ells)) * nb]
    return res


def _vjp(mods, mesh, box, kb, ells, b0, i22, i33, dldp, dldb, prec, assign=3):
    A, _, B = mods
    n = mesh.shape[0]
    spec = A.make_spec(n, box, (0, 0, 0), assign, 0, 1, (0.0, 0.0, 1.0))
    kbs = B.npc_kbins(*kb)
    emask = sum(1 << l for l in ells)
    grad = torch.empty_like(mesh)
    dp = np.ascontiguousarray(np.stack([dldp[l] for l in sorted(ells)]) if ells else np.zeros(1))
    db = np.ascontiguousarray(dldb if b0 else np.zeros(1))
    h = A.context(0)
    B.check(B.npc_mesh_multipoles_vjp(h, C.byref(spec), C.c_void_p(mesh.data_ptr()), C.byref(kbs), emask, int(b0),
                                      i22, i33, dp.ctypes.data_as(C.c_void_p) if ells else None,
                                      db.ctypes.data_as(C.c_void_p) if b0 else None, 0, A._prec(prec),
                                      C.c_void_p(grad.data_ptr())), h)
    torch.cuda.synchronize()
    return grad


CASES = [("fp64", 32, 1e-10, 1e-9), ("mixed", 32, 2e-5, 2e-4), ("mixed", 64, 2e-5, 2e-4), ("fp64", 16, 1e-10, 1e-9)]


@pytest.mark.parametrize("prec,n,ptol,gtol", CASES)
def test_forward_matches_oracle(mods, prec, n, ptol, gtol):
    box = 93.75 * n / 32
    kb = (0.1, 0.1, 4)
    m, _ = _oracle_mesh(n, box, 40 * n * n, seed=11 + n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    i22, n0, i33 = 2.5e-3, 40.0, 1.5e-6
    res = _forward(mods, _dev(m, dt), box, kb, (0, 2, 4), True, i22, n0, i33, prec)
    orc = OA.power_from_mesh(m, box, 3, kb, (0, 2, 4), i22, n0)
    b, _ = OM.bin_index(n, box, *kb)
    cnt = np.bincount(b[b >= 0], minlength=kb[2])
    np.testing.assert_array_equal(res["nmodes"], cnt)
    scale = np.abs(orc[0]) + n0
    for l in (0, 2, 4):
        err = np.abs(res[l] - orc[l]) / scale
        assert err.max() < ptol, (l, err.max())
    b0 = OA.bispec0_equilateral(m, box, 3, kb, i33)
    np.testing.assert_allclose(res["B0"], b0, rtol=gtol)
    # triangle counts: integers equal to the counts from the oracle's indicator fields -- exact in
    # FP64; float32 shells keep the count exact only while its rounding error stays under half a
    # triangle, so large counts may be off by a few (relative <= 2e-5, inside the B_0 tolerance)
    I = OA._shells(None, n, box, kb, ones=True)
    nt = np.round(np.array([np.sum(f ** 3) / n**3 for f in I]))
    np.testing.assert_array_equal(res["NT"], np.round(res["NT"]))
    np.testing.assert_allclose(res["NT"], nt, rtol=0 if prec == "fp64" else 2e-5, atol=0)


@pytest.mark.parametrize("prec,n,box,kb,tol", [("fp64", 64, 187.5, (0.05, 0.05, 3), 1e-9),
                                               ("mixed", 128, 375.0, (0.05, 0.05, 3), 2e-4)])
def test_shells_on_coarser_grid(mods, prec, n, box, kb, tol):
    """Bins far below k_N: the B_0 shells run on a coarser grid (32 for the 64^3 mesh, 48 for the
    128^3 mesh, the smallest length >= 3 K + 1); values and gradients must not change."""
    m, _ = _oracle_mesh(n, box, 20 * n * n, seed=51 + n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    i22, n0, i33 = 2.5e-3, 40.0, 1.5e-6
    res = _forward(mods, _dev(m, dt), box, kb, (0,), True, i22, n0, i33, prec)
    np.testing.assert_allclose(res["B0"], OA.bispec0_equilateral(m, box, 3, kb, i33), rtol=tol)
    I = OA._shells(None, n, box, kb, ones=True)
    np.testing.assert_allclose(res["NT"], np.round([np.sum(f ** 3) / n**3 for f in I]),
                               rtol=0 if prec == "fp64" else 2e-5, atol=0)
    rng = np.random.default_rng(8)
    dldb = rng.standard_normal(kb[2])
    g = _host(_vjp(mods, _dev(m, dt), box, kb, (), True, i22, i33, None, dldb, prec))
    ref = OA.bispec0_mesh_grad(m, box, 3, kb, i33, dldb)
    assert np.abs(g - ref).max() / np.abs(ref).max() < tol


@pytest.mark.parametrize("prec,n,ptol,gtol", CASES)
def test_vjp_matches_oracle(mods, prec, n, ptol, gtol):
    box = 93.75 * n / 32
    kb = (0.1, 0.1, 4)
    m, _ = _oracle_mesh(n, box, 40 * n * n, seed=21 + n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    i22, i33 = 2.5e-3, 1.5e-6
    rng = np.random.default_rng(5)
    dldp = {l: rng.standard_normal(kb[2]) for l in (0, 2, 4)}
    dldb = rng.standard_normal(kb[2])
    g = _host(_vjp(mods, _dev(m, dt), box, kb, (0, 2, 4), True, i22, i33, dldp, dldb, prec))
    ref = OA.power_mesh_grad(m, box, 3, kb, (0, 2, 4), i22, dldp) + OA.bispec0_mesh_grad(m, box, 3, kb, i33, dldb)
    err = np.abs(g - ref).max() / np.abs(ref).max()
    assert err < gtol, err
    # each part alone
    gp = _host(_vjp(mods, _dev(m, dt), box, kb, (0, 2, 4), False, i22, i33, dldp, None, prec))
    rp = OA.power_mesh_grad(m, box, 3, kb, (0, 2, 4), i22, dldp)
    assert np.abs(gp - rp).max() / np.abs(rp).max() < gtol
    gb = _host(_vjp(mods, _dev(m, dt), box, kb, (), True, i22, i33, None, dldb, prec))
    rb = OA.bispec0_mesh_grad(m, box, 3, kb, i33, dldb)
    assert np.abs(gb - rb).max() / np.abs(rb).max() < gtol


def test_vjp_finite_differences_fp64_32(mods):
    """Directional derivatives of the GPU forward (FP64, 32^3) against the GPU gradient.  P_l is
    quadratic and B_0 cubic in the mesh, so the central difference has no truncation error for P and
    an error exactly proportional to eps^2 for B_0, removed by one Richardson step."""
    w = workload("adjoint_32")
    n, box = w["n"], w["box"]
    kb = (w["kmin"], w["dk"], w["nbins"])
    m, _ = _oracle_mesh(n, box, w["n_gal"] * 20, seed=w["seed"])
    i22, n0, i33 = 2.5e-3, 40.0, 1.5e-6
    rng = np.random.default_rng(9)
    dldp = {l: rng.standard_normal(kb[2]) for l in (0, 2, 4)}
    dldb = rng.standard_normal(kb[2])
    mesh = _dev(m, torch.float64)
    g = _vjp(mods, mesh, box, kb, (0, 2, 4), True, i22, i33, dldp, dldb, "fp64")

    def loss(t):
        r = _forward(mods, t, box, kb, (0, 2, 4), True, i22, n0, i33, "fp64")
        return sum(np.dot(dldp[l], r[l]) for l in (0, 2, 4)) + np.dot(dldb, r["B0"])

    for trial in range(3):
        v = torch.tensor(rng.standard_normal((n, n, n)), dtype=torch.float64, device="cuda") * float(m.std())
        eps = 0.1

        def D(e):
            return (loss(mesh + e * v) - loss(mesh - e * v)) / (2 * e)

        fd = (4 * D(eps / 2) - D(eps)) / 3
        an = float((g * v).sum())
        assert fd == pytest.approx(an, rel=1e-7, abs=1e-9 * abs(an)), trial


@pytest.mark.parametrize("assign", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_paint_and_adjoint_match_oracle(mods, assign, prec):
    A, AG, B = mods
    n, box = 32, 100.0
    rng = np.random.default_rng(31 + assign)
    npart = 3000
    pos = rng.random((npart, 3)) * box
    w = 0.5 + rng.random(npart)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tpos = torch.tensor(pos, dtype=dt, device="cuda")
    tw = torch.tensor(w, dtype=dt, device="cuda")
    mesh = AG.paint(tpos, tw, n, box, assign=assign, precision=prec)
    s = OM.grid_coords(tpos.double().cpu().numpy(), (0, 0, 0), box, n)
    ref = OM.paint(s, tw.double().cpu().numpy(), n, assign)
    ref -= ref.mean()
    tol = 1e-12 if prec == "fp64" else 2e-6
    np.testing.assert_allclose(_host(mesh), ref, atol=tol * np.abs(ref).max())
    # adjoint: cotangent mesh G
    G = rng.standard_normal((n, n, n))
    cat = AG._Cat(tpos, tw)
    keep = A._Keep()
    c = A.make_catalog(cat, keep)
    spec = A.make_spec(n, box, (0, 0, 0), assign, 0, 1, (0, 0, 1))
    gpos = torch.empty_like(tpos)
    gw = torch.empty_like(tw)
    tG = _dev(G, dt)
    h = A.context(0)
    B.check(B.npc_paint_adjoint(h, C.byref(spec), C.byref(c), C.c_void_p(tG.data_ptr()), A._prec(prec),
                                C.c_void_p(gpos.data_ptr()), C.c_void_p(gw.data_ptr())), h)
    torch.cuda.synchronize()
    sd = tpos.double().cpu().numpy()
    s = OM.grid_coords(sd, (0, 0, 0), box, n)
    wd = tw.double().cpu().numpy()
    if assign == 3:
        ref_s = OA.tsc_adjoint(s, wd, G)
    else:
        ref_s = _cic_adjoint(s, wd, G)
    ref_x = ref_s * (n / box)
    tol = 1e-11 if prec == "fp64" else 3e-5
    np.testing.assert_allclose(gpos.double().cpu().numpy(), ref_x, atol=tol * np.abs(ref_x).max())
    # dL/dw_p = sum_c G(c) W(c - s_p): one particle at a time through the oracle's painting
    for p in range(0, npart, 500):
        one = OM.paint(s[p:p + 1], np.ones(1), n, assign)
        assert float(gw[p]) == pytest.approx(float(np.sum(G * one)), rel=1e-4 if prec == "mixed" else 1e-11,
                                             abs=1e-6)


def _cic_adjoint(s, w, G):
    """dL/ds for CIC, written out from the window W(d) = 1 - |d| (|d| < 1) per axis."""
    n = G.shape[0]
    i0 = np.floor(s).astype(np.int64)
    d = s - i0
    Wt = [1.0 - d, d]
    dW = [-np.ones_like(d), np.ones_like(d)]
    out = np.zeros_like(s)
    for ox in range(2):
        for oy in range(2):
            for oz in range(2):
                gv = G[(i0[:, 0] + ox) % n, (i0[:, 1] + oy) % n, (i0[:, 2] + oz) % n]
                out[:, 0] += gv * dW[ox][:, 0] * Wt[oy][:, 1] * Wt[oz][:, 2]
                out[:, 1] += gv * Wt[ox][:, 0] * dW[oy][:, 1] * Wt[oz][:, 2]
                out[:, 2] += gv * Wt[ox][:, 0] * Wt[oy][:, 1] * dW[oz][:, 2]
    return out * w[:, None]


def test_autograd_positions_fd_fp64(mods):
    """pos -> paint -> P_l, B_0 -> loss, backward through torch.autograd; central differences of the
    same chain on a few coordinates (TSC is continuously differentiable)."""
    _, AG, _ = mods
    w = workload("adjoint_32")
    n, box = w["n"], w["box"]
    kb = (w["kmin"], w["dk"], w["nbins"])
    cat = make_periodic_catalog(w["n_gal"], box, w["n_gen"], seed=w["seed"], dtype=np.float64)
    pos = torch.tensor(cat.pos, dtype=torch.float64, device="cuda", requires_grad=True)
    wt = torch.tensor(cat.w, dtype=torch.float64, device="cuda", requires_grad=True)
    i22, n0, i33 = AG.periodic_normalisations(pos, wt, box)
    rng = np.random.default_rng(3)
    cp = torch.tensor(rng.standard_normal((3, kb[2])), device="cuda")
    cb = torch.tensor(rng.standard_normal(kb[2]), device="cuda")

    def run(p, ww):
        mesh = AG.paint(p, ww, n, box, assign=3, precision="fp64")
        r = AG.mesh_multipoles(mesh, box, kb, (0, 2, 4), True, i22, n0, i33, precision="fp64")
        return (r["P"] * cp).sum() + (r["B0"] * cb).sum()

    L = run(pos, wt)
    L.backward()
    gpos = pos.grad.double().cpu().numpy()
    gw = wt.grad.double().cpu().numpy()
    eps = 1e-5
    for p in (0, 17, 123, 999):
        for a in range(3):
            with torch.no_grad():
                q = pos.detach().clone()
                q[p, a] += eps
                lp = float(run(q, wt.detach()))
                q[p, a] -= 2 * eps
                lm = float(run(q, wt.detach()))
            fd = (lp - lm) / (2 * eps)
            assert fd == pytest.approx(gpos[p, a], rel=2e-4, abs=1e-6 * np.abs(gpos).max()), (p, a)
        with torch.no_grad():
            v = wt.detach().clone()
            v[p] += eps
            lp = float(run(pos.detach(), v))
            v[p] -= 2 * eps
            lm = float(run(pos.detach(), v))
        assert (lp - lm) / (2 * eps) == pytest.approx(gw[p], rel=2e-4, abs=1e-6 * np.abs(gw).max()), p


def test_rejects(mods):
    A, _, B = mods
    mesh = torch.zeros((32, 32, 32), dtype=torch.float32, device="cuda")
    kbs = B.npc_kbins(0.1, 0.1, 4)
    h = A.context(0)
    out = np.zeros(64)
    for spec in (A.make_spec(32, 93.75, (0, 0, 0), 3, 1, 1, (0, 0, 1)),     # interlaced
                 A.make_spec(32, 93.75, (0, 0, 0), 3, 0, 0, (0, 0, 1)),     # survey
                 A.make_spec(32, 93.75, (0, 0, 0), 3, 0, 1, None)):         # endpoint LOS
        st = B.npc_mesh_multipoles(h, C.byref(spec), C.c_void_p(mesh.data_ptr()), C.byref(kbs), 1, 0, 1.0, 0.0,
                                   1.0, B.NPC_PREC_MIXED, out.ctypes.data_as(C.c_void_p), 0)
        assert st == 4
    spec = A.make_spec(32, 93.75, (0, 0, 0), 3, 0, 1, (0, 0, 1))
    big = B.npc_kbins(0.1, 0.2, 4)   # k_max = 0.9 > k_N/2
    st = B.npc_mesh_multipoles(h, C.byref(spec), C.c_void_p(mesh.data_ptr()), C.byref(big), 0, 1, 1.0, 0.0, 1.0,
                               B.NPC_PREC_MIXED, out.ctypes.data_as(C.c_void_p), 0)
    assert st == 4
    st = B.npc_mesh_multipoles(h, C.byref(spec), None, C.byref(kbs), 1, 0, 1.0, 0.0, 1.0, B.NPC_PREC_MIXED,
                               out.ctypes.data_as(C.c_void_p), 0)
    assert st == 1
    st = B.npc_mesh_multipoles(h, C.byref(spec), C.c_void_p(mesh.data_ptr()), C.byref(kbs), 1, 0, -1.0, 0.0, 1.0,
                               B.NPC_PREC_MIXED, out.ctypes.data_as(C.c_void_p), 0)
    assert st == 6


def test_mesh_power_agrees_with_catalogue_path(mods):
    """P_l of the painted mesh equals npc_power_multipoles on the same periodic catalogue (no
    interlacing, global LOS), which paints and transforms along its own path."""
    A, AG, _ = mods
    n, box = 64, 500.0
    kb = (0.0, 0.02, 12)
    cat = make_periodic_catalog(200_000, box, 64, seed=77, dtype=np.float32)
    ref = A.power_multipoles(cat, None, n=n, box=box, assign=3, interlace=0, kbins=kb, ells=(0, 2, 4),
                             precision="mixed", los_dir=(0, 0, 1))
    sc = ref["scalars"]
    pos = torch.tensor(cat.pos, device="cuda")
    mesh = AG.paint(pos, None, n, box, assign=3, precision="mixed")
    r = AG.mesh_multipoles(mesh, box, kb, (0, 2, 4), False, sc["I22"], sc["N0"], 1.0, precision="mixed")
    P = r["P"].cpu().numpy()
    scale = np.abs(ref["P"][0]) + sc["N0"]
    for e, l in enumerate((0, 2, 4)):
        assert np.max(np.abs(P[e] - ref["P"][l]) / scale) < 1e-5, l
    np.testing.assert_allclose(r["k_eff"].cpu().numpy(), ref["k_eff"], rtol=1e-6)


@pytest.mark.slow
def test_full_size_1024(mods):
    """Periodic 1024^3, 1e7 lognormal galaxies, P_0,2,4 and B_0 on 19 bins: the gradient with respect
    to the mesh against directional differences of the forward values (exact for the quadratic P
    part, one Richardson step for the cubic B_0 part), and the position gradient against the
    adjoint identity sum_p grad_pos . u_p = d/dt L(pos + t u)."""
    _, AG, _ = mods
    w = workload("adjoint_1024")
    n, box = w["n"], w["box"]
    kb = (w["kmin"], w["dk"], w["nbins"])
    cat = make_periodic_catalog(w["n_gal"], box, w["n_gen"], seed=w["seed"], dtype=np.float32)
    pos = torch.tensor(cat.pos, device="cuda")
    i22, n0, i33 = AG.periodic_normalisations(pos, None, box)
    mesh = AG.paint(pos, None, n, box, assign=3, precision="mixed")
    rng = np.random.default_rng(4)
    cp = torch.tensor(rng.standard_normal((3, kb[2])), device="cuda")
    cb = torch.tensor(rng.standard_normal(kb[2]), device="cuda")

    def loss(m):
        r = AG.mesh_multipoles(m, box, kb, (0, 2, 4), True, i22, n0, i33, precision="mixed")
        return float((r["P"] * cp).sum() + (r["B0"] * cb).sum()), r

    m = mesh.detach().requires_grad_(True)
    r = AG.mesh_multipoles(m, box, kb, (0, 2, 4), True, i22, n0, i33, precision="mixed")
    assert torch.all(r["nmodes"] > 0) and torch.all(r["NT"] > 0)
    ((r["P"] * cp).sum() + (r["B0"] * cb).sum()).backward()
    g = m.grad
    gen = torch.Generator(device="cuda").manual_seed(1)
    v = torch.randn(m.shape, device="cuda", generator=gen) * mesh.std()
    an = float((g.double() * v.double()).sum())
    eps = 0.25

    def D(e):
        return (loss(mesh + e * v)[0] - loss(mesh - e * v)[0]) / (2 * e)

    fd = (4 * D(eps / 2) - D(eps)) / 3
    assert fd == pytest.approx(an, rel=2e-3)
    del g, v
    torch.cuda.empty_cache()


def test_single_purpose_entry_points(mods):
    """npc_power_vjp, npc_bispec0_vjp and npc_tsc_adjoint equal the general calls bit for bit."""
    A, _, B = mods
    n, box = 32, 400.0
    m, cat = _oracle_mesh(n, box, 20000, seed=171)
    mesh = _dev(m, torch.float32)
    kb = (0.02, 0.02, 5)
    i22, i33 = 1.7e3, 2.3e5
    rng = np.random.default_rng(5)
    dldp = {l: rng.standard_normal(kb[2]) for l in (0, 2)}
    dldb = rng.standard_normal(kb[2])
    spec = A.make_spec(n, box, (0, 0, 0), 3, 0, 1, (0.0, 0.0, 1.0))
    kbs = B.npc_kbins(*kb)
    h = A.context(0)
    g_ref = _vjp(mods, mesh, box, kb, (0, 2), False, i22, i33, dldp, None, "mixed")
    g = torch.empty_like(mesh)
    dp = np.ascontiguousarray(np.stack([dldp[0], dldp[2]]))
    B.check(B.npc_power_vjp(h, C.c_void_p(mesh.data_ptr()), C.byref(spec), C.byref(kbs), 5, i22,
                            dp.ctypes.data_as(C.c_void_p), C.c_void_p(g.data_ptr())), h)
    torch.cuda.synchronize()
    assert torch.equal(g, g_ref)
    g_ref = _vjp(mods, mesh, box, kb, (), True, i22, i33, {}, dldb, "mixed")
    db = np.ascontiguousarray(dldb)
    B.check(B.npc_bispec0_vjp(h, C.c_void_p(mesh.data_ptr()), C.byref(spec), C.byref(kbs), i33,
                              db.ctypes.data_as(C.c_void_p), C.c_void_p(g.data_ptr())), h)
    torch.cuda.synchronize()
    assert torch.equal(g, g_ref)
    # TSC adjoint against the general paint adjoint
    pos = torch.tensor(cat.pos, dtype=torch.float32, device="cuda")
    w = torch.tensor(cat.w, dtype=torch.float32, device="cuda")
    from types import SimpleNamespace

    keep = A._Keep()
    dc = A.make_catalog(SimpleNamespace(pos=pos, w=w, nbar=None), keep)
    gp_ref = torch.zeros_like(pos)
    gw = torch.zeros_like(w)
    B.check(B.npc_paint_adjoint(h, C.byref(spec), C.byref(dc), C.c_void_p(mesh.data_ptr()), A._prec("mixed"),
                                C.c_void_p(gp_ref.data_ptr()), C.c_void_p(gw.data_ptr())), h)
    gp = torch.zeros_like(pos)
    B.check(B.npc_tsc_adjoint(h, C.byref(spec), C.byref(dc), C.c_void_p(mesh.data_ptr()), C.c_void_p(gp.data_ptr())),
            h)
    torch.cuda.synchronize()
    assert torch.equal(gp, gp_ref)
