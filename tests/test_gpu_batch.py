"""GPU: batches of uneven mocks (npc_batch_run) -- every item equals its single call bit for bit,
graph replays equal the eager run, refilled catalogues are picked up by replays, the autotuner
keeps a valid configuration; one survey item is also checked against the FP64 oracle."""
from types import SimpleNamespace

import numpy as np
import pytest

from helpers import ensure_built
from synthetic import make_periodic_catalog, make_survey_catalogs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    ensure_built()
    from paper_2605_04864_gb300 import api as A

    return A


def _dev(c):
    return SimpleNamespace(pos=torch.from_numpy(np.ascontiguousarray(c.pos)).cuda(),
                           w=torch.from_numpy(np.ascontiguousarray(c.w)).cuda(),
                           nbar=torch.from_numpy(np.ascontiguousarray(c.nbar)).cuda())


def _items():
    """Survey and periodic mocks on 32^3, 48^3 (radix 3) and 64^3 meshes, with and without B_0."""
    out = []
    for i, (n, box, survey, nb_b) in enumerate([(32, 600.0, True, 3), (48, 500.0, False, 5), (64, 900.0, True, 0),
                                               (32, 300.0, False, 3), (48, 700.0, True, 4), (64, 400.0, False, 6)]):
        kf = 2 * np.pi / box
        pk = (0.0, 2 * kf, max(3, int(n / 2 / 2 / 2)))
        bk = (2 * kf, 1.5 * kf, nb_b) if nb_b else None
        if survey:
            g, r, origin = make_survey_catalogs(3000 + 700 * i, 30000 + 7000 * i, box, 1.5 * box, 16, seed=500 + i,
                                                fkp_p0=1e4)
            out.append(dict(n=n, box=box, origin=tuple(origin), data=_dev(g), randoms=_dev(r), power_bins=pk,
                            bispec_bins=bk, host=(g, r, origin)))
        else:
            c = make_periodic_catalog(4000 + 900 * i, box, 16, seed=600 + i)
            out.append(dict(n=n, box=box, data=_dev(c), power_bins=pk, bispec_bins=bk, los_dir=(0, 0, 1),
                            host=(c, None, (0.0, 0.0, 0.0))))
    return out


def _single(api, it, ells, prec):
    """The item through the single-measurement calls (device outputs)."""
    n, box = it["n"], it["box"]
    rnd = it.get("randoms")
    p = api.power_multipoles(it["data"], rnd, n=n, box=box, origin=it.get("origin", (0, 0, 0)), assign=3,
                             interlace=1, kbins=it["power_bins"], ells=ells, precision=prec,
                             los_dir=it.get("los_dir"))
    b = None
    if it.get("bispec_bins"):
        b = api.bispectrum(it["data"], n=n, box=box, kbins=it["bispec_bins"], scoc_ells=(0,), tripo_ells=(),
                           precision=prec, origin=it.get("origin", (0, 0, 0)), randoms=rnd,
                           los_dir=it.get("los_dir") or (0.0, 0.0, 1.0))
    return p, b


def _flat_power(p, nb, ells):
    rows = [p["k_eff"], p["nmodes"]] + [p["P"][l] for l in sorted(ells)]
    sc = [p["scalars"][k] for k in ("alpha", "I22", "I33", "N0", "S3", "sum_wg", "sum_wr", "sum_w2")]
    return np.concatenate([np.concatenate(rows), np.array(sc)])


def _flat_bispec(b):
    sc = [b["scalars"][k] for k in ("alpha", "I22", "I33", "N0", "S3", "sum_wg", "sum_wr", "sum_w2")]
    return np.concatenate([b["B"][0], b["shot_B"][0], b["NT"], b["nmodes"], np.array(sc)])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_equals_single_calls(api, prec):
    items = _items()
    arr, keep = api.make_batch(items)
    total, offs = api.batch_layout(arr)
    assert total > 0
    ells = (0, 2, 4)
    for graph in (False, True, True):    # eager, warm + capture, replay
        out = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        api.batch_run(arr, out, ells, precision=prec, graph=graph)
        torch.cuda.synchronize()
        res = out.cpu().numpy()
        for it, (op, ob) in zip(items, offs):
            p, b = _single(api, it, ells, prec)
            fp = _flat_power(p, it["power_bins"][2], ells)
            np.testing.assert_array_equal(res[op:op + len(fp)], fp)
            if b is not None:
                fb = _flat_bispec(b)
                np.testing.assert_array_equal(res[ob:ob + len(fb)], fb)
            else:
                assert ob == -1
    del keep


def test_graph_replay_sees_refilled_catalogues(api):
    items = _items()
    arr, keep = api.make_batch(items)
    total, offs = api.batch_layout(arr)
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    api.batch_run(arr, out, graph=True)
    api.batch_run(arr, out, graph=True)
    # new positions for item 1 (periodic), written in place
    it = items[1]
    c = make_periodic_catalog(it["data"].pos.shape[0], it["box"], 16, seed=999)
    it["data"].pos.copy_(torch.from_numpy(c.pos))
    api.batch_run(arr, out, graph=True)           # replay of the captured graph
    torch.cuda.synchronize()
    p, b = _single(api, it, (0, 2, 4), "mixed")
    op, ob = offs[1]
    fp = _flat_power(p, it["power_bins"][2], (0, 2, 4))
    np.testing.assert_array_equal(out.cpu().numpy()[op:op + len(fp)], fp)
    fb = _flat_bispec(b)
    np.testing.assert_array_equal(out.cpu().numpy()[ob:ob + len(fb)], fb)
    del keep


def test_tuner_and_branches(api):
    items = _items()
    arr, keep = api.make_batch(items)
    total, offs = api.batch_layout(arr)
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    path = api.get_option("tcgen05_triple")
    nb = api.batch_tune(arr, out)   # sets the context's triple-product path to the faster one
    assert nb in (1, 2, 4, 6)
    assert api.get_option("tcgen05_triple") in (0, 1)
    ref = torch.zeros_like(out)
    api.batch_set_branches(1)
    api.batch_run(arr, ref, graph=False)
    for b in (2, 3, 6):
        api.batch_set_branches(b)
        api.batch_run(arr, out, graph=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    api.batch_set_branches(0)
    api.set_option("tcgen05_triple", path)   # leave the context as the other tests expect
    del keep


def test_survey_item_matches_oracle(api):
    from oracle import bispec as OB
    from oracle import power as P

    items = _items()[:1]
    arr, keep = api.make_batch(items)
    total, offs = api.batch_layout(arr)
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    api.batch_run(arr, out, precision="fp64")
    res = out.cpu().numpy()
    it = items[0]
    g, r, origin = it["host"]
    spec = dict(n=it["n"], box=it["box"], origin=tuple(origin), assign=3, interlace=1, los="endpoint",
                observer=(0.0, 0.0, 0.0))
    orc = P.power_multipoles(spec, g, r, it["power_bins"], (0, 2, 4), (), method="plain")
    nb = it["power_bins"][2]
    op, ob = offs[0]
    scale = np.abs(orc["P"][0]) + orc["scalars"]["N0"]
    for e, l in enumerate((0, 2, 4)):
        got = res[op + (2 + e) * nb:op + (3 + e) * nb]
        assert np.max(np.abs(got - orc["P"][l]) / scale) < 1e-12
    bspec = dict(n=it["n"], box=it["box"], origin=tuple(origin), assign=3, interlace=1, los="global",
                 los_dir=(0.0, 0.0, 1.0), periodic=0)
    ob_orc = OB.bispectrum(bspec, g, r, it["bispec_bins"], (0,), (), shot=True)
    ntri = len(ob_orc["tri"])
    B0 = res[ob:ob + ntri]
    shot = res[ob + ntri:ob + 2 * ntri]
    scale_t = np.abs(ob_orc["B"][0]) + np.abs(ob_orc["shot_B"][0])
    assert np.max(np.abs(B0 + shot - ob_orc["B"][0]) / scale_t) < 1e-10
    assert np.max(np.abs(shot - ob_orc["shot_B"][0]) / scale_t) < 1e-10
    del keep


def test_batch_rejects(api):
    items = _items()[:2]
    arr, keep = api.make_batch(items)
    total, _ = api.batch_layout(arr)
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    arr[0].data.on_device = 0
    with pytest.raises(api.B.NpcError):
        api.batch_run(arr, out)
    arr[0].data.on_device = 1
    arr[1].bispec_bins.dk = 1.0          # beyond k_N/2
    with pytest.raises(api.B.NpcError) as ei:
        api.batch_run(arr, out)
    assert ei.value.status == 4
    del keep
