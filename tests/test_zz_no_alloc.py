"""The allocation-free catalogue-scalar entry point, called through the C ABI, reproduces the
context entry point (npc_catalog_scalars) on the same device-resident catalogues, on two calls in
a row.  This file sorts last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import ensure_built
from synthetic import make_periodic_catalog, make_survey_catalogs

pytestmark = pytest.mark.gpu


def _dev_catalog(B, cat, torch, dtype):
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(cat, k), dtype=dtype)).cuda() for k in ("pos", "w", "nbar")}
    c = B.npc_catalog()
    c.pos, c.w, c.nbar = t["pos"].data_ptr(), t["w"].data_ptr(), t["nbar"].data_ptr()
    c.n = t["pos"].shape[0]
    c.dtype = 1 if dtype == np.float64 else 0
    c.on_device = 1
    return c, t


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_matches_context_entry_point(dtype):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_built()
    from paper_2605_04864_gb300 import binding as B

    torch.cuda.set_device(0)
    g, r, _ = make_survey_catalogs(60000, 600000, 800.0, 1300.0, 32, seed=91, fkp_p0=1e4)
    per = make_periodic_catalog(50000, 500.0, 32, seed=92)
    dg, keep1 = _dev_catalog(B, g, torch, dtype)
    dr, keep2 = _dev_catalog(B, r, torch, dtype)
    dp, keep3 = _dev_catalog(B, per, torch, dtype)
    ctx = C.c_void_p()
    B.check(B.npc_create(C.byref(ctx), 0, None))
    try:
        for data, rand, box in ((dg, dr, 800.0), (dp, None, 500.0)):
            ref = torch.zeros(8, dtype=torch.float64, device="cuda")
            B.check(B.npc_catalog_scalars(ctx, C.byref(data), C.byref(rand) if rand else None, box,
                                          C.c_void_p(ref.data_ptr()), 1), ctx)
            torch.cuda.synchronize()
            want = ref.cpu().numpy()
            for _ in range(2):   # two calls in a row share the static scratch
                got = torch.full((8,), np.nan, dtype=torch.float64, device="cuda")
                err = C.create_string_buffer(256)
                st = B.npc_catalog_scalars_noalloc(C.byref(data), C.byref(rand) if rand else None, box,
                                                   C.c_void_p(got.data_ptr()), None, err, 256)
                assert st == 0, err.value
                torch.cuda.synchronize()
                np.testing.assert_allclose(got.cpu().numpy(), want, rtol=1e-12, atol=0)
    finally:
        B.npc_destroy(ctx)
    del keep1, keep2, keep3


def test_noalloc_many_blocks():
    """5.5e6 objects: the call reduces over more blocks (1,221) than the context call's fixed 1,024,
    so the two trees differ; the results still agree to rounding, and two calls agree bit for bit."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_built()
    from paper_2605_04864_gb300 import binding as B

    torch.cuda.set_device(0)
    g, r, _ = make_survey_catalogs(500_000, 5_000_000, 1500.0, 2000.0, 32, seed=93, fkp_p0=1e4)
    dg, keep1 = _dev_catalog(B, g, torch, np.float32)
    dr, keep2 = _dev_catalog(B, r, torch, np.float32)
    ctx = C.c_void_p()
    B.check(B.npc_create(C.byref(ctx), 0, None))
    try:
        ref = torch.zeros(8, dtype=torch.float64, device="cuda")
        B.check(B.npc_catalog_scalars(ctx, C.byref(dg), C.byref(dr), 1500.0, C.c_void_p(ref.data_ptr()), 1), ctx)
        torch.cuda.synchronize()
        want = ref.cpu().numpy()
        outs = []
        for _ in range(2):
            got = torch.full((8,), np.nan, dtype=torch.float64, device="cuda")
            err = C.create_string_buffer(256)
            st = B.npc_catalog_scalars_noalloc(C.byref(dg), C.byref(dr), 1500.0, C.c_void_p(got.data_ptr()),
                                               None, err, 256)
            assert st == 0, err.value
            torch.cuda.synchronize()
            outs.append(got.cpu().numpy())
            np.testing.assert_allclose(outs[-1], want, rtol=1e-12, atol=0)
        np.testing.assert_array_equal(outs[0], outs[1])
    finally:
        B.npc_destroy(ctx)
    del keep1, keep2


def test_noalloc_rejects_host_pointers_and_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_built()
    from paper_2605_04864_gb300 import binding as B

    torch.cuda.set_device(0)
    host = np.ones((10, 3), np.float32)
    c = B.npc_catalog()
    c.pos, c.n, c.dtype, c.on_device = host.ctypes.data, 10, 0, 0
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    err = C.create_string_buffer(256)
    assert B.npc_catalog_scalars_noalloc(C.byref(c), None, 10.0, C.c_void_p(out.data_ptr()), None, err, 256) == 1
    assert b"device" in err.value
    dev = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    c = B.npc_catalog()
    c.pos, c.n, c.dtype, c.on_device = dev.data_ptr(), 40_000_000, 0, 1
    assert B.npc_catalog_scalars_noalloc(C.byref(c), None, 10.0, C.c_void_p(out.data_ptr()), None, err, 256) == 1
    assert b"capacity" in err.value
