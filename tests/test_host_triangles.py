"""The library's triangle and pair lists (host code of the C ABI, no GPU needed) against the oracle's,
index by index, over binnings with and without flat triangles (bin centres with c_k = c_i + c_j)."""
import ctypes as C

import numpy as np
import pytest

from helpers import ensure_built
from oracle import bispec as OB


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2605_04864_gb300 import binding

    return binding


BINNINGS = [(0.01, 0.01, 19),            # the 256^3 workload: 805 triangles
            (0.0, 0.01, 24), (0.0, 0.02, 1), (0.0, 0.02, 2),
            (0.005, 0.01, 24),            # kmin = dk/2: flat triangles sit exactly on the rule
            (0.0037, 0.0113, 17), (0.013, 0.017, 7), (0.3, 0.05, 12), (0.02, 0.03, 3)]


@pytest.mark.parametrize("kb", BINNINGS)
def test_triangles_match_the_oracle(B, kb):
    want = OB.triangles(kb)
    bins = B.npc_kbins(*kb)
    nt = C.c_int64(-1)
    cap = max(len(want), 1) + 4
    buf = (C.c_int32 * (3 * cap))()
    assert B.npc_bispectrum_triangles(C.byref(bins), buf, cap, C.byref(nt)) == 0
    got = np.frombuffer(buf, dtype=np.int32)[: 3 * nt.value].reshape(-1, 3)
    np.testing.assert_array_equal(got, want)
    ntri, npair, length = C.c_int64(-1), C.c_int64(-1), C.c_int64(-1)
    assert B.npc_bispectrum_layout(C.byref(bins), 0b101, 0b101, C.byref(ntri), C.byref(npair),
                                   C.byref(length)) == 0
    assert ntri.value == len(want)
    assert npair.value == len(OB.pairs(kb))
    if kb == (0.01, 0.01, 19):
        assert len(want) == 805


def test_flat_triangles_are_closed():
    """With bins starting at dk/2 the centres are whole multiples of dk, so c_k = c_i + c_j happens;
    both sides count such a flat triangle as closed (the bin-centre reading of the paper's closed
    triangles)."""
    kb = (0.005, 0.01, 6)
    want = OB.triangles(kb)
    c = [kb[0] + (b + 0.5) * kb[1] for b in range(kb[2])]
    flat = [tuple(t) for t in want if abs(c[t[2]] - c[t[0]] - c[t[1]]) < 1e-12]
    assert (0, 0, 1) in flat and (0, 1, 2) in flat


def test_capacity_too_small_is_reported(B):
    """A buffer smaller than the triangle count is left untouched: the call returns NPC_ERR_INVALID_ARG
    with the count needed; a NULL buffer only asks for the count."""
    kb = (0.01, 0.01, 19)
    bins = B.npc_kbins(*kb)
    nt = C.c_int64(-1)
    buf = (C.c_int32 * (3 * 10 + 3))()
    guard = 0x5A5A5A5A
    buf[30], buf[31], buf[32] = guard, guard, guard
    st = B.npc_bispectrum_triangles(C.byref(bins), buf, 10, C.byref(nt))
    assert st == 1 and nt.value == 805
    assert (buf[30], buf[31], buf[32]) == (guard, guard, guard)
    assert all(buf[i] == 0 for i in range(30))
    nt2 = C.c_int64(-1)
    assert B.npc_bispectrum_triangles(C.byref(bins), None, 0, C.byref(nt2)) == 0 and nt2.value == 805
