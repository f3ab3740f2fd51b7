"""Host-side layout logic of the Python front end against the lengths the C ABI reports (no GPU)."""
import ctypes as C

import numpy as np

from helpers import ensure_built


def _api():
    ensure_built()
    from paper_2605_04864_gb300 import api as A
    from paper_2605_04864_gb300 import binding as B

    return A, B


def test_unpack_sugiyama_covers_the_abi_length():
    A, B = _api()
    kbins = (0.01, 0.01, 7)
    mps = [(0, 0, 0), (2, 0, 2), (1, 1, 2)]
    kb = B.npc_kbins(*kbins[:2], kbins[2])
    length = B.npc_bispectrum_sugiyama_len(C.byref(kb), len(mps))
    assert length == 2 * 3 * 49 + 7 + 8
    buf = np.arange(length, dtype=np.float64)
    res = A.unpack_sugiyama(buf, kbins, mps)
    # B blocks, then shot blocks, row k1 = bin i, column k2 = bin j
    assert res["B"][(0, 0, 0)][2, 5] == 2 * 7 + 5
    assert res["B"][(1, 1, 2)][0, 0] == 2 * 49
    assert res["shot"][(0, 0, 0)][0, 1] == 3 * 49 + 1
    assert res["shot"][(1, 1, 2)][6, 6] == 6 * 49 - 1
    np.testing.assert_array_equal(res["nmodes"], np.arange(6 * 49, 6 * 49 + 7))
    assert res["scalars"]["alpha"] == 6 * 49 + 7 and res["scalars"]["sum_w2"] == length - 1


def test_unpack_bispectrum_covers_the_abi_length():
    A, B = _api()
    kbins = (0.01, 0.01, 5)
    kb = B.npc_kbins(*kbins[:2], kbins[2])
    ntri, npair, length = C.c_int64(), C.c_int64(), C.c_int64()
    assert B.npc_bispectrum_layout(C.byref(kb), 5, 5, C.byref(ntri), C.byref(npair), C.byref(length)) == 0
    nt, npr = ntri.value, npair.value
    assert npr == 15 and length.value == 5 * nt + 4 * npr + 5 + 8
    buf = np.arange(length.value, dtype=np.float64)
    res = A.unpack_bispectrum(buf, kbins, (0, 2), (0, 2))
    assert res["B"][2][0] == nt and res["shot_B"][0][0] == 2 * nt and res["NT"][0] == 4 * nt
    assert res["BB"][0][0] == 5 * nt and res["shot_BB"][2][-1] == 5 * nt + 4 * npr - 1
    assert res["scalars"]["alpha"] == 5 * nt + 4 * npr + 5
    assert len(res["tri"]) == nt
