"""ctypes binding of libnpc.so: the C ABI declared in include/npc.h, names unchanged.

Argument marshalling only.  Every step of the estimators runs in the library's CUDA kernels; if
the shared library is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnpc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
lib = C.CDLL(LIB_PATH)

NPC_OK = 0
STATUS = {0: "NPC_OK", 1: "NPC_ERR_INVALID_ARG", 2: "NPC_ERR_OOM", 3: "NPC_ERR_CUDA",
          4: "NPC_ERR_UNSUPPORTED", 5: "NPC_ERR_TIMEOUT", 6: "NPC_ERR_NUMERIC"}
NPC_PREC_FP64 = 0
NPC_PREC_MIXED = 1


class npc_mesh_spec(C.Structure):
    _fields_ = [("n", C.c_int32), ("box", C.c_double), ("origin", C.c_double * 3),
                ("assign", C.c_int32), ("interlace", C.c_int32), ("periodic", C.c_int32),
                ("los", C.c_int32), ("los_dir", C.c_double * 3), ("observer", C.c_double * 3)]


class npc_catalog(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("w", C.c_void_p), ("nbar", C.c_void_p), ("n", C.c_int64),
                ("dtype", C.c_int32), ("on_device", C.c_int32)]


class npc_kbins(C.Structure):
    _fields_ = [("kmin", C.c_double), ("dk", C.c_double), ("nbins", C.c_int32)]


class npc_batch_item(C.Structure):
    _fields_ = [("mesh", npc_mesh_spec), ("data", npc_catalog), ("randoms", npc_catalog),
                ("power_bins", npc_kbins), ("bispec_bins", npc_kbins)]


NPC_BATCH_GRAPH = 1


class npc_stats(C.Structure):
    _fields_ = [("n_transforms", C.c_int32), ("n_r2c_equivalent", C.c_int32), ("n_phases", C.c_int32),
                ("n_kernel_launches", C.c_int32), ("workspace_bytes", C.c_int64),
                ("contraction_flops", C.c_double), ("contraction_launches", C.c_int32), ("reserved", C.c_int32),
                ("contraction_issued_flops", C.c_double)]


_P = C.POINTER
_sig = {
    "npc_create": (C.c_int, [_P(C.c_void_p), C.c_int, C.c_void_p]),
    "npc_destroy": (C.c_int, [C.c_void_p]),
    "npc_status_string": (C.c_char_p, [C.c_int]),
    "npc_last_error": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t]),
    "npc_version": (C.c_char_p, []),
    "npc_last_stats": (C.c_int, [C.c_void_p, _P(npc_stats)]),
    "npc_device_status": (C.c_int, [C.c_void_p]),
    "npc_set_wait_limit": (C.c_int, [C.c_void_p, C.c_longlong]),
    "npc_set_option": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int64]),
    "npc_get_option": (C.c_int, [C.c_void_p, C.c_char_p, _P(C.c_int64)]),
    "npc_catalog_scalars": (C.c_int, [C.c_void_p, _P(npc_catalog), _P(npc_catalog), C.c_double,
                                      C.c_void_p, C.c_int32]),
    "npc_power_multipoles": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), _P(npc_catalog),
                                       _P(npc_kbins), C.c_uint32, C.c_uint32, C.c_int, C.c_void_p,
                                       C.c_int32]),
    "npc_power_out_len": (C.c_int64, [_P(npc_kbins), C.c_uint32, C.c_uint32]),
    "npc_cross_power_multipoles": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), _P(npc_catalog),
                                             _P(npc_catalog), _P(npc_catalog), _P(npc_kbins), C.c_uint32, C.c_int,
                                             C.c_void_p, C.c_int32]),
    "npc_bispectrum": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), _P(npc_catalog),
                                 _P(npc_kbins), C.c_uint32, C.c_uint32, C.c_int32, C.c_int, C.c_void_p,
                                 C.c_int32]),
    "npc_cross_bispectrum": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), _P(npc_catalog),
                                       _P(npc_kbins), C.c_uint32, C.c_uint32, C.c_int, C.c_void_p, C.c_int32]),
    "npc_bispectrum_layout": (C.c_int, [_P(npc_kbins), C.c_uint32, C.c_uint32, _P(C.c_int64),
                                        _P(C.c_int64), _P(C.c_int64)]),
    "npc_bispectrum_triangles": (C.c_int, [_P(npc_kbins), _P(C.c_int32), C.c_int64, _P(C.c_int64)]),
    "npc_bispectrum_sugiyama": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), _P(npc_catalog),
                                          _P(npc_kbins), C.c_int32, _P(C.c_int32), C.c_int32, C.c_int,
                                          C.c_void_p, C.c_int32]),
    "npc_bispectrum_sugiyama_len": (C.c_int64, [_P(npc_kbins), C.c_int32]),
    "npc_catalog_scalars_noalloc": (C.c_int, [_P(npc_catalog), _P(npc_catalog), C.c_double, C.c_void_p,
                                              C.c_void_p, C.c_char_p, C.c_size_t]),
    "npc_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "npc_batch_layout": (C.c_int64, [C.c_int32, _P(npc_batch_item), C.c_uint32, _P(C.c_int64)]),
    "npc_batch_run": (C.c_int, [C.c_void_p, C.c_int32, _P(npc_batch_item), C.c_uint32, C.c_int, C.c_void_p,
                                C.c_int32]),
    "npc_batch_tune": (C.c_int, [C.c_void_p, C.c_int32, _P(npc_batch_item), C.c_uint32, C.c_int, C.c_void_p,
                                 _P(C.c_int32)]),
    "npc_batch_set_branches": (C.c_int, [C.c_void_p, C.c_int32]),
    "npc_tune_transforms": (C.c_int, [C.c_void_p, C.c_int32, C.c_int]),
    "npc_mesh_multipoles_len": (C.c_int64, [_P(npc_kbins), C.c_uint32, C.c_int32]),
    "npc_mesh_multipoles": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), C.c_void_p, _P(npc_kbins), C.c_uint32,
                                      C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int, C.c_void_p,
                                      C.c_int32]),
    "npc_mesh_multipoles_vjp": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), C.c_void_p, _P(npc_kbins), C.c_uint32,
                                          C.c_int32, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_int32,
                                          C.c_int, C.c_void_p]),
    "npc_paint_mesh": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), C.c_int, C.c_void_p]),
    "npc_paint_adjoint": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), C.c_void_p, C.c_int,
                                    C.c_void_p, C.c_void_p]),
    "npc_power_vjp": (C.c_int, [C.c_void_p, C.c_void_p, _P(npc_mesh_spec), _P(npc_kbins), C.c_uint32, C.c_double,
                                C.c_void_p, C.c_void_p]),
    "npc_bispec0_vjp": (C.c_int, [C.c_void_p, C.c_void_p, _P(npc_mesh_spec), _P(npc_kbins), C.c_double,
                                  C.c_void_p, C.c_void_p]),
    "npc_tsc_adjoint": (C.c_int, [C.c_void_p, _P(npc_mesh_spec), _P(npc_catalog), C.c_void_p, C.c_void_p]),
    "npc_stage_times": (C.c_int, [C.c_void_p, C.c_char_p, _P(C.c_double), _P(C.c_int32), C.c_int32,
                                  _P(C.c_int32)]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_sig)


class NpcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def check(status, ctx=None):
    if status != NPC_OK:
        msg = ""
        if ctx is not None:
            buf = C.create_string_buffer(1024)
            npc_last_error(ctx, buf, 1024)
            msg = buf.value.decode(errors="replace")
        raise NpcError(status, msg or npc_status_string(status).decode())
