"""Python front end over the C ABI: builds the C structs from NumPy arrays or torch tensors,
calls the library, and reshapes the flat output.  PyTorch supplies device memory and the current
CUDA stream; no estimator arithmetic happens here.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B

_CTX = {}


def _stream_ptr(device):
    try:
        import torch

        if torch.cuda.is_available():
            # torch's default stream is the legacy default stream (handle 0); the library takes
            # NULL to mean "own stream", so pass cudaStreamLegacy (0x1) explicitly
            return C.c_void_p(torch.cuda.current_stream(device).cuda_stream or 1)
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return C.c_void_p(0)


def context(device=0):
    """A library context bound to ``device`` and torch's current stream on it (cached)."""
    stream = _stream_ptr(device)
    key = (device, stream.value)
    if key not in _CTX:
        h = C.c_void_p()
        B.check(B.npc_create(C.byref(h), device, stream))
        _CTX[key] = h
    return _CTX[key]


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class _Keep:
    """Holds converted arrays alive for the duration of a call."""

    def __init__(self):
        self.refs = []

    def keep(self, x):
        self.refs.append(x)
        return x


def make_catalog(cat, keep, dtype=None):
    """npc_catalog from an object with .pos/.w/.nbar (NumPy or torch; device tensors stay on device)."""
    if cat is None:
        return None
    pos, w, nbar = cat.pos, getattr(cat, "w", None), getattr(cat, "nbar", None)
    c = B.npc_catalog()
    if _is_torch(pos):
        import torch

        dt = pos.dtype
        assert dt in (torch.float32, torch.float64)
        for t in (pos, w, nbar):
            if t is not None:
                assert t.dtype == dt and t.is_contiguous() and t.device == pos.device
        c.pos = pos.data_ptr() if pos.numel() else None
        c.w = w.data_ptr() if w is not None and w.numel() else None
        c.nbar = nbar.data_ptr() if nbar is not None and nbar.numel() else None
        c.n = pos.shape[0]
        c.dtype = 1 if dt == torch.float64 else 0
        c.on_device = 1 if pos.is_cuda else 0
        keep.keep((pos, w, nbar))
        return c
    dt = np.dtype(dtype or np.asarray(pos).dtype)
    if dt not in (np.float32, np.float64):
        dt = np.dtype(np.float64)
    pos = keep.keep(np.ascontiguousarray(pos, dtype=dt).reshape(-1, 3))
    c.pos = pos.ctypes.data if pos.size else None
    if w is not None:
        w = keep.keep(np.ascontiguousarray(w, dtype=dt))
        c.w = w.ctypes.data
    if nbar is not None:
        nbar = keep.keep(np.ascontiguousarray(nbar, dtype=dt))
        c.nbar = nbar.ctypes.data
    c.n = pos.shape[0]
    c.dtype = 1 if dt == np.float64 else 0
    c.on_device = 0
    return c


def make_spec(n, box, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, periodic=0, los_dir=None,
              observer=(0.0, 0.0, 0.0)):
    s = B.npc_mesh_spec()
    s.n, s.box = int(n), float(box)
    s.origin[:] = [float(v) for v in origin]
    s.assign, s.interlace, s.periodic = int(assign), int(interlace), int(periodic)
    if los_dir is None:
        s.los = 0
        s.los_dir[:] = [0.0, 0.0, 1.0]
    else:
        s.los = 1
        s.los_dir[:] = [float(v) for v in los_dir]
    s.observer[:] = [float(v) for v in observer]
    return s


def _prec(p):
    return {"fp64": B.NPC_PREC_FP64, "mixed": B.NPC_PREC_MIXED}[p] if isinstance(p, str) else int(p)


def power_multipoles(data, randoms, n, box, origin=(0.0, 0.0, 0.0), assign=3, interlace=1, kbins=(0.0, 0.01, 10),
                     ells=(0, 2, 4), modified=(), precision="mixed", periodic=None, los_dir=None,
                     observer=(0.0, 0.0, 0.0), device=0, out=None, two_index=()):
    """Yamamoto P_l (and P_lb; ``two_index`` lists (l, l') of P_22, P_42, P_44 to report).  Returns
    a dict of NumPy arrays, or fills the device tensor ``out``."""
    keep = _Keep()
    if periodic is None:
        periodic = randoms is None
    spec = make_spec(n, box, origin, assign, interlace, periodic, los_dir, observer)
    kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
    emask = sum(1 << int(l) for l in ells)
    mmask = sum(1 << int(l) for l in modified)
    ll_bits = {(2, 2): 16, (4, 2): 17, (4, 4): 18}
    mmask += sum(1 << ll_bits[tuple(p)] for p in two_index)
    length = max(int(B.npc_power_out_len(C.byref(kb), emask, mmask)), 1)  # the library rejects bad requests
    d = make_catalog(data, keep)
    r = make_catalog(randoms, keep)
    ctx = context(device)
    if out is not None:
        B.check(B.npc_power_multipoles(ctx, C.byref(spec), C.byref(d), C.byref(r) if r else None, C.byref(kb),
                                       emask, mmask, _prec(precision), C.c_void_p(out.data_ptr()), 1), ctx)
        return out
    buf = np.zeros(length)
    B.check(B.npc_power_multipoles(ctx, C.byref(spec), C.byref(d), C.byref(r) if r else None, C.byref(kb),
                                   emask, mmask, _prec(precision), buf.ctypes.data_as(C.c_void_p), 0), ctx)
    return unpack_power(buf, kbins[2], ells, modified, two_index)


def cross_power_multipoles(data_a, randoms_a, data_b, randoms_b, n, box, origin=(0.0, 0.0, 0.0), assign=3,
                           interlace=1, kbins=(0.0, 0.01, 10), ells=(0, 2, 4), precision="mixed", periodic=None,
                           los_dir=None, observer=(0.0, 0.0, 0.0), device=0, out=None):
    """Cross multipoles P_l^AB of tracers A and B (line of sight on B, no shot noise).  Returns a
    dict of NumPy arrays (scalars: alpha_A, I22_AB, alpha_B, 0, I22_A, I22_B, sum w_A, sum w_B), or
    fills the device tensor ``out``."""
    keep = _Keep()
    if periodic is None:
        periodic = randoms_a is None
    spec = make_spec(n, box, origin, assign, interlace, periodic, los_dir, observer)
    kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
    emask = sum(1 << int(l) for l in ells)
    length = max(int(B.npc_power_out_len(C.byref(kb), emask, 0)), 1)
    da, db = make_catalog(data_a, keep), make_catalog(data_b, keep)
    ra, rb = make_catalog(randoms_a, keep), make_catalog(randoms_b, keep)
    ctx = context(device)
    args = (ctx, C.byref(spec), C.byref(da), C.byref(ra) if ra else None, C.byref(db),
            C.byref(rb) if rb else None, C.byref(kb), emask, _prec(precision))
    if out is not None:
        B.check(B.npc_cross_power_multipoles(*args, C.c_void_p(out.data_ptr()), 1), ctx)
        return out
    buf = np.zeros(length)
    B.check(B.npc_cross_power_multipoles(*args, buf.ctypes.data_as(C.c_void_p), 0), ctx)
    res = unpack_power(buf, kbins[2], ells, ())
    raw = buf[-8:]
    res["scalars"] = dict(zip(("alpha_a", "I22_ab", "alpha_b", "zero", "I22_a", "I22_b", "sum_w_a", "sum_w_b"), raw))
    return res


def unpack_power(buf, nbins, ells, modified, two_index=()):
    buf = np.asarray(buf)
    res = {"k_eff": buf[0:nbins].copy(), "nmodes": buf[nbins:2 * nbins].copy(), "P": {}, "Pmod": {}, "Pll": {}}
    row = 2
    for l in sorted(ells):
        res["P"][l] = buf[row * nbins:(row + 1) * nbins].copy()
        row += 1
    for l in sorted(modified):
        res["Pmod"][l] = buf[row * nbins:(row + 1) * nbins].copy()
        row += 1
    for p in ((2, 2), (4, 2), (4, 4)):
        if p in {tuple(q) for q in two_index}:
            res["Pll"][p] = buf[row * nbins:(row + 1) * nbins].copy()
            row += 1
    sc = buf[row * nbins:row * nbins + 8]
    res["scalars"] = dict(zip(("alpha", "I22", "I33", "N0", "S3", "sum_wg", "sum_wr", "sum_w2"), sc))
    return res


def catalog_scalars(data, randoms=None, box=0.0, device=0):
    keep = _Keep()
    d = make_catalog(data, keep)
    r = make_catalog(randoms, keep)
    out = np.zeros(8)
    ctx = context(device)
    B.check(B.npc_catalog_scalars(ctx, C.byref(d), C.byref(r) if r else None, float(box),
                                  out.ctypes.data_as(C.c_void_p), 0), ctx)
    return dict(zip(("alpha", "I22", "I33", "N0", "S3", "sum_wg", "sum_wr", "sum_w2"), out))


def last_stats(device=0):
    st = B.npc_stats()
    B.check(B.npc_last_stats(context(device), C.byref(st)))
    return {k: getattr(st, k) for k, _ in B.npc_stats._fields_}


def set_option(name, value, device=0):
    """Implementation switch of the context (npc_set_option), e.g. ("tcgen05_triple", 0)."""
    B.check(B.npc_set_option(context(device), name.encode(), int(value)), context(device))


def get_option(name, device=0):
    """Current value of a context option (npc_get_option)."""
    v = C.c_int64()
    B.check(B.npc_get_option(context(device), name.encode(), C.byref(v)), context(device))
    return v.value


def set_wait_limit(cycles, device=0):
    """Bound of the device-side waits in clock cycles (<= 0: the default); see npc_set_wait_limit."""
    B.check(B.npc_set_wait_limit(context(device), int(cycles)))


def device_status(device=0):
    """npc_device_status: raises NpcError when a bounded device wait gave up since the last check."""
    ctx = context(device)
    B.check(B.npc_device_status(ctx), ctx)


def set_profiling(on=True, device=0):
    B.check(B.npc_set_profiling(context(device), 1 if on else 0))


def stage_times(device=0, cap=64):
    """[(name, ms, launches)] for the stages of the last call (waits for the stream)."""
    ctx = context(device)
    names = C.create_string_buffer(32 * cap)
    ms = (C.c_double * cap)()
    nl = (C.c_int32 * cap)()
    n = C.c_int32(0)
    B.check(B.npc_stage_times(ctx, names, ms, nl, cap, C.byref(n)), ctx)
    raw = names.raw
    return [(raw[32 * i:32 * i + 32].split(b"\0")[0].decode(), ms[i], nl[i]) for i in range(n.value)]


def bispectrum(data, n, box, kbins, scoc_ells=(0, 2), tripo_ells=(0, 2), shot=True, assign=3, interlace=1,
               los_dir=(0.0, 0.0, 1.0), precision="mixed", origin=(0.0, 0.0, 0.0), device=0, out=None,
               randoms=None, observer=(0.0, 0.0, 0.0)):
    """Scoccimarro B_l and compressed B_l0l: periodic box with a global line of sight, or (with
    ``randoms``) survey geometry, where ``los_dir=None`` puts the line of sight from ``observer``
    to each grid point (Yamamoto X_2).  shot: False/0 raw, True/1 analytic shot noise, "fft"/2 the
    FFT-method shot noise."""
    keep = _Keep()
    shot = 2 if shot == "fft" else int(shot)
    spec = make_spec(n, box, origin, assign, interlace, 1 if randoms is None else 0, los_dir, observer)
    kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
    sm = sum(1 << int(l) for l in scoc_ells)
    tm = sum(1 << int(l) for l in tripo_ells)
    ntri, npair, length = C.c_int64(), C.c_int64(), C.c_int64()
    st = B.npc_bispectrum_layout(C.byref(kb), sm, tm, C.byref(ntri), C.byref(npair), C.byref(length))
    d = make_catalog(data, keep)
    r = make_catalog(randoms, keep)
    rp = C.byref(r) if r is not None else None
    ctx = context(device)
    if out is not None:
        B.check(B.npc_bispectrum(ctx, C.byref(spec), C.byref(d), rp, C.byref(kb), sm, tm, int(shot),
                                 _prec(precision), C.c_void_p(out.data_ptr()), 1), ctx)
        return out
    buf = np.zeros(max(length.value, 1) if st == 0 else 1)
    B.check(B.npc_bispectrum(ctx, C.byref(spec), C.byref(d), rp, C.byref(kb), sm, tm, int(shot),
                             _prec(precision), buf.ctypes.data_as(C.c_void_p), 0), ctx)
    return unpack_bispectrum(buf, kbins, scoc_ells, tripo_ells)


def cross_bispectrum(tracers, n, box, kbins, scoc_ells=(0, 2), tripo_ells=(0,), assign=3, interlace=1,
                     los_dir=(0.0, 0.0, 1.0), precision="mixed", origin=(0.0, 0.0, 0.0), device=0, out=None):
    """Multi-tracer bispectra (npc_cross_bispectrum): ``tracers`` = three (data, randoms) pairs
    (randoms None for a periodic box), tracer 1 on leg 1 (the line-of-sight leg of B_l), tracers 2
    and 3 on legs 2 and 3; global line of sight; raw estimates."""
    keep = _Keep()
    periodic = tracers[0][1] is None
    spec = make_spec(n, box, origin, assign, interlace, 1 if periodic else 0, los_dir, (0.0, 0.0, 0.0))
    kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
    sm = sum(1 << int(l) for l in scoc_ells)
    tm = sum(1 << int(l) for l in tripo_ells)
    ntri, npair, length = C.c_int64(), C.c_int64(), C.c_int64()
    st = B.npc_bispectrum_layout(C.byref(kb), sm, tm, C.byref(ntri), C.byref(npair), C.byref(length))
    darr = (B.npc_catalog * 3)(*[make_catalog(t[0], keep) for t in tracers])
    rarr = None if periodic else (B.npc_catalog * 3)(*[make_catalog(t[1], keep) for t in tracers])
    ctx = context(device)
    if out is not None:
        B.check(B.npc_cross_bispectrum(ctx, C.byref(spec), darr, rarr, C.byref(kb), sm, tm, _prec(precision),
                                       C.c_void_p(out.data_ptr()), 1), ctx)
        return out
    buf = np.zeros(max(length.value, 1) if st == 0 else 1)
    B.check(B.npc_cross_bispectrum(ctx, C.byref(spec), darr, rarr, C.byref(kb), sm, tm, _prec(precision),
                                   buf.ctypes.data_as(C.c_void_p), 0), ctx)
    return unpack_bispectrum(buf, kbins, scoc_ells, tripo_ells)


def bispectrum_sugiyama(data, n, box, kbins, multipoles=((0, 0, 0), (2, 0, 2)), shot=False, assign=3, interlace=1,
                        los_dir=(0.0, 0.0, 1.0), precision="mixed", origin=(0.0, 0.0, 0.0), device=0, out=None,
                        randoms=None):
    """Sugiyama TripoSH multipoles B_{l1 l2 L}(k1, k2) for every bin pair, global line of sight
    ``los_dir``; periodic box, or survey geometry with ``randoms``.  shot: True/1 subtracts the
    analytic shot noise, "fft"/2 the FFT-method (exact) one.  Returns {"B": {(l1, l2, L): (nb, nb) array, row k1, column k2}, "shot": {...},
    "nmodes", "scalars"}."""
    keep = _Keep()
    shot = 2 if shot == "fft" else int(shot)
    spec = make_spec(n, box, origin, assign, interlace, 1 if randoms is None else 0, los_dir, (0.0, 0.0, 0.0))
    kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
    mps = [tuple(int(v) for v in mp) for mp in multipoles]
    arr = (C.c_int32 * (3 * len(mps)))(*[v for mp in mps for v in mp])
    length = B.npc_bispectrum_sugiyama_len(C.byref(kb), len(mps))
    d = make_catalog(data, keep)
    r = make_catalog(randoms, keep)
    rp = C.byref(r) if r is not None else None
    ctx = context(device)
    if out is not None:
        B.check(B.npc_bispectrum_sugiyama(ctx, C.byref(spec), C.byref(d), rp, C.byref(kb), len(mps), arr,
                                          int(shot), _prec(precision), C.c_void_p(out.data_ptr()), 1), ctx)
        return out
    buf = np.zeros(max(int(length), 1))
    B.check(B.npc_bispectrum_sugiyama(ctx, C.byref(spec), C.byref(d), rp, C.byref(kb), len(mps), arr,
                                      int(shot), _prec(precision), buf.ctypes.data_as(C.c_void_p), 0), ctx)
    return unpack_sugiyama(buf, kbins, mps)


def unpack_sugiyama(buf, kbins, multipoles):
    nb = int(kbins[2])
    buf = np.asarray(buf)
    res = {"B": {}, "shot": {}}
    o = 0
    for key in ("B", "shot"):
        for mp in multipoles:
            res[key][tuple(mp)] = buf[o:o + nb * nb].reshape(nb, nb).copy()
            o += nb * nb
    res["nmodes"] = buf[o:o + nb].copy()
    o += nb
    res["scalars"] = dict(zip(("alpha", "I22", "I33", "N0", "S3", "sum_wg", "sum_wr", "sum_w2"), buf[o:o + 8]))
    return res


def bispectrum_triangles(kbins):
    kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
    n = C.c_int64()
    B.check(B.npc_bispectrum_triangles(C.byref(kb), None, 0, C.byref(n)))
    tri = np.zeros((n.value, 3), dtype=np.int32)
    B.check(B.npc_bispectrum_triangles(C.byref(kb), tri.ctypes.data_as(C.POINTER(C.c_int32)), n.value, C.byref(n)))
    return tri


def unpack_bispectrum(buf, kbins, scoc_ells, tripo_ells):
    kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
    ntri, npair = C.c_int64(), C.c_int64()
    sm = sum(1 << int(l) for l in scoc_ells)
    tm = sum(1 << int(l) for l in tripo_ells)
    B.check(B.npc_bispectrum_layout(C.byref(kb), sm, tm, C.byref(ntri), C.byref(npair), None))
    nt, npr, nb = ntri.value, npair.value, int(kbins[2])
    buf = np.asarray(buf)
    o = 0
    res = {"B": {}, "shot_B": {}, "BB": {}, "shot_BB": {}}
    for l in sorted(scoc_ells):
        res["B"][l] = buf[o:o + nt].copy()
        o += nt
    for l in sorted(scoc_ells):
        res["shot_B"][l] = buf[o:o + nt].copy()
        o += nt
    res["NT"] = buf[o:o + nt].copy()
    o += nt
    for l in sorted(tripo_ells):
        res["BB"][l] = buf[o:o + npr].copy()
        o += npr
    for l in sorted(tripo_ells):
        res["shot_BB"][l] = buf[o:o + npr].copy()
        o += npr
    res["nmodes"] = buf[o:o + nb].copy()
    o += nb
    res["scalars"] = dict(zip(("alpha", "I22", "I33", "N0", "S3", "sum_wg", "sum_wr", "sum_w2"), buf[o:o + 8]))
    res["tri"] = bispectrum_triangles(kbins)
    return res


def make_batch(items):
    """ctypes array of npc_batch_item from dicts with keys n, box, data, and optionally origin,
    assign, interlace, randoms, los_dir, observer, power_bins (kmin, dk, nbins), bispec_bins."""
    keep = _Keep()
    arr = (B.npc_batch_item * len(items))()
    for i, it in enumerate(items):
        rnd = it.get("randoms")
        a = arr[i]
        a.mesh = make_spec(it["n"], it["box"], it.get("origin", (0.0, 0.0, 0.0)), it.get("assign", 3),
                           it.get("interlace", 1), 0 if rnd is not None else 1, it.get("los_dir"),
                           it.get("observer", (0.0, 0.0, 0.0)))
        a.data = make_catalog(it["data"], keep)
        if rnd is not None:
            a.randoms = make_catalog(rnd, keep)
        a.power_bins = B.npc_kbins(*[float(v) for v in it["power_bins"][:2]], int(it["power_bins"][2]))
        bb = it.get("bispec_bins")
        a.bispec_bins = B.npc_kbins(*[float(v) for v in bb[:2]], int(bb[2])) if bb else B.npc_kbins(0.0, 1.0, 0)
    return arr, keep


def batch_layout(arr, ells=(0, 2, 4)):
    emask = sum(1 << int(l) for l in ells)
    offs = (C.c_int64 * (2 * len(arr)))()
    total = B.npc_batch_layout(len(arr), arr, emask, offs)
    return int(total), [(offs[2 * i], offs[2 * i + 1]) for i in range(len(arr))]


def batch_run(arr, out, ells=(0, 2, 4), precision="mixed", graph=True, device=0):
    """Runs the batch into the device tensor ``out`` (float64, batch_layout() long)."""
    emask = sum(1 << int(l) for l in ells)
    ctx = context(device)
    B.check(B.npc_batch_run(ctx, len(arr), arr, emask, _prec(precision), C.c_void_p(out.data_ptr()),
                            B.NPC_BATCH_GRAPH if graph else 0), ctx)
    return out


def batch_tune(arr, out, ells=(0, 2, 4), precision="mixed", device=0):
    emask = sum(1 << int(l) for l in ells)
    ctx = context(device)
    nb = C.c_int32(0)
    B.check(B.npc_batch_tune(ctx, len(arr), arr, emask, _prec(precision), C.c_void_p(out.data_ptr()),
                             C.byref(nb)), ctx)
    return nb.value


def batch_set_branches(n, device=0):
    B.check(B.npc_batch_set_branches(context(device), int(n)))


def tune_transforms(n, precision="mixed", device=0):
    """Autotune the transform passes for mesh size n on this context (kept for later calls)."""
    ctx = context(device)
    B.check(B.npc_tune_transforms(ctx, int(n), _prec(precision)), ctx)
