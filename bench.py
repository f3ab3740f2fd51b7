"""Benchmark: Yamamoto P_0,2,4 + modified P_4b,6b,8b at 512^3 (catalogue -> multipoles per step).

Workload: 2e6 lognormal galaxies + 2e7 uniform randoms, box 2000 Mpc/h at 2500 Mpc/h from the
observer, 512^3 TSC + interlacing, FKP weights, 80 bins of 0.01 h/Mpc, float32 transforms with
float64 bin and normalisation accumulators.  One step = one full measurement through the C ABI
(catalogue scalars, painting of both interlacing phases, 15 real-field transforms per phase,
contraction, normalisation).  Metric: P_l meshes/s (measurements per second, whole job).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one independent measurement per rank per step (replicas; the estimator has no
exchange step), launched with torch.distributed.run; value = all ranks' measurements / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "p024b_mixed_512"
METRIC = "P_l meshes/s @512^3 (P_0,2,4 + P_4b,6b,8b, catalogue to multipoles)"
UNIT = "meshes/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _src_hash(files=None):
    """Hash of the CUDA sources (all of csrc/, or the listed repo-relative files)."""
    h = hashlib.sha256()
    if files is None:
        csrc = os.path.join("paper_2605_04864_gb300", "csrc")
        files = [os.path.join(csrc, fn) for fn in sorted(os.listdir(os.path.join(ROOT, csrc)))]
    for rel in files:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(os.path.basename(rel).encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload=WORKLOAD):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current source of
    the kernel (its translation unit and the headers it includes, as listed in the record)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        rec = d.get(workload, {}).get(kernel)
        if rec and rec.get("src_hash") == _src_hash(rec.get("src_files")):
            return float(rec["bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_collectives(world, device):
    """Barrier and max-over-ranks for replicas (one measurement per rank, no data-path exchange):
    the timed region of every leg is bracketed by barriers and the slowest rank's time is reported."""
    import torch

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def replica_throughput(world, units_per_rank, max_seconds):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / max_seconds


def make_inputs(w, rank=0):
    from synthetic import make_survey_catalogs

    g, r, origin = make_survey_catalogs(w["n_gal"], w["n_ran"], w["box"], w["distance"], w["n_gen"],
                                        seed=w["seed"] + rank, fkp_p0=w["fkp_p0"])
    return g, r, origin


def active_row_fraction(w):
    """Fraction of the half-spectrum rows (ky, kz) that hold a binned mode (ky^2 + kz^2 below the
    largest bin edge in grid units); the others are neither stored by the y pass nor read by the
    contraction."""
    import math

    n = w["n"]
    r2 = ((w["kmin"] + w["nbins"] * w["dk"]) * w["box"] / (2 * math.pi)) ** 2
    lim = math.floor(r2) + 1
    act = 0
    for kz in range(n // 2):
        for jy in range(-n // 2, n // 2):
            act += jy * jy + kz * kz <= lim
    return act / ((n // 2) * n)


def algorithmic_bytes(w, stage, nf):
    """Bytes each stage must move at least once (float32 meshes / complex64 half spectra)."""
    n = w["n"]
    mesh = 4 * n**3            # one real float32 mesh
    half = 8 * (n // 2) * n * n  # one complex64 half spectrum = 4 n^3
    nph = 2 if w["interlace"] else 1
    ntot = w["n_gal"] + w["n_ran"]
    act = active_row_fraction(w)
    if stage == "fft_z_weighted":
        return nph * mesh + nf * half
    if stage == "fft_y":
        return nf * half * (1 + act)
    if stage == "fft_x_contract":
        return nf * half * act
    tiles = nph * mesh * ((16 + 4) / 16) ** 3   # (bs+4)^3 tiles per bs^3 brick, per phase
    if stage == "paint_count":      # positions in, brick id + rank out
        return ntot * (12 + 8)
    if stage == "paint_scatter":    # positions + weight + brick id + rank in, 16 B records out
        return ntot * (16 + 8 + 16)
    if stage == "paint_tiles":      # records in, tiles out
        return ntot * 16 + tiles
    if stage == "paint_fold":       # tiles in, meshes out
        return tiles + nph * mesh
    return 0


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _power_spec(w, origin):
    return dict(n=w["n"], box=w["box"], origin=tuple(float(v) for v in origin), assign=w["assign"],
                interlace=w["interlace"], los="endpoint", observer=(0.0, 0.0, 0.0))


def cpu_baseline(w, g, r, origin):
    """The FP64 oracle's half-spectrum pipeline (oracle.power.HalfSpectrumPower: painting of each
    interlacing phase, one stage per phase and (l, m >= 0) with its Y_lm-weighted real-to-complex
    transforms, then interlacing, compensation and binning) on the bench's own catalogues at the full
    512^3 configuration, scipy.fft with every available core.  A bounded sample of its stages is
    timed: the painting of phase 0, one one-transform stage (l = 0, m = 0), one two-transform stage
    (l = 2, m = 1) and the binning stage (run on accumulators of the full set's shapes: its cost does
    not depend on the values).  The measurement's time is the sum over all stages of the timed
    stage of the same kind (each phase paints the whole catalogue; m = 0 stages make one transform,
    m > 0 stages two)."""
    from oracle import power as P

    cores = _cores()
    spec = _power_spec(w, origin)
    kb = (w["kmin"], w["dk"], w["nbins"])
    run = P.HalfSpectrumPower(spec, g, r, kb, w["ells"], w["modified"], workers=cores)
    stages = dict(run.stages())
    timed = {}

    def tick(name, f):
        t0 = time.perf_counter()
        f()
        timed[name] = time.perf_counter() - t0

    tick("paint", stages["paint phase 0"])
    tick("transform_m0", stages["transform phase 0 l=0 m=0"])
    tick("transform_m1", stages["transform phase 0 l=2 m=1"])
    have = run.acc[0][2]
    for ph in range(run.nph):
        for ell in run.need:
            run.acc[ph].setdefault(ell, have)
    tick("bin", stages["combine and bin"])
    n_m0 = run.nph * len(run.need)
    n_m1 = run.nph * sum(ell for ell in run.need)
    total = run.nph * timed["paint"] + n_m0 * timed["transform_m0"] + n_m1 * timed["transform_m1"] + timed["bin"]
    desc = (f"oracle.power.HalfSpectrumPower (numpy/scipy float64) on the full workload ({w['n']}^3, "
            f"{len(g.w)} galaxies + {len(r.w)} randoms); timed stages: painting of phase 0, one "
            f"one-transform and one two-transform (l, m) stage of phase 0 and the binning stage "
            f"({sum(timed.values()):.1f} s); measurement time = {run.nph} x painting + {n_m0} x "
            f"one-transform + {n_m1} x two-transform stages + binning = {total:.1f} s; scipy.fft "
            f"workers = {cores} (the elementwise numpy work runs on one core)")
    return {"value": 1.0 / total, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
            "sample_seconds": sum(timed.values()), "stage_seconds": {k: round(v, 3) for k, v in timed.items()},
            "measurement_seconds": total}


REFERENCE_MESH = 128


def run_reference(args, w):
    """The reference arm: the FP64 oracle (there is no reference implementation to install) timed on
    the host cores, one full catalogue -> multipoles measurement per step, on a sample of the bench
    workload small enough that the steps fit in a few minutes: the same survey geometry, FKP weights,
    TSC interlacing and bins of 0.01 h/Mpc, on a 128^3 mesh with the objects scaled by (128/512)^3
    (the same objects per cell).  The line names that sample in its config; its rate is the measured
    rate of the sample, not scaled to 512^3."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import math

    from oracle import power as P
    from synthetic import make_survey_catalogs

    cores = _cores()
    ns = REFERENCE_MESH
    f = (ns / w["n"]) ** 3
    g, r, origin = make_survey_catalogs(int(w["n_gal"] * f), int(w["n_ran"] * f), w["box"], w["distance"],
                                        min(w["n_gen"], ns), seed=w["seed"], fkp_p0=w["fkp_p0"])
    spec = _power_spec(dict(w, n=ns), origin)
    nb = min(w["nbins"], int(math.pi * ns / w["box"] / w["dk"]))
    kb = (w["kmin"], w["dk"], nb)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        P.power_multipoles_rfft(spec, g, r, kb, w["ells"], w["modified"], workers=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = len(times) / tot
    desc = (f"oracle.power.power_multipoles_rfft (numpy/scipy float64), one full measurement per step of the "
            f"{w['n']}^3 workload sampled at {ns}^3 with {len(g.w)} galaxies + {len(r.w)} randoms (same box, "
            f"geometry, weights and objects per cell; {nb} bins up to the sample's Nyquist); scipy.fft workers "
            f"= {cores}; the rate is the sample's own, not scaled")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} sampled at {ns}^3", "mesh": ns, "n_gal": len(g.w),
                       "n_ran": len(r.w), "nbins": nb, "global_batch": 1, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def power_errors(w, g, r, ours, nb):
    """Per-multipole error of the library's output against the FP64 oracle values stored for the
    same inputs (tests/golden/full_size_p024b_mixed_512.json, written by the oracle), in the
    monopole-scale metric |X - X_orc| / max(|X_orc|, |P_0,orc| + N_0); None when the stored values
    were computed from other input bytes."""
    import numpy as np

    from synthetic import fingerprint

    path = os.path.join(ROOT, "tests", "golden", "full_size_p024b_mixed_512.json")
    if not os.path.exists(path):
        return {"available": False, "reason": "no stored oracle values"}
    with open(path) as f:
        orc = json.load(f)
    if orc.get("fingerprint") != fingerprint(g, r):
        return {"available": False, "reason": "stored oracle values were computed from other input bytes"}
    from paper_2605_04864_gb300 import api

    res = api.unpack_power(ours, nb, w["ells"], w["modified"])
    scale = np.abs(np.asarray(orc["P"]["0"])) + orc["scalars"]["N0"]
    err = {}
    for l in w["ells"]:
        o = np.asarray(orc["P"][str(l)])
        err[f"P{l}"] = float(np.max(np.abs(res["P"][l] - o) / np.maximum(np.abs(o), scale)))
    for l in w["modified"]:
        o = np.asarray(orc["Pmod"][str(l)])
        err[f"P{l}b"] = float(np.max(np.abs(res["Pmod"][l] - o) / np.maximum(np.abs(o), scale)))
    return {"available": True, "metric": "max over bins of |X - X_orc| / max(|X_orc|, |P_0,orc| + N_0)",
            "tolerance": 1e-5, "oracle": orc.get("oracle"), "max": err}


def _tf32_peak():
    """Dense tf32 tensor peak: the measured bf16 burst figure times the nominal tf32 / bf16 ratio
    (1.1 / 2.25 PFLOP/s dense)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x nominal tf32/bf16"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x nominal tf32/bf16"


def _f16_peak():
    """Dense f16 tensor peak: the measured bf16 burst figure (f16 and bf16 share the dense rate)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured bf16 (f16 has the same dense rate)"
    except Exception:
        return 1900.0, "fallback bf16 (f16 has the same dense rate)"


def bispec_errors(cat, res):
    """Error of every B_0, B_2 triangle and B_000, B_202 pair (raw estimate and analytic shot noise)
    against the FP64 oracle values stored for the same catalogue (tests/golden/full_size_bispec_256.json,
    written by the oracle), relative to the monopole scale |B_0,orc| + |N_0,orc| of the same
    triangle or pair; None when the stored values were computed from other input bytes."""
    import numpy as np

    from synthetic import fingerprint

    path = os.path.join(ROOT, "tests", "golden", "full_size_bispec_256.json")
    if not os.path.exists(path):
        return {"available": False, "reason": "no stored oracle values"}
    with open(path) as f:
        orc = json.load(f)
    if orc.get("fingerprint") != fingerprint(cat):
        return {"available": False, "reason": "stored oracle values were computed from other input bytes"}
    a = lambda v: np.asarray(v)
    out = {}
    st = a(orc["B_raw"]["0"]).__abs__() + a(orc["shot_B"]["0"]).__abs__()
    sp = a(orc["BB_raw"]["0"]).__abs__() + a(orc["shot_BB"]["0"]).__abs__()
    for l in (0, 2):
        o = a(orc["B_raw"][str(l)])
        out[f"B{l}"] = float(np.max(np.abs(res["B"][l] + res["shot_B"][l] - o) / np.maximum(np.abs(o), st)))
        o = a(orc["shot_B"][str(l)])
        out[f"shot_B{l}"] = float(np.max(np.abs(res["shot_B"][l] - o) / np.maximum(np.abs(o), st)))
        o = a(orc["BB_raw"][str(l)])
        out[f"B{l}0{l}"] = float(np.max(np.abs(res["BB"][l] + res["shot_BB"][l] - o) / np.maximum(np.abs(o), sp)))
        o = a(orc["shot_BB"][str(l)])
        out[f"shot_B{l}0{l}"] = float(np.max(np.abs(res["shot_BB"][l] - o) / np.maximum(np.abs(o), sp)))
    return {"available": True, "metric": "max over triangles (pairs) of |X - X_orc| / max(|X_orc|, |B_0,orc| + |N_0,orc|)",
            "tolerance": 1e-4, "max": out}


BISPEC_SAMPLE_BINS = 4


def bispec_cpu_baseline(w, cat):
    """The FP64 oracle (oracle.bispec.bispectrum with its analytic shot noise) on the bench's own
    256^3 catalogue, restricted to the first BISPEC_SAMPLE_BINS k-bins (a bounded sample: the full
    19-bin set takes the oracle several minutes); rate in the leg's unit over the sample's triangles."""
    from oracle import bispec as OB

    kb = (w["kmin"], w["dk"], BISPEC_SAMPLE_BINS)
    spec = dict(n=w["n"], box=w["box"], origin=(0.0, 0.0, 0.0), assign=w["assign"], interlace=w["interlace"],
                los="global", los_dir=(0.0, 0.0, 1.0), periodic=1)
    t0 = time.perf_counter()
    res = OB.bispectrum(spec, cat, None, kb, w["scoc_ells"], w["tripo_ells"], shot=True)
    dt = time.perf_counter() - t0
    ntri = len(res["tri"])
    return {"value": ntri * len(w["scoc_ells"]) / dt, "unit": "triangles/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle.bispec.bispectrum (numpy float64, analytic shot noise, B_0, B_2, B_000, B_202) on the "
                      f"full {w['n']}^3 catalogue with the first {BISPEC_SAMPLE_BINS} of {w['nbins']} bins "
                      f"({ntri} triangles, {dt:.1f} s); numpy's transforms run on one core",
            "sample_seconds": dt}


def bispec_leg(args, world, rank, barrier, max_over_ranks):
    """B_l triangles/s at 256^3: 1e6 lognormal particles, periodic, TSC interlaced, 19 bins,
    805 closed triangles, B_0 and B_2 (plus the compressed B_000, B_202) with analytic shot noise."""
    import ctypes as C
    from types import SimpleNamespace

    import numpy as np
    import torch

    from paper_2605_04864_gb300 import api
    from paper_2605_04864_gb300 import binding as B
    from synthetic import make_periodic_catalog, workload

    w = workload("bispec_256")
    cat = make_periodic_catalog(w["n_gal"], w["box"], w["n_gen"], seed=w["seed"] + rank)
    cd = SimpleNamespace(pos=torch.from_numpy(cat.pos).cuda(), w=torch.from_numpy(cat.w).cuda(),
                         nbar=torch.from_numpy(cat.nbar).cuda())
    kb = (w["kmin"], w["dk"], w["nbins"])
    kbs = B.npc_kbins(*kb)
    ntri, npair, length = C.c_int64(), C.c_int64(), C.c_int64()
    B.check(B.npc_bispectrum_layout(C.byref(kbs), 5, 5, C.byref(ntri), C.byref(npair), C.byref(length)))
    out = torch.zeros(length.value, dtype=torch.float64, device="cuda")
    kw = dict(n=w["n"], box=w["box"], kbins=kb, scoc_ells=w["scoc_ells"], tripo_ells=w["tripo_ells"], shot=True,
              precision=w["precision"], out=out)
    for _ in range(args.warmup):
        api.bispectrum(cd, **kw)
    torch.cuda.synchronize()
    launches = api.last_stats()["n_kernel_launches"]
    barrier()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        api.bispectrum(cd, **kw)
    e.record()
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(s.elapsed_time(e)) / args.steps
    nmult = len(w["scoc_ells"])
    api.set_profiling(True)
    acc = {}
    for _ in range(args.steps):
        api.bispectrum(cd, **kw)
        for name, t, nl in api.stage_times():
            a = acc.setdefault(name, [0.0, 0, 0])
            a[0] += t
            a[1] += nl
            a[2] += 1
    api.set_profiling(False)
    stages = {k: round(v[0] / v[2], 4) for k, v in acc.items()}
    # the same measurement with the FFT-method (exact triplet) shot noise of B_l
    kwf = dict(kw, shot="fft")
    for _ in range(args.warmup):
        api.bispectrum(cd, **kwf)
    torch.cuda.synchronize()
    barrier()
    s.record()
    for _ in range(args.steps):
        api.bispectrum(cd, **kwf)
    e.record()
    torch.cuda.synchronize()
    barrier()
    ms_fft = max_over_ranks(s.elapsed_time(e)) / args.steps
    # end to end: pinned host catalogue in, host arrays out (the public Python call), every step
    pin = lambda a: torch.from_numpy(a).pin_memory()
    ch = SimpleNamespace(pos=pin(cat.pos), w=pin(cat.w), nbar=pin(cat.nbar))
    kwh = {k: v for k, v in kw.items() if k != "out"}
    api.bispectrum(ch, **kwh)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host_res = api.bispectrum(ch, **kwh)
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * ntri.value * nmult * args.steps / e2e_s, "unit": "triangles/s",
           "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in (ch.pos, ch.w, ch.nbar)),
           "d2h_bytes_per_step": length.value * 8, "ms_per_step": e2e_s / args.steps * 1e3}
    # the dense triple-product contraction: tensor-bound (float32 shell fields split into f16 hi + lo
    # on the tcgen05 path, tf32 hi + lo on mma.sync)
    st = api.last_stats()
    tri_ms, tri_nl, tri_rep = acc.get("triple", [0.0, 0, 1])
    tri_launch_ms = tri_ms / max(tri_nl, 1)
    tri_flops = st["contraction_flops"] / max(st["contraction_launches"], 1)
    tri_issued = st["contraction_issued_flops"] / max(st["contraction_launches"], 1)
    tc_path = bool(api.get_option("tcgen05_triple"))
    tpeak, tpeak_src = _f16_peak() if tc_path else _tf32_peak()
    achieved = tri_flops / (tri_launch_ms / 1e3) / 1e12
    roofline = {"bound": "tensor", "kernel": "triple", "achieved": achieved, "peak": tpeak, "unit": "TFLOP/s",
                "frac": achieved / tpeak, "traffic": _traffic("triple", "bispec_256"), "peak_source": tpeak_src,
                "flops_per_launch": tri_flops, "launch_ms": tri_launch_ms,
                "issued_flops_per_launch": tri_issued,
                "issued_frac": tri_issued / (tri_launch_ms / 1e3) / 1e12 / tpeak,
                "note": "useful multiply-adds 2 x rows x columns x cells of the 128^3 shell grid (frac); "
                        "issued_frac counts what the tensor cores execute: padded 128-row tiles and N "
                        "columns, two f16 products per k step for the hi + lo split (tcgen05) or three "
                        "tf32 products on 16 x 8 tiles (mma.sync)"}
    errs = bispec_errors(cat, host_res) if rank == 0 else None
    # Sugiyama TripoSH multipoles on the same catalogue (every (k1, k2) bin pair, raw estimator)
    mps = [(0, 0, 0), (1, 1, 0), (1, 1, 2), (2, 0, 2), (2, 2, 0), (2, 2, 2)]
    nbn = w["nbins"]
    sout = torch.zeros(2 * len(mps) * nbn * nbn + nbn + 8, dtype=torch.float64, device="cuda")
    kws = dict(n=w["n"], box=w["box"], kbins=kb, multipoles=mps, shot=True, precision=w["precision"], out=sout)
    for _ in range(args.warmup):
        api.bispectrum_sugiyama(cd, **kws)
    torch.cuda.synchronize()
    barrier()
    s.record()
    for _ in range(args.steps):
        api.bispectrum_sugiyama(cd, **kws)
    e.record()
    torch.cuda.synchronize()
    barrier()
    ms_sug = max_over_ranks(s.elapsed_time(e)) / args.steps
    api.set_profiling(True)
    sacc = {}
    for _ in range(max(1, args.steps // 4)):
        api.bispectrum_sugiyama(cd, **kws)
        for name, t, _ in api.stage_times():
            a = sacc.setdefault(name, [0.0, 0])
            a[0] += t
            a[1] += 1
    api.set_profiling(False)
    sugiyama = {"multipoles": mps, "bin_pairs": nbn * nbn, "ms_per_step": ms_sug,
                "value": world * len(mps) * nbn * nbn / (ms_sug / 1e3), "unit": "multipole values/s",
                "stages_ms": {k: round(v[0] / v[1], 4) for k, v in sacc.items()},
                "note": "TripoSH B_l1l2L with analytic shot noise for all 361 (k1, k2) pairs, global line of sight"}
    plain = None
    if not args.no_plain and rank == 0:
        # the plain float64 form (full inverse transforms, direct float64 triangle sums), compared
        # value by value with the library's raw B_0, B_2
        kwn = {k: v for k, v in kw.items() if k != "out"}
        ours = api.bispectrum(cd, **kwn)
        tri = ours["tri"]
        plain_gpu_bispec(cd, w, tri)                     # warm-up (plans, caches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            b0, b2 = plain_gpu_bispec(cd, w, tri)
        torch.cuda.synchronize()
        pms = (time.perf_counter() - t0) / reps * 1e3
        raw0 = ours["B"][0] + ours["shot_B"][0]
        raw2 = ours["B"][2] + ours["shot_B"][2]
        scale = np.abs(raw0)
        diff = max(float(np.max(np.abs(b0.cpu().numpy() - raw0) / scale)),
                   float(np.max(np.abs(b2.cpu().numpy() - raw2) / scale)))
        plain = {"value": ntri.value * nmult / (pms / 1e3), "unit": "triangles/s", "ms_per_step": pms,
                 "method": "float64 torch.fft (cuFFT) shell fields by full inverse transforms, float64 atomic "
                           "painting, direct float64 triangle sums (matrix-vector products, no tensor cores)",
                 "max_rel_diff_vs_ours": diff, "speedup_of_ours": pms / ms}
    return {"metric": "B_l triangles/s @256^3 (805 closed triangles x B_0, B_2; + B_000, B_202, shot noise)",
            "value": world * ntri.value * nmult / (ms / 1e3), "unit": "triangles/s", "ms_per_step": ms,
            "measurements_per_s": world / (ms / 1e3), "triangles": ntri.value, "pairs": npair.value,
            "config": {"workload": "bispec_256", "mesh": w["n"], "n_gal": w["n_gal"], "nbins": w["nbins"],
                       "assign": "TSC", "interlace": True},
            "stages_ms": stages, "gpu_launches": launches * args.steps,
            "roofline": roofline, "e2e": e2e, "err_vs_fp64": errs,
            "cpu_baseline": bispec_cpu_baseline(w, cat) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None,
            "plain_gpu": plain,
            "sugiyama": sugiyama,
            "fft_method_shot": {"value": world * ntri.value * nmult / (ms_fft / 1e3), "ms_per_step": ms_fft,
                                "note": "shot noise of B_l and B_l0l by the FFT method (exact sums of the two-object terms)"},
            "triple_product": ("f16 hi+lo split after exact power-of-two scales: tcgen05.mma kind::f16 M=128 with the "
                               "product rows written to tensor memory and the hi/lo columns packed along N, fields "
                               "staged by bulk asynchronous copies, for launches of more than 32 rows (3xTF32 "
                               "mma.sync m16n8k8 for the rest); FP32 within 4096-cell flushes (tcgen05, compensated "
                               "sums) or 128-cell chunks (mma.sync), FP64 across them"
                               if api.get_option("tcgen05_triple") else
                               "3xTF32 split hi+lo tensor-core products (mma.sync m16n8k8), FP32 within 128-cell "
                               "chunks, FP64 across chunks")}


def adjoint_leg(args, world, rank, barrier, max_over_ranks):
    """Gradients/s at 1024^3: 1e7 lognormal galaxies, periodic, TSC; one step = paint -> P_0,2,4
    (global LOS) and equilateral B_0 on 19 bins -> scalar loss -> backward through the mesh adjoint
    and the TSC adjoint to the positions (torch.autograd over the library's calls)."""
    import torch

    from paper_2605_04864_gb300 import autograd as AG
    from synthetic import make_periodic_catalog, workload

    w = workload("adjoint_1024")
    n, box = w["n"], w["box"]
    kb = (w["kmin"], w["dk"], w["nbins"])
    cat = make_periodic_catalog(w["n_gal"], box, w["n_gen"], seed=w["seed"] + rank)
    pos0 = torch.from_numpy(cat.pos).cuda()
    i22, n0, i33 = AG.periodic_normalisations(pos0, None, box)
    g = torch.Generator(device="cuda").manual_seed(7)
    cp = torch.randn(len(w["ells"]), kb[2], device="cuda", dtype=torch.float64, generator=g)
    cb = torch.randn(kb[2], device="cuda", dtype=torch.float64, generator=g)

    def step():
        pos = pos0.detach().requires_grad_(True)
        mesh = AG.paint(pos, None, n, box, assign=w["assign"], precision=w["precision"])
        r = AG.mesh_multipoles(mesh, box, kb, w["ells"], True, i22, n0, i33, assign=w["assign"],
                               precision=w["precision"])
        loss = (r["P"] * cp).sum() + (r["B0"] * cb).sum()
        loss.backward()
        return pos.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        step()
    e.record()
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(s.elapsed_time(e)) / args.steps
    return {"metric": "gradients/s @1024^3 (dL/dpos of P_0,2,4 + equilateral B_0, 1e7 galaxies)",
            "value": world / (ms / 1e3), "unit": "gradients/s", "ms_per_step": ms,
            "config": {"workload": "adjoint_1024", "mesh": n, "n_gal": w["n_gal"], "nbins": w["nbins"],
                       "assign": "TSC", "interlace": False, "precision": w["precision"]}}


def batch_leg(args, world, rank, barrier, max_over_ranks):
    """Mocks/s for 96 survey mocks of uneven size in one batch (32 each at 128^3, 192^3, 256^3):
    P_0,2,4 and B_0 with analytic shot noise per mock, through npc_batch_run.  The graph form (one
    graph launch per batch after the first call) and the eager form are both timed; the autotuner
    picks the y-pass tile per mesh size and the number of concurrent branches first."""
    from types import SimpleNamespace

    import torch

    from paper_2605_04864_gb300 import api
    from synthetic import base_catalogues, batch_plan, workload

    w = workload("batch_96")
    plan = batch_plan(w)
    gmax = max(m["n_gal"] for m in plan)
    rmax = max(m["n_ran"] for m in plan)
    gb, rb = base_catalogues(gmax, rmax, 256, w["seed"] + rank)
    gb, rb = torch.from_numpy(gb).cuda(), torch.from_numpy(rb).cuda()
    items = []
    for m in plan:
        o = torch.tensor(m["origin"], dtype=torch.float32, device="cuda")
        cat = lambda base, k: SimpleNamespace(pos=(base[:k] * m["box"] + o).contiguous(),
                                              w=torch.full((k,), m["weight"], device="cuda"),
                                              nbar=torch.full((k,), m["nbar"], device="cuda"))
        items.append(dict(n=m["n"], box=m["box"], origin=m["origin"], assign=w["assign"], interlace=w["interlace"],
                          data=cat(gb, m["n_gal"]), randoms=cat(rb, m["n_ran"]),
                          power_bins=(0.0, w["dk"], m["pk_nbins"]),
                          bispec_bins=(w["bk_kmin"], w["dk"], m["bk_nbins"])))
    del gb, rb
    arr, keep = api.make_batch(items)
    total, _ = api.batch_layout(arr, w["ells"])
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    branches = api.batch_tune(arr, out, w["ells"], precision=w["precision"])
    tune_s = time.perf_counter() - t0

    def timed(graph):
        for _ in range(args.warmup):
            api.batch_run(arr, out, w["ells"], precision=w["precision"], graph=graph)
        torch.cuda.synchronize()
        barrier()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(args.steps):
            api.batch_run(arr, out, w["ells"], precision=w["precision"], graph=graph)
        e.record()
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(s.elapsed_time(e)) / args.steps

    ms_graph = timed(True)
    launches = api.last_stats()["n_kernel_launches"]
    ms_eager = timed(False)
    nm = len(plan)
    triple_path = "tcgen05" if api.get_option("tcgen05_triple") else "mma.sync"
    plain = None
    if not args.no_plain and rank == 0:
        # the plain form of the same batch, mock by mock: float64 cuFFT Hand+17 P_0,2,4 and a float64
        # B_0 by full inverse transforms and direct triangle sums (no tensor cores, no graph)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it, m in zip(items, plan):
            wpk = dict(n=m["n"], box=m["box"], assign=w["assign"], kmin=0.0, dk=w["dk"], nbins=m["pk_nbins"])
            plain_gpu_power(it["data"], it["randoms"], m["origin"], wpk)
            if m["bk_nbins"] > 0:
                kbb = (w["bk_kmin"], w["dk"], m["bk_nbins"])
                plain_gpu_bispec0_survey(it["data"], it["randoms"], m["origin"], m["n"], m["box"], kbb,
                                         api.bispectrum_triangles(kbb))
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t0
        plain = {"value": nm / plain_s, "unit": "mocks/s", "ms_per_batch": plain_s * 1e3,
                 "method": "float64 torch.fft (cuFFT) Hand+17 P_0,2,4 and B_0 by full inverse transforms with direct "
                           "float64 triangle sums, mock by mock (one pass, after the library's timed runs)",
                 "speedup_of_graph": plain_s * 1e3 / ms_graph}
    del keep, items, arr, out
    torch.cuda.empty_cache()
    return {"metric": "mocks/s (96 survey mocks, 32 each at 128^3/192^3/256^3, P_0,2,4 + B_0 with shot noise)",
            "value": world * nm / (ms_graph / 1e3), "unit": "mocks/s", "ms_per_batch": ms_graph,
            "eager": {"value": world * nm / (ms_eager / 1e3), "ms_per_batch": ms_eager},
            "branches": branches, "tune_seconds": tune_s, "kernels_per_batch": launches,
            "tuned_triple_path": triple_path, "plain_gpu": plain,
            "config": {"workload": "batch_96", "mocks": nm, "n_gal_total": sum(m["n_gal"] for m in plan),
                       "n_ran_total": sum(m["n_ran"] for m in plan), "precision": w["precision"]}}


def plain_gpu_power(gd, rd, origin, w, dev="cuda", dtype=None):
    """The plain GPU form of the same measurement, timed beside the library: float64 throughout,
    cuFFT through torch.fft, painting with float64 atomics (index_add_), the Hand+17 estimator with
    all 2l+1 real spherical-harmonic fields per multipole (1 + 5 + 9 = 15 real transforms per
    interlacing phase).  Returns P_l (l = 0, 2, 4) on the workload's bins."""
    import math

    import numpy as np
    import torch

    n, box, p = w["n"], w["box"], w["assign"]
    f64 = dtype or torch.float64
    H = box / n
    pg, wg = gd.pos.to(f64), gd.w.to(f64)
    pr, wr, nr = rd.pos.to(f64), rd.w.to(f64), rd.nbar.to(f64)
    alpha = wg.sum() / wr.sum()
    i22 = alpha * (nr * wr * wr).sum()
    n0 = ((wg * wg).sum() + alpha * alpha * (wr * wr).sum()) / i22
    o = torch.tensor(origin, dtype=f64, device=dev)

    def paint(shift):
        mesh = torch.zeros(n ** 3, dtype=f64, device=dev)
        for pos, wt in ((pg, wg), (pr, -alpha * wr)):
            s = (pos - o) * (n / box) + shift
            i0 = torch.floor(s + 0.5) if p == 3 else torch.floor(s)
            d = s - i0
            if p == 3:
                taps = [(-1, 0.5 * (0.5 - d) ** 2), (0, 0.75 - d * d), (1, 0.5 * (0.5 + d) ** 2)]
            else:
                taps = [(0, 1.0 - d), (1, d)]
            i0 = i0.long()
            for ox, wx in taps:
                ix = (i0[:, 0] + ox) % n
                for oy, wy in taps:
                    iy = (i0[:, 1] + oy) % n
                    for oz, wz in taps:
                        iz = (i0[:, 2] + oz) % n
                        mesh.index_add_(0, (iz * n + iy) * n + ix, wt * wx[:, 0] * wy[:, 1] * wz[:, 2])
        return mesh.view(n, n, n)     # index (z, y, x)

    def real_harmonics(l, ux, uy, uz):
        """Orthonormal real spherical harmonics of degree l at unit vectors (2l+1 tensors)."""
        out = []
        for m in range(0, l + 1):
            c = np.zeros(l + 1)
            c[l] = 1.0
            dq = np.polynomial.legendre.leg2poly(np.polynomial.legendre.legder(c, m)) if m <= l else [0.0]
            q = torch.zeros_like(uz)
            for a in reversed(dq):
                q = q * uz + float(a)
            q = q * (-1) ** m
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            cre, cim = torch.ones_like(ux), torch.zeros_like(ux)
            for _ in range(m):
                cre, cim = cre * ux - cim * uy, cre * uy + cim * ux
            if m == 0:
                out.append(norm * q)
            else:
                out.append(math.sqrt(2.0) * norm * q * cre)
                out.append(math.sqrt(2.0) * norm * q * cim)
        return out

    # grid-point directions from the observer (at the coordinate origin), per phase
    j = torch.arange(n, dtype=f64, device=dev)
    # k-space: rfftn over (z, y, x) -> last axis x is halved
    kfreq = torch.fft.fftfreq(n, d=1.0 / n).to(dev).to(f64)
    kx = torch.arange(n // 2 + 1, dtype=f64, device=dev)
    KZ, KY, KX = kfreq.view(n, 1, 1), kfreq.view(1, n, 1), kx.view(1, 1, -1)
    kk = torch.sqrt(KX * KX + KY * KY + KZ * KZ)
    kk_safe = torch.where(kk > 0, kk, torch.ones_like(kk))
    uxk, uyk, uzk = KX / kk_safe, KY / kk_safe, KZ / kk_safe
    sinc = lambda a: torch.where(a == 0, torch.ones_like(a), torch.sin(a) / torch.where(a == 0, torch.ones_like(a), a))
    W = (sinc(math.pi * KX / n) * sinc(math.pi * KY / n) * sinc(math.pi * KZ / n)) ** p
    F = {}
    for ph, shift in ((0, 0.0), (1, 0.5)):
        mesh = paint(shift)
        zc = o[2] + (j - shift) * H
        yc = o[1] + (j - shift) * H
        xc = o[0] + (j - shift) * H
        Z, Y, X = zc.view(n, 1, 1), yc.view(1, n, 1), xc.view(1, 1, n)
        r = torch.sqrt(X * X + Y * Y + Z * Z)
        ux, uy, uz = X / r, Y / r, Z / r
        for l in (0, 2, 4):
            acc = None
            for rx, rk in zip(real_harmonics(l, ux, uy, uz), real_harmonics(l, uxk, uyk, uzk)):
                t = torch.fft.rfftn(mesh * rx) * rk
                acc = t if acc is None else acc + t
            acc = acc * (4 * math.pi / (2 * l + 1))
            F[(ph, l)] = acc
        del mesh
    phase = torch.exp(1j * math.pi * (KX + KY + KZ) / n).to(F[(0, 0)].dtype)
    Fl = {l: 0.5 * (F[(0, l)] + phase * F[(1, l)]) / W for l in (0, 2, 4)}
    # bins: half spectrum, kx = 0 and kx = n/2 planes counted once, Nyquist planes excluded
    wgt = torch.full_like(kk, 2.0)
    wgt[:, :, 0] = 1.0
    nyq = (KX == n // 2) | (KY == -n // 2) | (KZ == -n // 2)
    kf = 2 * math.pi / box
    b = torch.floor((kf * kk - w["kmin"]) / w["dk"])
    ok = (~nyq) & (kk > 0) & (b >= 0) & (b < w["nbins"])
    bi = torch.where(ok, b, torch.zeros_like(b)).long().flatten()
    wv = torch.where(ok, wgt, torch.zeros_like(wgt)).flatten()
    cnt = torch.bincount(bi, weights=wv, minlength=w["nbins"])
    res = {}
    for l in (0, 2, 4):
        pw = (Fl[0] * Fl[l].conj()).real.flatten()
        s_ = torch.bincount(bi, weights=wv * pw, minlength=w["nbins"])
        res[l] = (2 * l + 1) / i22 * s_ / torch.clamp(cnt, min=1) - (n0 if l == 0 else 0.0)
    return res, float(n0)


def plain_gpu_bispec(cd, w, tri, dev="cuda"):
    """The plain GPU form of the bispectrum measurement: float64 throughout, painting with float64
    atomics, cuFFT through torch.fft, every shell field F_b, F^(2)_b and indicator I_b by a full
    inverse transform, and the closed-triangle sums by direct float64 reductions (matrix-vector
    products over the cells; no tensor cores).  Returns raw B_0, B_2 (no shot noise) for ``tri``."""
    import math

    import torch

    n, box, p = w["n"], w["box"], w["assign"]
    f64 = torch.float64
    pos, wt = cd.pos.to(f64), cd.w.to(f64)
    wsum = wt.sum()
    i33 = wsum ** 3 / box ** 6

    def paint(shift):
        mesh = torch.zeros(n ** 3, dtype=f64, device=dev)
        s = pos * (n / box) + shift
        i0 = torch.floor(s + 0.5) if p == 3 else torch.floor(s)
        d = s - i0
        if p == 3:
            taps = [(-1, 0.5 * (0.5 - d) ** 2), (0, 0.75 - d * d), (1, 0.5 * (0.5 + d) ** 2)]
        else:
            taps = [(0, 1.0 - d), (1, d)]
        i0 = i0.long()
        for ox, wx in taps:
            ix = (i0[:, 0] + ox) % n
            for oy, wy in taps:
                iy = (i0[:, 1] + oy) % n
                for oz, wz in taps:
                    iz = (i0[:, 2] + oz) % n
                    mesh.index_add_(0, (iz * n + iy) * n + ix, wt * wx[:, 0] * wy[:, 1] * wz[:, 2])
        return (mesh - wsum / n ** 3).view(n, n, n)     # index (z, y, x), periodic: minus the mean

    kfreq = torch.fft.fftfreq(n, d=1.0 / n).to(dev).to(f64)
    kx = torch.arange(n // 2 + 1, dtype=f64, device=dev)
    KZ, KY, KX = kfreq.view(n, 1, 1), kfreq.view(1, n, 1), kx.view(1, 1, -1)
    kk = torch.sqrt(KX * KX + KY * KY + KZ * KZ)
    sinc = lambda a: torch.where(a == 0, torch.ones_like(a), torch.sin(a) / torch.where(a == 0, torch.ones_like(a), a))
    W = (sinc(math.pi * KX / n) * sinc(math.pi * KY / n) * sinc(math.pi * KZ / n)) ** p
    phase = torch.exp(1j * math.pi * (KX + KY + KZ) / n)
    X0 = 0.5 * (torch.fft.rfftn(paint(0.0)) + phase * torch.fft.rfftn(paint(0.5))) / W
    mu = torch.where(kk > 0, KZ / torch.where(kk > 0, kk, torch.ones_like(kk)), torch.zeros_like(kk))
    X2 = (1.5 * mu * mu - 0.5) * X0
    nyq = (KX == n // 2) | (KY == -n // 2) | (KZ == -n // 2)
    kf = 2 * math.pi / box
    b = torch.floor((kf * kk - w["kmin"]) / w["dk"])
    nb = w["nbins"]
    F0, F2, I = [], [], []
    for ib in range(nb):
        m = ((b == ib) & (~nyq) & (kk > 0)).to(f64)
        F0.append(torch.fft.irfftn(X0 * m, s=(n, n, n)).flatten() * n ** 3)
        F2.append(torch.fft.irfftn(X2 * m, s=(n, n, n)).flatten() * n ** 3)
        I.append(torch.fft.irfftn(m.to(X0.dtype), s=(n, n, n)).flatten() * n ** 3)
    F0, F2, I = torch.stack(F0), torch.stack(F2), torch.stack(I)
    out0, out2 = torch.zeros(len(tri), dtype=f64, device=dev), torch.zeros(len(tri), dtype=f64, device=dev)
    pairs = sorted({(int(i), int(j)) for i, j, _ in tri})
    col = {pr: q for q, pr in enumerate(pairs)}
    S0 = torch.zeros(len(pairs), nb, dtype=f64, device=dev)
    S2, NT = torch.zeros_like(S0), torch.zeros_like(S0)
    for q, (i, j) in enumerate(pairs):
        S0[q] = torch.mv(F0, F0[i] * F0[j])
        S2[q] = torch.mv(F0, F2[i] * F0[j])
        NT[q] = torch.mv(I, I[i] * I[j])
    for t, (i, j, k) in enumerate(tri):
        q = col[(int(i), int(j))]
        out0[t] = S0[q, k] / (i33 * NT[q, k])
        out2[t] = 5.0 * S2[q, k] / (i33 * NT[q, k])
    return out0, out2


def plain_gpu_bispec0_survey(gd, rd, origin, n, box, kb, tri, p=3, dev="cuda"):
    """The plain GPU form of a survey-geometry B_0: float64 throughout, the FKP field data - alpha
    randoms painted with float64 atomics on both interlacing phases, cuFFT through torch.fft, every
    shell field F_b and indicator I_b by a full inverse transform, direct float64 triangle sums.
    Returns the raw B_0 for ``tri``."""
    import math

    import torch

    f64 = torch.float64
    pg, wg = gd.pos.to(f64), gd.w.to(f64)
    pr, wr, nr = rd.pos.to(f64), rd.w.to(f64), rd.nbar.to(f64)
    alpha = wg.sum() / wr.sum()
    i33 = alpha * (nr * nr * wr * wr * wr).sum()
    o = torch.tensor(origin, dtype=f64, device=dev)

    def paint(shift):
        mesh = torch.zeros(n ** 3, dtype=f64, device=dev)
        for pos, wt in ((pg, wg), (pr, -alpha * wr)):
            s = (pos - o) * (n / box) + shift
            i0 = torch.floor(s + 0.5) if p == 3 else torch.floor(s)
            d = s - i0
            taps = ([(-1, 0.5 * (0.5 - d) ** 2), (0, 0.75 - d * d), (1, 0.5 * (0.5 + d) ** 2)] if p == 3
                    else [(0, 1.0 - d), (1, d)])
            i0 = i0.long()
            for ox, wx in taps:
                ix = (i0[:, 0] + ox) % n
                for oy, wy in taps:
                    iy = (i0[:, 1] + oy) % n
                    for oz, wz in taps:
                        iz = (i0[:, 2] + oz) % n
                        mesh.index_add_(0, (iz * n + iy) * n + ix, wt * wx[:, 0] * wy[:, 1] * wz[:, 2])
        return mesh.view(n, n, n)

    kfreq = torch.fft.fftfreq(n, d=1.0 / n).to(dev).to(f64)
    kx = torch.arange(n // 2 + 1, dtype=f64, device=dev)
    KZ, KY, KX = kfreq.view(n, 1, 1), kfreq.view(1, n, 1), kx.view(1, 1, -1)
    kk = torch.sqrt(KX * KX + KY * KY + KZ * KZ)
    sinc = lambda a: torch.where(a == 0, torch.ones_like(a), torch.sin(a) / torch.where(a == 0, torch.ones_like(a), a))
    W = (sinc(math.pi * KX / n) * sinc(math.pi * KY / n) * sinc(math.pi * KZ / n)) ** p
    phase = torch.exp(1j * math.pi * (KX + KY + KZ) / n)
    X0 = 0.5 * (torch.fft.rfftn(paint(0.0)) + phase * torch.fft.rfftn(paint(0.5))) / W
    nyq = (KX == n // 2) | (KY == -n // 2) | (KZ == -n // 2)
    b = torch.floor((2 * math.pi / box * kk - kb[0]) / kb[1])
    F0, I = [], []
    for ib in range(kb[2]):
        m = ((b == ib) & (~nyq) & (kk > 0)).to(f64)
        F0.append(torch.fft.irfftn(X0 * m, s=(n, n, n)).flatten() * n ** 3)
        I.append(torch.fft.irfftn(m.to(X0.dtype), s=(n, n, n)).flatten() * n ** 3)
    F0, I = torch.stack(F0), torch.stack(I)
    out = torch.zeros(len(tri), dtype=f64, device=dev)
    for t, (i, j, k) in enumerate(tri):
        s0 = torch.dot(F0[i] * F0[j], F0[k])
        nt = torch.dot(I[i] * I[j], I[k])
        out[t] = s0 / (i33 * nt)
    return out


def power_leg(args, w, world, local, rank, barrier, max_over_ranks):
    """The headline leg: catalogue -> P_l measurements at 512^3, device-resident and end to end."""
    import ctypes as C
    from types import SimpleNamespace

    import torch

    from paper_2605_04864_gb300 import api
    from paper_2605_04864_gb300 import binding as B

    g, r, origin = make_inputs(w, rank)
    dev = lambda c: SimpleNamespace(pos=torch.from_numpy(c.pos).cuda(), w=torch.from_numpy(c.w).cuda(),
                                    nbar=torch.from_numpy(c.nbar).cuda())
    gd, rd = dev(g), dev(r)
    kb = (w["kmin"], w["dk"], w["nbins"])
    kbs = B.npc_kbins(*kb)
    emask = sum(1 << l for l in w["ells"])
    mmask = sum(1 << l for l in w["modified"])
    out_len = B.npc_power_out_len(C.byref(kbs), emask, mmask)
    out = torch.zeros(out_len, dtype=torch.float64, device="cuda")
    kw = dict(n=w["n"], box=w["box"], origin=origin, assign=w["assign"], interlace=w["interlace"], kbins=kb,
              ells=w["ells"], modified=w["modified"], precision=w["precision"])

    def step_dev():
        api.power_multipoles(gd, rd, out=out, **kw)

    api.tune_transforms(w["n"], w["precision"])     # the library's autotuner, before any timing
    for _ in range(args.warmup):
        step_dev()
    torch.cuda.synchronize()
    launches = api.last_stats()["n_kernel_launches"]
    nf = 2 * api.last_stats()["n_r2c_equivalent"] * api.last_stats()["n_phases"] // 2

    # --- device-resident timed region ---
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    s.record()
    marks[0].record()
    for k in range(args.steps):
        step_dev()
        marks[k + 1].record()
    e.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(s.elapsed_time(e))
    ms_per_step = ms / args.steps
    per_step = sorted(marks[k].elapsed_time(marks[k + 1]) for k in range(args.steps))
    pct = lambda q: per_step[min(len(per_step) - 1, int(q * (len(per_step) - 1) + 0.5))]
    step_stats = {"p10": pct(0.1), "median": pct(0.5), "p90": pct(0.9)}
    value = world * args.steps / (ms / 1e3)

    # --- per-stage device times (CUDA events recorded by the library on the same stream) ---
    api.set_profiling(True)
    acc = {}
    for _ in range(args.steps):
        step_dev()
        for name, t, nl in api.stage_times():
            a = acc.setdefault(name, [0.0, 0, 0])
            a[0] += t
            a[1] += nl
            a[2] += 1
    api.set_profiling(False)
    kernel_stages = {k: v for k, v in acc.items()
                     if k in ("paint_count", "paint_scatter", "paint_tiles", "paint_fold", "fft_z_weighted",
                              "fft_y", "fft_x_contract")}
    dom = max(kernel_stages, key=lambda k: kernel_stages[k][0])
    tot_ms, tot_launch, nrep = kernel_stages[dom]
    per_launch_ms = tot_ms / max(tot_launch, 1)
    launches_per_call = tot_launch / nrep
    bytes_call = algorithmic_bytes(w, dom, nf)
    bytes_launch = bytes_call / max(launches_per_call, 1)
    peak, peak_kind = _peaks()
    achieved = bytes_launch / (per_launch_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _traffic(dom), "peak_source": peak_kind,
                "bytes_per_launch": bytes_launch, "launch_ms": per_launch_ms}
    stages = {k: round(v[0] / v[2], 4) for k, v in acc.items()}

    # --- end to end through the C ABI with pinned host catalogues and a host result ---
    pin = lambda c: SimpleNamespace(pos=torch.from_numpy(c.pos).pin_memory(), w=torch.from_numpy(c.w).pin_memory(),
                                    nbar=torch.from_numpy(c.nbar).pin_memory())
    gh, rh = pin(g), pin(r)
    h2d = sum(t.numel() * t.element_size() for c in (gh, rh) for t in (c.pos, c.w, c.nbar))
    d2h = out_len * 8
    api.power_multipoles(gh, rh, **kw)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    s.record()
    for _ in range(args.steps):
        api.power_multipoles(gh, rh, **kw)
    e.record()
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": e2e_s / args.steps * 1e3}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 transforms, f64 accumulators", "data": "synthetic",
            "config": {"workload": args.workload, "mesh": w["n"], "assign": "TSC", "interlace": True,
                       "n_gal": w["n_gal"], "n_ran": w["n_ran"], "ells": list(w["ells"]),
                       "modified": list(w["modified"]), "nbins": w["nbins"], "global_batch": world,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (catalogues 440 MB, meshes 2x537 MB, spectra 16 GB)"},
            "roofline": roofline, "stages_ms": stages, "e2e": e2e, "gpu_launches": launches * args.steps,
            "clocks": clocks, "step_ms": step_stats}
    line["err_vs_fp64"] = power_errors(w, g, r, out.cpu().numpy(), w["nbins"]) if rank == 0 else None
    # the plain GPU form (float64 cuFFT, Hand+17 full-m fields, atomic painting) beside it
    if not args.no_plain:
        ours = out.cpu().numpy()
        del gh, rh
        torch.cuda.empty_cache()
        res, n0 = plain_gpu_power(gd, rd, origin, w)      # warm-up (plans, caches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nrep = 2
        for _ in range(nrep):
            res, n0 = plain_gpu_power(gd, rd, origin, w)
        torch.cuda.synchronize()
        plain_s = (time.perf_counter() - t0) / nrep
        nb = w["nbins"]
        scale = abs(res[0].cpu().numpy()) + n0
        diff = max(float((abs(ours[(2 + e) * nb:(3 + e) * nb] - res[l].cpu().numpy()) / scale).max())
                   for e, l in enumerate((0, 2, 4)))
        line["plain_gpu"] = {"value": world / plain_s, "unit": UNIT, "ms_per_step": plain_s * 1e3,
                             "method": "float64 torch.fft (cuFFT) Hand+17 with 2l+1 real-harmonic fields per l, "
                                       "float64 atomic painting",
                             "max_rel_diff_vs_ours": diff, "speedup_of_ours": value * plain_s / world}
        del res
        # the same plain form in float32 (second GPU baseline)
        res, n0 = plain_gpu_power(gd, rd, origin, w, dtype=torch.float32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(nrep):
            res, n0 = plain_gpu_power(gd, rd, origin, w, dtype=torch.float32)
        torch.cuda.synchronize()
        plain32_s = (time.perf_counter() - t0) / nrep
        diff32 = max(float((abs(ours[(2 + e) * nb:(3 + e) * nb] - res[l].double().cpu().numpy()) / scale).max())
                     for e, l in enumerate((0, 2, 4)))
        line["plain_gpu_f32"] = {"value": world / plain32_s, "unit": UNIT, "ms_per_step": plain32_s * 1e3,
                                 "method": "the same plain form in float32 (cuFFT C2C/R2C float, float atomics)",
                                 "max_rel_diff_vs_ours": diff32, "speedup_of_ours": value * plain32_s / world}
        del res
    del gd, rd, out
    torch.cuda.empty_cache()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, help="power workload name (profiling uses a smaller one)")
    ap.add_argument("--no-power", action="store_true", help="skip the headline leg (profiling of the others)")
    ap.add_argument("--no-bispec", action="store_true", help="skip the 256^3 bispectrum leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 1024^3 gradient leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 96-mock batch leg")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain float64 cuFFT forms of the P_l and B_l legs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    from synthetic import workload

    w = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if not os.path.exists(os.path.join(ROOT, "paper_2605_04864_gb300", "libnpc.so")):
        import __graft_entry__

        __graft_entry__.build()

    barrier, max_over_ranks = rank_collectives(world, "cuda")

    line = {} if args.no_power else power_leg(args, w, world, local, rank, barrier, max_over_ranks)
    if not args.no_bispec:
        sec = bispec_leg(args, world, rank, barrier, max_over_ranks)
        line["secondary"] = sec
        line["gpu_launches"] = line.get("gpu_launches", 0) + sec["gpu_launches"]
    if not args.no_adjoint:
        line["gradient"] = adjoint_leg(args, world, rank, barrier, max_over_ranks)
    if not args.no_batch:
        line["batch"] = batch_leg(args, world, rank, barrier, max_over_ranks)
    if rank == 0 and not args.no_power and not args.no_cpu_baseline and world == 1:
        g, r, origin = make_inputs(w, 0)
        line["cpu_baseline"] = cpu_baseline(w, g, r, origin)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
