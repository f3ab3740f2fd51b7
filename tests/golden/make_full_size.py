"""Writes the stored oracle values for the full-size parity tests (tests/golden/full_size_*.json).

Every number written here comes from ``oracle/`` evaluated on the seeded synthetic inputs of
``synthetic/``; nothing is read from the CUDA library.  Each file records the SHA-256 fingerprint of
the catalogues it was computed from, so a test on another machine can tell whether its own
generated inputs are the same bytes (if not, the tests evaluate the oracle again on their inputs).

    python tests/golden/make_full_size.py power      # 512^3 survey P_l, P_lb (about 10 minutes)
    python tests/golden/make_full_size.py bispec     # 256^3 B_l, B_l0l with analytic shot noise
    python tests/golden/make_full_size.py sugiyama   # 256^3 TripoSH B_000, B_202 (raw)
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))

POWER_FILE = os.path.join(HERE, "full_size_p024b_mixed_512.json")
BISPEC_FILE = os.path.join(HERE, "full_size_bispec_256.json")
SUGIYAMA_FILE = os.path.join(HERE, "full_size_sugiyama_256.json")
SUGIYAMA_MULTIPOLES = ((0, 0, 0), (2, 0, 2))


def _list(a):
    return [float(v) for v in a]


def power_inputs():
    from synthetic import make_survey_catalogs, workload

    w = workload("p024b_mixed_512")
    g, r, origin = make_survey_catalogs(w["n_gal"], w["n_ran"], w["box"], w["distance"], w["n_gen"],
                                        seed=w["seed"], fkp_p0=w["fkp_p0"])
    spec = dict(n=w["n"], box=w["box"], origin=tuple(float(v) for v in origin), assign=w["assign"],
                interlace=w["interlace"], los="endpoint", observer=(0.0, 0.0, 0.0))
    return w, g, r, spec


def power_oracle(w, g, r, spec, workers=None):
    from oracle import power as P

    kb = (w["kmin"], w["dk"], w["nbins"])
    return P.power_multipoles_rfft(spec, g, r, kb, w["ells"], w["modified"], workers=workers)


def bispec_inputs():
    from synthetic import make_periodic_catalog, workload

    w = workload("bispec_256")
    cat = make_periodic_catalog(w["n_gal"], w["box"], w["n_gen"], seed=w["seed"])
    spec = dict(n=w["n"], box=w["box"], origin=(0.0, 0.0, 0.0), assign=w["assign"], interlace=w["interlace"],
                los="global", los_dir=(0.0, 0.0, 1.0), periodic=1)
    return w, cat, spec


def bispec_oracle(w, cat, spec):
    from oracle import bispec as OB

    kb = (w["kmin"], w["dk"], w["nbins"])
    return OB.bispectrum(spec, cat, None, kb, w["scoc_ells"], w["tripo_ells"], shot=True)


def sugiyama_oracle(w, cat, spec):
    import numpy as np

    from oracle import power as P
    from oracle import sugiyama as OS

    kb = (w["kmin"], w["dk"], w["nbins"])
    sc = P.catalog_scalars(cat, None, spec["box"])
    meshes = P.fkp_meshes(spec, cat, None, sc)
    res = OS.sugiyama_fft(spec, meshes, kb, SUGIYAMA_MULTIPOLES, sc["I33"])
    return {mp: np.real(v) for mp, v in res.items()}, OS.mode_counts(spec, kb)


def write_power():
    from synthetic import fingerprint

    w, g, r, spec = power_inputs()
    t0 = time.perf_counter()
    res = power_oracle(w, g, r, spec, workers=os.cpu_count())
    out = {"workload": "p024b_mixed_512", "oracle": "oracle.power.power_multipoles_rfft",
           "fingerprint": fingerprint(g, r), "seconds": time.perf_counter() - t0,
           "k_eff": _list(res["k_eff"]), "nmodes": _list(res["nmodes"]),
           "P": {str(l): _list(v) for l, v in res["P"].items()},
           "Pmod": {str(l): _list(v) for l, v in res["Pmod"].items()},
           "Pll": {f"{a}{c}": _list(v) for (a, c), v in res["Pll"].items()},
           "scalars": {k: float(res["scalars"][k]) for k in ("alpha", "I22", "N0")}}
    with open(POWER_FILE, "w") as f:
        json.dump(out, f, indent=1)


def write_bispec():
    from synthetic import fingerprint

    w, cat, spec = bispec_inputs()
    t0 = time.perf_counter()
    res = bispec_oracle(w, cat, spec)
    out = {"workload": "bispec_256", "oracle": "oracle.bispec.bispectrum (analytic shot noise)",
           "fingerprint": fingerprint(cat), "seconds": time.perf_counter() - t0,
           "tri": res["tri"].tolist(), "pairs": res["pairs"].tolist(), "NT": _list(res["NT"]),
           "B_raw": {str(l): _list(v) for l, v in res["B"].items()},
           "shot_B": {str(l): _list(v) for l, v in res["shot_B"].items()},
           "BB_raw": {str(l): _list(v) for l, v in res["BB"].items()},
           "shot_BB": {str(l): _list(v) for l, v in res["shot_BB"].items()},
           "scalars": {k: float(res["scalars"][k]) for k in ("I33", "S3")}}
    with open(BISPEC_FILE, "w") as f:
        json.dump(out, f, indent=1)


def write_sugiyama():
    from synthetic import fingerprint

    w, cat, spec = bispec_inputs()
    t0 = time.perf_counter()
    res, cnt = sugiyama_oracle(w, cat, spec)
    out = {"workload": "bispec_256", "oracle": "oracle.sugiyama.sugiyama_fft (raw, every sub-configuration)",
           "fingerprint": fingerprint(cat), "seconds": time.perf_counter() - t0, "nmodes": _list(cnt),
           "B_raw": {"".join(str(v) for v in mp): [_list(row) for row in res[mp]] for mp in SUGIYAMA_MULTIPOLES}}
    with open(SUGIYAMA_FILE, "w") as f:
        json.dump(out, f, indent=1)


def load(path):
    with open(path) as f:
        return json.load(f)


if __name__ == "__main__":
    which = sys.argv[1:] or ["power", "bispec", "sugiyama"]
    for name in which:
        {"power": write_power, "bispec": write_bispec, "sugiyama": write_sugiyama}[name]()
        print("wrote", name, flush=True)
