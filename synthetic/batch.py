"""Inputs of the batched-mocks workload: per-mock sizes and a shared pool of base catalogues.

Every mock takes a prefix of one shuffled lognormal galaxy catalogue and of one uniform random
catalogue generated once (a 1 Gpc/h box rescaled to unit side), scaled to the mock's side L and placed at distance
``distance_factor * L`` from the observer.  (The clustering pattern is therefore one realisation
stretched to each L; the sizes, densities and geometry are those of the workload.)
"""
from __future__ import annotations

import math

import numpy as np

from .catalogs import lognormal_positions, survey_box, uniform_positions


def batch_plan(w):
    """Per-mock dicts (n, box, n_gal, n_ran, distance, origin, nbar, weight, pk_nbins, bk_nbins)."""
    rng = np.random.default_rng(w["seed"])
    out = []
    lo, hi = (math.log(v) for v in w["n_gal_range"])
    for n in w["sizes"]:
        for _ in range(w["per_size"]):
            box = float(rng.uniform(*w["box_range"]))
            n_gal = int(round(math.exp(rng.uniform(lo, hi))))
            n_ran = w["ran_factor"] * n_gal
            dist = w["distance_factor"] * box
            nbar = n_gal / box**3
            k_nyq = math.pi * n / box
            pk_nb = min(w["pk_nbins_max"], int(math.floor(k_nyq / w["dk"] - 1e-9)))
            bk_nb = min(w["bk_nbins"], int(math.floor((0.5 * k_nyq - w["bk_kmin"]) / w["dk"] - 1e-9)))
            out.append(dict(n=n, box=box, n_gal=n_gal, n_ran=n_ran, distance=dist,
                            origin=tuple(float(v) for v in survey_box(box, dist)), nbar=nbar,
                            weight=1.0 / (1.0 + nbar * w["fkp_p0"]), pk_nbins=pk_nb, bk_nbins=bk_nb))
    return out


def base_catalogues(n_gal_max, n_ran_max, n_gen, seed):
    """Unit-box galaxies (lognormal) and randoms (uniform), float32, shuffled so that every prefix is
    a uniform subsample."""
    rng = np.random.default_rng(seed + 17)
    g = lognormal_positions(n_gal_max, 1000.0, n_gen, seed) / 1000.0   # clustered at 1 Gpc/h, rescaled
    g = g[rng.permutation(len(g))]
    r = uniform_positions(n_ran_max, 1.0, seed + 1)
    return g.astype(np.float32), r.astype(np.float32)
