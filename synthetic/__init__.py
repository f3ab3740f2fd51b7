"""Seeded synthetic inputs shared by the FP64 oracle, the GPU tests and the benchmark.

This package generates catalogues only: lognormal galaxies with a Kaiser boost, uniform randoms,
and the workload definitions they are drawn for.  It contains none of the estimator arithmetic
(no painting, no Y_lm weighting, no binning): both sides receive the same arrays and compute
independently from them.
"""
from .catalogs import (  # noqa: F401
    power_law_pk,
    gaussian_field,
    lognormal_positions,
    uniform_positions,
    survey_box,
    Catalog,
    make_survey_catalogs,
    make_periodic_catalog,
    fingerprint,
)
from .configs import WORKLOADS, workload  # noqa: F401
from .batch import batch_plan, base_catalogues  # noqa: F401
