"""Shared test helpers (no estimator arithmetic)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    lib = os.path.join(ROOT, "paper_2605_04864_gb300", "libnpc.so")
    if not os.path.exists(lib):
        sys.path.insert(0, ROOT)
        import __graft_entry__

        __graft_entry__.build()
    return lib


def p_error(gpu, orc, mono_scale):
    """Error metric for multipoles that cross zero: |X_gpu - X_orc| / max(|X_orc|, |P_0| + N_0)."""
    gpu, orc = np.asarray(gpu), np.asarray(orc)
    return np.abs(gpu - orc) / np.maximum(np.abs(orc), mono_scale)
