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


def golden_module():
    """tests/golden/make_full_size.py as a module (input recipes and the oracle calls it stores)."""
    import importlib.util

    path = os.path.join(ROOT, "tests", "golden", "make_full_size.py")
    spec = importlib.util.spec_from_file_location("make_full_size", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def stored_or_live(path, fp, live):
    """The stored oracle values at ``path`` when they were computed from inputs with fingerprint
    ``fp``; otherwise ``live()`` (the same oracle call on the inputs generated here)."""
    import json

    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if d.get("fingerprint") == fp:
            return d, True
    return live(), False
