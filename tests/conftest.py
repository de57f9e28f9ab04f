import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU-only checks")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Rows of a golden fixture; entries are exact expressions (fractions, sqrt)."""
    import math
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            rows.append([eval(tok, {"sqrt": math.sqrt, "__builtins__": {}}) if tok != "-" else None
                         for tok in line.split()])
    return rows


def rhs_scale(u, dt_idp):
    """Per-variable scale of a right-hand side: max(|rhs|) is dominated by
    cancellation of much larger flux terms, so residuals are compared against
    max|u_v| / dt_idp, the size of the change of u_v over one IDP step
    (dt_idp = min_i m_i / sum_j 2 d_ij)."""
    import numpy as np
    return np.abs(u).reshape(4, -1).max(axis=1) / dt_idp


def rel_err(a, b, scale):
    """max_v max_i |a - b| / scale_v"""
    import numpy as np
    d = np.abs(np.asarray(a) - np.asarray(b)).reshape(4, -1).max(axis=1)
    return float((d / scale).max())
