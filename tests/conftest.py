import json
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def _num(v):
    if isinstance(v, str):
        return {"inf": math.inf, "-inf": -math.inf}[v]
    return v


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    return d


def arr(values):
    return np.array([_num(v) for v in values], dtype=np.float64)
