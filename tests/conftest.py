import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built solver library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


def _decode(v):
    if isinstance(v, str):
        return {"inf": np.inf, "-inf": -np.inf}[v]
    return v


class DictLP:
    """Minimal LP record with the fields the oracle and the solver binding read."""

    def __init__(self, d):
        self.m, self.n, self.n_eq = int(d["m"]), int(d["n"]), int(d["n_eq"])
        self.row_ptr = np.array(d["row_ptr"], dtype=np.int32)
        self.col_idx = np.array(d["col_idx"], dtype=np.int32)
        self.val = np.array(d["val"], dtype=np.float64)
        self.c = np.array(d["c"], dtype=np.float64)
        self.q = np.array(d["q"], dtype=np.float64)
        self.l = np.array([_decode(v) for v in d["l"]], dtype=np.float64)
        self.u = np.array([_decode(v) for v in d["u"]], dtype=np.float64)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


@pytest.fixture(scope="session")
def golden():
    with open(os.path.join(HERE, "golden", "hand_examples.json")) as f:
        return json.load(f)
