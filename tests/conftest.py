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
    config.addinivalue_line("markers", "slow: long-running check")


def load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def lattice_golden():
    rows = load_golden("d2q9_eq19.txt")
    c = np.array([[int(r[1]), int(r[2])] for r in rows], dtype=np.float64)
    w = np.array([int(r[3]) / int(r[4]) for r in rows])
    return c, w


@pytest.fixture(scope="session")
def M_golden():
    return np.array(load_golden("mrt_matrix_eq24.txt"), dtype=np.float64)


@pytest.fixture(scope="session")
def constants_golden():
    return {r[0]: float(r[1]) for r in load_golden("model_constants.txt")}
