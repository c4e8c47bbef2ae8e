import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CUTS_FILE = os.path.join(ROOT, "paper_2501_05520_gb300", "params", "cuts_v1.json")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def load_cuts(which: str = "pt_min_0p45") -> dict:
    with open(CUTS_FILE) as f:
        d = json.load(f)[which]
    return {k: d[k] for k in ("kmax", "z0max", "cotmax", "rz0", "rz1", "dca_b0", "dca_other")}


@pytest.fixture(scope="session")
def cuts():
    return load_cuts("pt_min_0p45")


@pytest.fixture(scope="session")
def cuts_low_pt():
    return load_cuts("pt_min_0p25")
