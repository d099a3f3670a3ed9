import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def _paper_parameters():
    """tests/golden/paper_parameters.txt: name -> value, each line citing where the paper prints it."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                out[name] = float(value)
    return out


@pytest.fixture(scope="session")
def paper():
    return _paper_parameters()
