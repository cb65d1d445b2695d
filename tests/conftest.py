import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def tiny():
    """Small random molecules: N=5 atoms, M=3 geometries, noisy enough that all kernel terms matter."""
    from paper_2212_12737_gb300 import synth
    tmpl = synth.template(5, 11)
    R = synth.geometries(tmpl, 3, 0.3, 12)
    return R, tmpl
