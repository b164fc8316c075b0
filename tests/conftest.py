import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built C-ABI library")


@pytest.fixture(scope="session")
def slab_1935():
    from paper_1701_05242_gb300 import synth
    return synth.make_slab(synth.named("slab_1935"))
