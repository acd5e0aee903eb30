import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def tiny():
    from synth import workload
    return workload("tiny")


@pytest.fixture(scope="session")
def tiny_rf(tiny):
    """The tiny ensemble (64 frames, 32+32 elements, 256 samples) as float32."""
    from synth import generate
    return generate(tiny)
