import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")


@pytest.fixture(scope="session", autouse=True)
def _built_cpu_parts():
    """The oracle and the input generator are plain C; build them once per session."""
    import oracle
    import synth

    oracle.build()
    synth.build()
    yield
