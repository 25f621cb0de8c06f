import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs libpam kernels)")
    config.addinivalue_line("markers", "slow: oracle work of more than a few seconds")


@pytest.fixture(autouse=True)
def _oracle_mutation_off():
    """Every test starts and ends with the oracle unmutated."""
    yield
    mod = sys.modules.get("oracle.oracle")
    if mod is not None and getattr(mod, "_lib", None) is not None:
        mod.set_mutation(0)
