import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built engine")


def pytest_collection_modifyitems(config, items):
    # A GPU test on a machine without a GPU is an error to surface, not a skip:
    # leave the marker selection (-m gpu / -m "not gpu") to the caller.
    pass


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.load()
