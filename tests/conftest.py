import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def pytest_collection_modifyitems(config, items):
    # GPU tests fail loudly (not skip) when no device is present: they are only
    # selected with -m gpu on a GPU machine.
    pass


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
