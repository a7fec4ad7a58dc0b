import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the mutation tests run the oracle pins against a copy of the oracle package
# with one planted mistake, found first on the path
if os.environ.get("AEB_ORACLE_PKG_ROOT"):
    sys.path.insert(0, os.environ["AEB_ORACLE_PKG_ROOT"])


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle
