import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# A copy of the oracle package with one planted mistake (test_oracle_mutants.py)
# is imported in place of the repository's when GBMC_ORACLE_DIR names it.
if os.environ.get("GBMC_ORACLE_DIR"):
    sys.path.insert(0, os.environ["GBMC_ORACLE_DIR"])


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
