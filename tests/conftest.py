import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    # the oracle's results do not depend on its thread count (pinned in test_oracle_lbm.py)
    oracle.set_threads(min(16, os.cpu_count() or 1))
    return oracle
