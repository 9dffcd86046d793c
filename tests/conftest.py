import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the CUDA library")
    config.addinivalue_line("markers", "slow: statistical test taking tens of seconds")


@pytest.fixture(scope="session")
def tiny_corpus():
    from paper_1510_08628_gb300 import corpus
    return corpus.generate("tiny", seed=1)
