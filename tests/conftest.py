import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the CUDA library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def philox_kat():
    """(counter[4], key[2], expected[4]) of the published Philox4x32-10
    known-answer vectors in tests/golden/philox4x32_10_kat.txt."""
    out = []
    for line in open(os.path.join(ROOT, "tests", "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert len(w) == 10
        out.append((w[0:4], w[4:6], w[6:10]))
    return out
