import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def bits_from_string(s):
    """'101010' -> bit mask with the leftmost character as orbital 1 (bit 0)."""
    return sum(1 << p for p, ch in enumerate(s) if ch == "1")


def string_from_bits(x, n):
    return "".join("1" if (x >> p) & 1 else "0" for p in range(n))


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
