import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); parity of the CUDA path")
    config.addinivalue_line("markers", "slow: full-size oracle work (tens of seconds)")


def golden_lines(name):
    """Non-comment lines of a golden fixture, plus the '# key=value' headers."""
    meta, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if line.startswith("#"):
                body = line[1:].strip()
                if "=" in body and " " not in body.split("=")[0]:
                    k, v = body.split("=", 1)
                    meta[k.strip()] = v.strip()
                continue
            if line.strip():
                rows.append(line.split())
    return meta, rows


@pytest.fixture(scope="session")
def golden():
    return golden_lines


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
