import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def golden(name):
    """key = value lines of tests/golden/<name>.txt (values: one number, or a
    list of numbers separated by spaces); '#' starts a comment."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + ".txt")
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (x.strip() for x in line.split("=", 1))
            nums = [float(v) for v in val.split()]
            out[key] = nums if len(nums) > 1 else nums[0]
    return out
