import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libaceapex.so")
    config.addinivalue_line("markers", "slow: large workloads (run on the GPU box)")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_hex_fixture(name):
    """Parse a hand-written sparse hex fixture: 'length', 'output', 'commands',
    'params' keys and '<offset> <hex bytes>' lines; unlisted bytes are zero."""
    import numpy as np

    meta = {}
    data = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, *rest = line.split()
            if head in ("length", "output", "commands", "params"):
                meta[head] = rest
            else:
                off = int(head)
                for i, h in enumerate(rest):
                    data[off + i] = int(h, 16)
    n = int(meta["length"][0])
    arc = np.zeros(n, dtype=np.uint8)
    for k, v in data.items():
        arc[k] = v
    return arc, meta
