import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def load_golden(path):
    """Parse a tests/golden fixture: image, params and expected (offset, distance) rows."""
    import numpy as np
    img_rows, expect, params, shape = [], [], {}, None
    with open(path) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        ln = lines[i]
        if ln.startswith("image"):
            _, H, W, C, dt = ln.split()
            shape = (int(H), int(W), int(C), dt)
            for r in range(int(H)):
                img_rows.append([float(v) for v in lines[i + 1 + r].split()])
            i += 1 + int(H)
            continue
        if ln.startswith("params"):
            for kv in ln.split()[1:]:
                k, v = kv.split("=")
                params[k] = int(v)
        else:
            expect.append([(int(a), float(b)) for a, b in (t.split(":") for t in ln.split())])
        i += 1
    H, W, C, dt = shape
    arr = np.array(img_rows, dtype=np.float64).reshape(H, W, C)
    arr = arr.astype(np.uint8 if dt == "u8" else np.float32)
    return arr, params, expect
