"""Comparison helpers between the CUDA path and the oracle (test infrastructure).

The rule itself (uint8 identical; float32 within 1e-4 relative with near-tie
swaps) lives in ``oracle/parity.py`` so that ``smoke()`` applies the same one.
"""
import numpy as np

from oracle.parity import REL_TOL, compare, window_ok  # noqa: F401


def sample_refs(n_ry, n_rx, count, seed):
    """Seeded reference sample that always includes the four grid corners and edges."""
    rng = np.random.default_rng(seed)
    total = n_ry * n_rx
    picks = set(rng.choice(total, size=min(count, total), replace=False).tolist())
    for ry in (0, n_ry - 1):
        for rx in (0, n_rx - 1, n_rx // 2):
            picks.add(ry * n_rx + rx)
    return sorted(picks)


def load_group_fixture(path):
    """Parse a tests/golden/groups fixture into a dict of numpy arrays and ints."""
    with open(path) as f:
        lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    out, i = {}, 0
    while i < len(lines):
        head = lines[i]
        key = head[0]
        if key == "image":
            H, W, C = map(int, head[1:4])
            rows = [list(map(float, r)) for r in lines[i + 1:i + 1 + H]]
            out["image"] = np.array(rows).reshape(H, W, C)
            i += 1 + H
        elif key == "patch":
            out["patch"] = int(head[1])
            i += 1
        elif key == "idx":
            nR, K = int(head[1]), int(head[2])
            out["idx"] = np.array([list(map(int, r)) for r in lines[i + 1:i + 1 + nR]],
                                  dtype=np.int32).reshape(nR, K)
            i += 1 + nR
        else:  # groups / z / weights (nR rows); out / weight / wout / wweight (H rows)
            nrows = out["idx"].shape[0] if key in ("groups", "z", "weights") else out["image"].shape[0]
            out[key] = np.array([list(map(float, r)) for r in lines[i + 1:i + 1 + nrows]])
            i += 1 + nrows
    nR, K = out["idx"].shape
    for key in ("groups", "z"):
        if key in out:
            out[key] = out[key].reshape(nR, K, -1)
    return out
