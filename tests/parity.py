"""Comparison rules between the CUDA path and the oracle (test infrastructure).

uint8: indices and distances must be identical (exact integers, fixed tie-break).
float32: |d_gpu - d_oracle| <= 1e-4 * max(d_oracle, 1) position by position;
where the indices differ, the GPU's candidate must be a near-tie of the
oracle's at that rank (its exact distance within the same tolerance), i.e.
the K-sets agree except for swaps among candidates whose exact distances
differ by less than the tolerance.
"""
import numpy as np

from oracle import oracle as O

REL_TOL = 1e-4


def window_ok(off, ry, rx, W, H, p, h):
    y, x = divmod(int(off), W)
    return abs(y - ry) <= h and abs(x - rx) <= h and 0 <= y <= H - p and 0 <= x <= W - p


def compare(img, patch, window, stride, K, gidx, gdist, refs=None, threads=0):
    """Assert GPU results (numpy, rows for `refs` or all refs) match the oracle."""
    img3 = img if img.ndim == 3 else img[:, :, None]
    H, W, _ = img3.shape
    oidx, odist = O.match(img3, patch, window, stride, K, refs=refs, threads=threads)
    if refs is not None:
        gidx = gidx[np.asarray(refs)]
        gdist = gdist[np.asarray(refs)]
    if img3.dtype == np.uint8:
        bad = np.argwhere((gidx != oidx) | (gdist.astype(np.int64) != odist))
        assert bad.size == 0, _report(bad, gidx, gdist, oidx, odist)
        return
    h = (window - 1) // 2
    nx = (W - patch) // stride + 1
    ref_ids = list(range(oidx.shape[0])) if refs is None else list(refs)
    assert np.array_equal(gidx < 0, oidx < 0), "padding pattern differs"
    fin = oidx >= 0
    assert np.all(np.isinf(gdist[~fin])) and np.all(np.isinf(odist[~fin]))
    err = np.abs(gdist[fin].astype(np.float64) - odist[fin])
    tol = REL_TOL * np.maximum(odist[fin], 1.0)
    assert np.all(err <= tol), f"max rel err {np.max(err / np.maximum(odist[fin], 1.0)):.3e}"
    for r, k in np.argwhere((gidx != oidx) & fin):
        rid = ref_ids[r]
        ry, rx = (rid // nx) * stride, (rid % nx) * stride
        off = int(gidx[r, k])
        assert window_ok(off, ry, rx, W, H, patch, h), (rid, k, off)
        cy, cx = divmod(off, W)
        d_true = O.pair_distance(img3, patch, (ry, rx), (cy, cx))
        assert abs(d_true - odist[r, k]) <= REL_TOL * max(odist[r, k], 1.0), \
            f"ref {rid} rank {k}: gpu offset {off} d={d_true} vs oracle {oidx[r, k]} d={odist[r, k]}"
    for r in range(gidx.shape[0]):
        v = gidx[r][gidx[r] >= 0]
        assert len(set(v.tolist())) == len(v), f"duplicate candidate in ref {ref_ids[r]}"


def _report(bad, gidx, gdist, oidx, odist, n=5):
    lines = [f"{len(bad)} mismatches"]
    for r, k in bad[:n]:
        lines.append(f"  ref {r} k {k}: gpu ({gidx[r, k]}, {gdist[r, k]}) oracle ({oidx[r, k]}, {odist[r, k]})")
    return "\n".join(lines)


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
