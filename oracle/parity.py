"""Comparison rule between a block-matching result and the oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and
``__graft_entry__.smoke()``; never by the product library.

The rule follows the exactness classes of the method (§III-A, Eq. equ:bm):
- uint8: indices and distances identical (exact integers, tie-break by the
  smaller row-major offset);
- float32: |d - d_oracle| <= 1e-4 * max(d_oracle, 1) position by position;
  where an index differs, the candidate given must lie in the reference's
  clipped window and be a near-tie of the oracle's at that rank (its exact
  distance within the same tolerance), so the K-sets agree except for swaps
  among candidates whose exact distances differ by less than the tolerance;
  no candidate twice in a row.
"""
import numpy as np

from oracle import oracle as O

REL_TOL = 1e-4


def window_ok(off, ry, rx, W, H, p, h):
    y, x = divmod(int(off), W)
    return abs(y - ry) <= h and abs(x - rx) <= h and 0 <= y <= H - p and 0 <= x <= W - p


def compare(img, patch, window, stride, K, gidx, gdist, refs=None, threads=0):
    """Assert results (numpy, rows for `refs` or all refs) match the oracle."""
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
            f"ref {rid} rank {k}: offset {off} d={d_true} vs oracle {oidx[r, k]} d={odist[r, k]}"
    dup = [r for r in range(gidx.shape[0])
           if len(set(gidx[r][gidx[r] >= 0].tolist())) != int((gidx[r] >= 0).sum())]
    assert not dup, f"duplicate candidate in ref {ref_ids[dup[0]]}"


def _report(bad, gidx, gdist, oidx, odist, n=5):
    lines = [f"{len(bad)} mismatches"]
    for r, k in bad[:n]:
        lines.append(f"  ref {r} k {k}: got ({gidx[r, k]}, {gdist[r, k]}) oracle ({oidx[r, k]}, {odist[r, k]})")
    return "\n".join(lines)
