"""3-D block matching across channels, plain numpy (int64 / float64).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``; never by
the product library.

Definition (§IV, the 3-D Self-Convolution after Eq. equ:self-convMM: patches
of depth d < C channels, searched across channels, the channel sum S(.)
omitted): a 3-D patch at (y, x, c) holds X[y + u][x + v][c + t] for
u, v < p, t < d.  References: the spatial stride grid of block matching at
every channel offset c_r in [0, C - d]; reference index
(ry * n_rx + rx) * (C - d + 1) + c_r.  Candidates of a reference: the clipped
spatial search window of block matching at every channel offset.  Distance:
    d(r, j) = sum_{u, v < p, t < d} (X_r - X_j)^2
(int64 for uint8, float64 for float32).  Output: the K nearest by (distance,
offset) with offset = (y * W + x) * C + c, the flat HWC index of the
candidate's first element; -1 / sentinel padding as in block matching.
"""
from __future__ import annotations

import numpy as np

SENTINEL_U8 = np.int64(2**31 - 1)


def _hwc(img):
    a = np.asarray(img)
    return a[:, :, None] if a.ndim == 2 else a


def match_3d(img, patch, depth, window, stride, K, refs=None):
    X = _hwc(img)
    H, W, C = X.shape
    exact = X.dtype == np.uint8
    Xv = X.astype(np.int64) if exact else X.astype(np.float64)
    p, d, h = patch, depth, (window - 1) // 2
    nc = C - d + 1
    ny, nx = (H - p) // stride + 1, (W - p) // stride + 1
    ids = list(range(ny * nx * nc)) if refs is None else list(refs)
    # all 3-D patches: [H-p+1, W-p+1, nc, p*p*d]
    P = np.lib.stride_tricks.sliding_window_view(Xv, (p, p, d))  # [H-p+1, W-p+1, nc, p, p, d]
    P = P.reshape(H - p + 1, W - p + 1, nc, p * p * d)
    out_idx = np.full((len(ids), K), -1, dtype=np.int32)
    out_d = np.full((len(ids), K), SENTINEL_U8 if exact else np.inf,
                    dtype=np.int64 if exact else np.float64)
    for o, r in enumerate(ids):
        rs, cr = divmod(int(r), nc)
        ry, rx = divmod(rs, nx)
        y, x = ry * stride, rx * stride
        y0, y1 = max(0, y - h), min(H - p, y + h)
        x0, x1 = max(0, x - h), min(W - p, x + h)
        cand = P[y0:y1 + 1, x0:x1 + 1]                        # [wy, wx, nc, n]
        dist = ((cand - P[y, x, cr]) ** 2).sum(axis=-1)      # [wy, wx, nc]
        yy, xx, cc = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), np.arange(nc),
                                 indexing="ij")
        off = (yy * W + xx) * C + cc
        order = np.lexsort((off.reshape(-1), dist.reshape(-1)))[:K]
        out_idx[o, :len(order)] = off.reshape(-1)[order]
        out_d[o, :len(order)] = dist.reshape(-1)[order]
    return out_idx, out_d
