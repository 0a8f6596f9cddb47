"""Patch groups and image reconstruction, plain numpy (float64 accumulation).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``; never by
the product library.

Definitions (§IV of the paper):
- group matrix (the equation after Eq. equ:self-convMM): Y_r = [y_S(1), ...,
  y_S(K)], the K matched patches of reference r.  Each patch is vectorised
  row-major over (patch row u, patch column v, channel c):
      Y[r][k][(u*p + v)*C + c] = X[y_k + u][x_k + v][c],  idx[r][k] = y_k*W + x_k.
  An index that is not a top-left corner of the candidate grid
  [0, H-p] x [0, W-p] (for example -1, "no match") gives a zero patch.
- reconstruction ("Image Reconstruction", §IV): each processed patch Z[r][k]
  is deposited back at idx[r][k]; every pixel is divided by the number of
  deposited patches that contain it.  With weights w[r][k] the division is
  by their sum: out = sum w Z / sum w.  Pixels that no patch covers are 0.
"""
from __future__ import annotations

import numpy as np


def _hwc(img):
    a = np.asarray(img)
    return a[:, :, None] if a.ndim == 2 else a


def valid_top_left(idx, H, W, patch):
    """Boolean mask: idx is a top-left corner of the candidate grid."""
    idx = np.asarray(idx, dtype=np.int64)
    y, x = np.divmod(np.where(idx >= 0, idx, 0), W)
    return (idx >= 0) & (idx < H * W) & (y <= H - patch) & (x <= W - patch)


def gather_groups(img, patch, idx):
    """Y[r][k] = the patch at idx[r][k], row-major (u, v, c); zero if invalid."""
    X = _hwc(img)
    H, W, C = X.shape
    idx = np.asarray(idx, dtype=np.int64)
    nR, K = idx.shape
    ok = valid_top_left(idx, H, W, patch)
    y, x = np.divmod(np.where(ok, idx, 0), W)
    u = np.arange(patch)
    rows = y[:, :, None, None] + u[None, None, :, None]          # [nR, K, p, 1]
    cols = x[:, :, None, None] + u[None, None, None, :]          # [nR, K, 1, p]
    patches = X[rows, cols]                                      # [nR, K, p, p, C]
    patches = np.where(ok[:, :, None, None, None], patches, 0).astype(X.dtype)
    return patches.reshape(nR, K, patch * patch * C)


def aggregate(groups, idx, H, W, C, patch, weights=None):
    """Reconstruction of §IV in float64.

    Returns (out [H, W, C], wsum [H, W], abs_sum [H, W, C], count [H, W]):
    out = sum w Z / sum w (0 where sum w == 0), wsum = sum w, abs_sum =
    sum |w Z| and count = number of covering patches (for error bounds).
    """
    Z = np.asarray(groups, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    nR, K = idx.shape
    w = np.ones((nR, K)) if weights is None else np.asarray(weights, dtype=np.float64)
    acc = np.zeros((H, W, C))
    absacc = np.zeros((H, W, C))
    wsum = np.zeros((H, W))
    count = np.zeros((H, W))
    ok = valid_top_left(idx, H, W, patch)
    for r, k in zip(*np.nonzero(ok)):
        y, x = divmod(int(idx[r, k]), W)
        z = Z[r, k].reshape(patch, patch, C)
        acc[y:y + patch, x:x + patch, :] += w[r, k] * z
        absacc[y:y + patch, x:x + patch, :] += np.abs(w[r, k] * z)
        wsum[y:y + patch, x:x + patch] += w[r, k]
        count[y:y + patch, x:x + patch] += 1.0
    out = np.zeros_like(acc)
    nz = wsum != 0
    out[nz] = acc[nz] / wsum[nz][:, None]
    return out, wsum, absacc, count
