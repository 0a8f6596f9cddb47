"""Non-local means weights and estimates, plain numpy (float64).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``; never by
the product library.

Definition (§III-A, Eq. equ:nlm; windowed as in the footnote to Eq.
eq:unifySelfConv; Prop. 1 gives the same weights through Self-Convolution):
for every reference patch X_r of the stride grid and every candidate X_j of
its clipped search window Omega_r (the same geometry as block matching),
    s_r(j) = exp(-||X_j - X_r||_F^2 / b^2) / Theta_r,
    Theta_r = sum_{j in Omega_r} exp(-||X_j - X_r||_F^2 / b^2),
and the estimate of the reference patch is the weighted average
    Xhat_r = sum_j s_r(j) X_j,
vectorised row-major over (patch row u, patch column v, channel c).  The
reference is its own candidate (distance 0), so Theta_r >= 1.
"""
from __future__ import annotations

import numpy as np


def _hwc(img):
    a = np.asarray(img)
    return a[:, :, None] if a.ndim == 2 else a


def nlm(img, patch, window, stride, b, refs=None):
    """Returns (est [n_refs, p*p*C] float64, theta [n_refs] float64, dist_min2 [n_refs])
    where dist_min2 is the smallest distance to a candidate other than the
    reference itself (inf if none), for tolerance reasoning in tests."""
    X = _hwc(img).astype(np.float64)
    H, W, C = X.shape
    p, h = patch, (window - 1) // 2
    ny, nx = (H - p) // stride + 1, (W - p) // stride + 1
    ids = range(ny * nx) if refs is None else refs
    inv_b2 = 1.0 / (float(b) * float(b))
    P = np.lib.stride_tricks.sliding_window_view(X, (p, p, C))[:, :, 0]  # [H-p+1, W-p+1, p, p, C]
    est, theta, dmin2 = [], [], []
    for r in ids:
        ry, rx = divmod(int(r), nx)
        y, x = ry * stride, rx * stride
        y0, y1 = max(0, y - h), min(H - p, y + h)
        x0, x1 = max(0, x - h), min(W - p, x + h)
        cand = P[y0:y1 + 1, x0:x1 + 1].reshape(-1, p * p * C)
        ref = P[y, x].reshape(-1)
        d = ((cand - ref) ** 2).sum(axis=1)
        w = np.exp(-d * inv_b2)
        t = w.sum()
        est.append((w[:, None] * cand).sum(axis=0) / t)
        theta.append(t)
        others = np.ones(len(d), bool)
        others[(y - y0) * (x1 - x0 + 1) + (x - x0)] = False
        dmin2.append(d[others].min() if others.any() else np.inf)
    return np.array(est), np.array(theta), np.array(dmin2)
