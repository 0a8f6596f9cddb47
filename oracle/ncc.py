"""Block matching by normalized cross-correlation, plain numpy / Python integers.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``; never by
the product library.

Definition (§III-A, Eq. equ:cor; Lemma 1 and Theorem 1, case 3, give the same
ranking through Self-Convolution): over the same clipped search windows and
reference grid as Euclidean block matching, the K candidates with the
largest
    ncc(r, j) = <X_r, X_j> / (||X_r||_F ||X_j||_F)
(the uncentred cosine; a patch of zero norm scores 0), ties broken by the
smaller row-major offset y*W + x.  uint8 images are ranked exactly: with
a_j = <X_r, X_j> >= 0 and n_j = ||X_j||^2 integers, a_j / sqrt(n_j) is
compared through a_j^2 n_k versus a_k^2 n_j in Python's unbounded integers.
float32 images are ranked by the float64 score.
Returns (idx int32 [n_refs, K] with -1 padding, score float64 [n_refs, K]
with -inf padding).
"""
from __future__ import annotations

import functools
import math

import numpy as np


def _hwc(img):
    a = np.asarray(img)
    return a[:, :, None] if a.ndim == 2 else a


def match_ncc(img, patch, window, stride, K, refs=None):
    X = _hwc(img)
    H, W, C = X.shape
    exact = X.dtype == np.uint8
    Xv = X.astype(np.int64) if exact else X.astype(np.float64)
    p, h = patch, (window - 1) // 2
    ny, nx = (H - p) // stride + 1, (W - p) // stride + 1
    ids = list(range(ny * nx)) if refs is None else list(refs)
    P = np.lib.stride_tricks.sliding_window_view(Xv, (p, p, C))[:, :, 0].reshape(H - p + 1, W - p + 1, -1)
    out_idx = np.full((len(ids), K), -1, dtype=np.int32)
    out_sc = np.full((len(ids), K), -np.inf)
    for o, r in enumerate(ids):
        ry, rx = divmod(int(r), nx)
        y, x = ry * stride, rx * stride
        y0, y1 = max(0, y - h), min(H - p, y + h)
        x0, x1 = max(0, x - h), min(W - p, x + h)
        ref = P[y, x]
        nr = int(ref @ ref) if exact else float(ref @ ref)
        cands = []
        for yy in range(y0, y1 + 1):
            for xx in range(x0, x1 + 1):
                c = P[yy, xx]
                a = c @ ref
                n = c @ c
                if exact:
                    a, n = int(a), int(n)
                    if n == 0 or nr == 0:
                        a, n = 0, 1
                cands.append((a, n, yy * W + xx))
        if exact:
            def cmp(s, t):
                lhs, rhs = s[0] * s[0] * t[1], t[0] * t[0] * s[1]
                if lhs != rhs:
                    return -1 if lhs > rhs else 1
                return -1 if s[2] < t[2] else (1 if s[2] > t[2] else 0)
            cands.sort(key=functools.cmp_to_key(cmp))
            top = cands[:K]
            scores = [a / math.sqrt(float(nr) * n) if nr > 0 else 0.0 for a, n, _ in top]
        else:
            sc = [(a / math.sqrt(nr * n) if nr > 0 and n > 0 else 0.0, off) for a, n, off in cands]
            order = sorted(range(len(sc)), key=lambda i: (-sc[i][0], sc[i][1]))[:K]
            top = [cands[i] for i in order]
            scores = [sc[i][0] for i in order]
        for k, ((_, _, off), s) in enumerate(zip(top, scores)):
            out_idx[o, k] = off
            out_sc[o, k] = s
    return out_idx, out_sc
