"""Seeded synthetic images standing in for the paper's workloads.

The paper measures on 512x512 and 256x256 grey-scale denoising and
inpainting images and on the IVRG RGB-NIR scene set (about 1024x768x4,
§V-A and §V-B); none of those images are available, so these generators
stand in for their shapes, value range and noise levels only.  This module
holds no block-matching arithmetic: it only draws pixels.  Both the CUDA
path's tests and the oracle take their inputs from here.

Recipe (numpy ``default_rng(seed)``), one channel:
  base = a*x/W + b*y/H                 linear ramp, a, b ~ U(-60, 60)
       + 12 axis-aligned rectangles / ellipses painted in order with
         constant levels ~ U(0, 255)   (piecewise-constant blobs)
       + 20*sin(2*pi*(fx*x + fy*y) + phi), fx, fy ~ U(1/32, 1/8)
  base is rescaled to [0, 255], then N(0, sigma^2) noise is added;
  uint8 images are rounded half-to-even (np.rint) and clipped to [0, 255],
  float32 images keep the noisy values unclipped.
RGB-NIR: R, G, B share the blob geometry with per-channel levels, ramps
and phases; NIR = 0.5 * (gradient magnitude of a blurred luma)^0.8
rescaled + 0.3 * luma + its own sinusoid; every channel gets its own
N(0, sigma^2) noise, then rounding and clipping.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["gray", "rgbnir", "batch_sizes", "serve_requests", "WNNM_SIZES"]

WNNM_SIZES = ((256, 256), (321, 481), (512, 512), (768, 1024), (1024, 1024))


def _shapes(rng, H, W, n_channels, n_shapes=12):
    layer = np.zeros((n_channels, H, W), dtype=np.float64)
    yy, xx = np.mgrid[0:H, 0:W]
    for _ in range(n_shapes):
        kind = rng.integers(0, 2)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        ry, rx = rng.uniform(H / 16, H / 3), rng.uniform(W / 16, W / 3)
        levels = rng.uniform(0, 255, size=n_channels)
        if kind == 0:
            mask = (np.abs(yy - cy) <= ry) & (np.abs(xx - cx) <= rx)
        else:
            mask = ((yy - cy) / ry) ** 2 + ((xx - cx) / rx) ** 2 <= 1.0
        for c in range(n_channels):
            layer[c][mask] = levels[c]
    return layer


def _ramp_and_wave(rng, H, W):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    a, b = rng.uniform(-60, 60, size=2)
    fx, fy = rng.uniform(1 / 32, 1 / 8, size=2)
    phi = rng.uniform(0, 2 * math.pi)
    return a * xx / W + b * yy / H + 20.0 * np.sin(2 * math.pi * (fx * xx + fy * yy) + phi)


def _rescale(x):
    lo, hi = float(x.min()), float(x.max())
    if hi - lo < 1e-12:
        return np.full_like(x, 127.5)
    return (x - lo) * (255.0 / (hi - lo))


def _finish(x, sigma, rng, dtype):
    x = x + rng.normal(0.0, sigma, size=x.shape)
    if dtype == np.uint8:
        return np.clip(np.rint(x), 0, 255).astype(np.uint8)
    return x.astype(np.float32)


def gray(H: int, W: int, sigma: float, seed: int, dtype=np.uint8) -> np.ndarray:
    """One H x W grey image (uint8 or float32) following the module recipe."""
    dtype = np.dtype(dtype).type
    rng = np.random.default_rng(seed)
    base = _shapes(rng, H, W, 1)[0] + _ramp_and_wave(rng, H, W)
    return _finish(_rescale(base), sigma, rng, dtype)


def _blur(x, s=1.5):
    r = int(math.ceil(3 * s))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / s) ** 2)
    k /= k.sum()
    return _blur_rows(_blur_cols(x, k, r), k, r)


def _blur_cols(x, k, r):
    p = np.pad(x, ((0, 0), (r, r)), mode="edge")
    return sum(k[i] * p[:, i:i + x.shape[1]] for i in range(2 * r + 1))


def _blur_rows(x, k, r):
    p = np.pad(x, ((r, r), (0, 0)), mode="edge")
    return sum(k[i] * p[i:i + x.shape[0], :] for i in range(2 * r + 1))


def rgbnir(H: int, W: int, sigma: float, seed: int) -> np.ndarray:
    """One H x W x 4 uint8 RGB-NIR stack following the module recipe."""
    rng = np.random.default_rng(seed)
    blobs = _shapes(rng, H, W, 3)
    rgb = np.stack([_rescale(blobs[c] + _ramp_and_wave(rng, H, W)) for c in range(3)])
    luma = 0.299 * rgb[0] + 0.587 * rgb[1] + 0.114 * rgb[2]
    sm = _blur(luma)
    gy = np.zeros_like(sm)
    gx = np.zeros_like(sm)
    gy[1:-1, :] = 0.5 * (sm[2:, :] - sm[:-2, :])
    gx[:, 1:-1] = 0.5 * (sm[:, 2:] - sm[:, :-2])
    edges = np.sqrt(gx * gx + gy * gy) ** 0.8
    nir = _rescale(0.5 * _rescale(edges) + 0.3 * luma + _ramp_and_wave(rng, H, W))
    stack = np.stack([rgb[0], rgb[1], rgb[2], nir], axis=-1)
    return _finish(stack, sigma, rng, np.uint8)


def batch_sizes(n: int, seed: int):
    """Seeded (H, W, sigma) draws for the uneven-size WNNM-shaped batch."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        H, W = WNNM_SIZES[int(rng.integers(0, len(WNNM_SIZES)))]
        sigma = float((15, 25, 50)[int(rng.integers(0, 3))])
        out.append((H, W, sigma))
    return out


def serve_requests(n: int, seed: int, rate_per_s: float):
    """Seeded Poisson arrival stream of mixed block-matching requests.

    Each entry: dict(t_arrival, H, W, C, dtype, patch, window, stride, K, seed).
    Stride is 3 for 8x8 patches and 4 for 7x7 patches.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        patch = int((7, 8)[int(rng.integers(0, 2))])
        out.append(dict(
            t_arrival=t,
            H=int(rng.integers(128, 2049)), W=int(rng.integers(128, 2049)),
            C=int((1, 4)[int(rng.integers(0, 2))]),
            dtype=("u8", "f32")[int(rng.integers(0, 2))],
            patch=patch, window=int((39, 61)[int(rng.integers(0, 2))]),
            stride=3 if patch == 8 else 4,
            K=int((16, 32, 70)[int(rng.integers(0, 3))]),
            seed=int(seed * 100003 + i)))
    return out
