"""Pins for the non-local means oracle (oracle/nlm.py), each against something
other than the oracle itself:

- a hand-worked case in closed form (binary image, patch 1: every weight is
  1 or e^(-1/b^2));
- limits: b -> infinity gives the plain mean of the window's patches
  (written out here with explicit loops), b -> 0 gives the reference patch;
- a constant image: estimate = the constant, Theta = the window size;
- invariants: shift by a constant, Theta >= 1, estimates inside the hull of
  the window's values, a zero second channel changes nothing in the first.
"""
import math

import numpy as np
import pytest

from oracle import nlm as N
from paper_2006_13714_gb300 import synth


def test_hand_worked_binary_patch_one():
    # image [[0 1 0], [1 0 1]], patch 1, window 3, stride 1, b 1: each weight
    # is 1 (same value) or e^-1 (other value).  Reference (0,0) = 0 sees
    # {0, 1, 1, 0} -> estimate 2 e^-1 / (2 + 2 e^-1) = 1 / (e + 1).
    img = np.array([[0, 1, 0], [1, 0, 1]], dtype=np.float64)
    est, theta, _ = N.nlm(img, 1, 3, 1, 1.0)
    e1 = math.exp(-1.0)
    # window of each pixel (clipped 3 x 3): counts of equal / other values
    expect, th = [], []
    for y in range(2):
        for x in range(3):
            v = img[y, x]
            same = other = 0
            for yy in range(max(0, y - 1), min(1, y + 1) + 1):
                for xx in range(max(0, x - 1), min(2, x + 1) + 1):
                    if img[yy, xx] == v:
                        same += 1
                    else:
                        other += 1
            t = same + other * e1
            expect.append((same * v + other * e1 * (1 - v)) / t)
            th.append(t)
    assert abs(est[0, 0] - 1.0 / (math.e + 1.0)) < 1e-15
    assert np.allclose(est[:, 0], expect, rtol=0, atol=1e-15)
    assert np.allclose(theta, th, rtol=1e-15, atol=0)


def _window_patches(img, p, h, y, x):
    H, W = img.shape[:2]
    out = []
    for yy in range(max(0, y - h), min(H - p, y + h) + 1):
        for xx in range(max(0, x - h), min(W - p, x + h) + 1):
            out.append(img[yy:yy + p, xx:xx + p].reshape(-1))
    return np.array(out, dtype=np.float64)


def test_large_b_is_the_window_mean_and_small_b_the_reference():
    img = synth.gray(30, 27, 25.0, 4, np.float32)
    p, win, s = 5, 9, 3
    est, theta, _ = N.nlm(img, p, win, s, 1e9)
    nx = (27 - p) // s + 1
    for r in range(est.shape[0]):
        y, x = (r // nx) * s, (r % nx) * s
        P = _window_patches(img, p, 4, y, x)
        assert np.allclose(est[r], P.mean(axis=0), rtol=1e-9, atol=1e-9)
        assert abs(theta[r] - len(P)) < 1e-6
    est0, theta0, _ = N.nlm(img, p, win, s, 1e-3)
    for r in range(est0.shape[0]):
        y, x = (r // nx) * s, (r % nx) * s
        assert np.array_equal(est0[r], img[y:y + p, x:x + p].astype(np.float64).reshape(-1))
        assert theta0[r] == 1.0


def test_constant_image():
    img = np.full((20, 17), 42.0, dtype=np.float32)
    est, theta, _ = N.nlm(img, 4, 7, 2, 10.0)
    assert np.all(est == 42.0)
    nx = (17 - 4) // 2 + 1
    for r in range(len(theta)):
        y, x = (r // nx) * 2, (r % nx) * 2
        ny_ = min(16, y + 3) - max(0, y - 3) + 1
        nx_ = min(13, x + 3) - max(0, x - 3) + 1
        assert theta[r] == ny_ * nx_


def test_shift_invariance_hull_and_theta():
    img = synth.gray(40, 36, 25.0, 9, np.float32).astype(np.float64)
    p, win, s, b = 6, 11, 2, 60.0
    est, theta, _ = N.nlm(img, p, win, s, b)
    est2, theta2, _ = N.nlm(img + 123.25, p, win, s, b)
    assert np.allclose(est2, est + 123.25, rtol=0, atol=1e-9)
    assert np.allclose(theta2, theta, rtol=1e-12)
    assert np.all(theta >= 1.0)
    nx = (36 - p) // s + 1
    for r in range(0, est.shape[0], 7):
        y, x = (r // nx) * s, (r % nx) * s
        P = _window_patches(img, p, 5, y, x)
        assert np.all(est[r] >= P.min(axis=0) - 1e-9) and np.all(est[r] <= P.max(axis=0) + 1e-9)


def test_zero_second_channel_changes_nothing():
    a = synth.gray(24, 22, 25.0, 13, np.float32)
    two = np.stack([a, np.zeros_like(a)], axis=-1)
    e1, t1, _ = N.nlm(a, 4, 7, 3, 40.0)
    e2, t2, _ = N.nlm(two, 4, 7, 3, 40.0)
    e2 = e2.reshape(len(t2), 16, 2)
    assert np.allclose(e2[..., 0], e1, rtol=1e-12, atol=1e-12)
    assert np.all(e2[..., 1] == 0) and np.allclose(t1, t2, rtol=1e-12)
