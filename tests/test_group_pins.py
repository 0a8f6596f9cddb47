"""Pins for the patch-group / reconstruction oracle (oracle/groups.py), each
against something other than the oracle itself:

- hand-worked fixtures under tests/golden/groups (derivations in their headers),
  which fix the element order (u, v, c) and the normalisation;
- a library special case: the group of a reference's own offset is numpy's
  row-major flattening of the image slice;
- reconstruction of unprocessed groups returns the image at every covered
  pixel (§IV: aggregation of the noisy patches themselves is the identity);
- closed form of the coverage count for self-matches on the stride grid;
- linearity, uniform weights, constant patches, invalid indices.
"""
import glob
import os

import numpy as np
import pytest

from oracle import groups as G
from oracle import oracle as O
from paper_2006_13714_gb300 import synth
from parity import load_group_fixture

FIX = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "groups", "*.txt")))


@pytest.mark.parametrize("path", FIX, ids=[os.path.basename(p) for p in FIX])
def test_group_fixture(path):
    f = load_group_fixture(path)
    img, p, idx = f["image"], f["patch"], f["idx"]
    H, W, C = img.shape
    assert np.array_equal(G.gather_groups(img, p, idx), f["groups"])
    out, wsum, _, count = G.aggregate(f["z"], idx, H, W, C, p)
    assert np.allclose(out.reshape(H, -1), f["out"], rtol=0, atol=1e-12)
    assert np.array_equal(count, f["weight"]) and np.array_equal(wsum, f["weight"])
    if "weights" in f:
        out, wsum, _, _ = G.aggregate(f["z"], idx, H, W, C, p, weights=f["weights"])
        assert np.allclose(out.reshape(H, -1), f["wout"], rtol=0, atol=1e-12)
        assert np.array_equal(wsum, f["wweight"])


def _self_idx(H, W, p, s):
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    ys, xs = np.meshgrid(np.arange(ny) * s, np.arange(nx) * s, indexing="ij")
    return (ys * W + xs).reshape(-1, 1).astype(np.int32), ny, nx


@pytest.mark.parametrize("C", [1, 3])
def test_self_group_is_the_flattened_slice(C):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(23, 19, C)).astype(np.uint8)
    p, s = 5, 3
    idx, ny, nx = _self_idx(23, 19, p, s)
    g = G.gather_groups(img, p, idx)
    for r in range(idx.shape[0]):
        y, x = divmod(int(idx[r, 0]), 19)
        assert np.array_equal(g[r, 0], img[y:y + p, x:x + p, :].flatten(order="C"))


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_reconstruction_of_unprocessed_groups_is_identity(dtype):
    img = synth.gray(60, 52, 25.0, 11, dtype)
    p, win, s, K = 7, 15, 3, 10
    idx, _ = O.match(img, p, win, s, K)
    g = G.gather_groups(img, p, idx).astype(np.float64)
    out, wsum, _, count = G.aggregate(g, idx, 60, 52, 1, p)
    cov = count > 0
    assert np.allclose(out[cov, 0], img.astype(np.float64)[cov], rtol=1e-12, atol=0)
    assert np.all(out[~cov] == 0) and np.array_equal(wsum, count)


def test_coverage_count_closed_form():
    H, W, p, s = 31, 26, 6, 4
    idx, ny, nx = _self_idx(H, W, p, s)
    Z = np.ones((idx.shape[0], 1, p * p))
    _, _, _, count = G.aggregate(Z, idx, H, W, 1, p)
    cy = [sum(1 for a in range(ny) if s * a <= y < s * a + p) for y in range(H)]
    cx = [sum(1 for b in range(nx) if s * b <= x < s * b + p) for x in range(W)]
    assert np.array_equal(count, np.outer(cy, cx).astype(float))


def test_linearity_constants_and_uniform_weights():
    rng = np.random.default_rng(5)
    H, W, C, p = 30, 28, 2, 4
    ok_max = (H - p + 1) * W
    idx = rng.integers(0, ok_max, size=(40, 6)).astype(np.int32)
    Z1 = rng.normal(size=(40, 6, p * p * C))
    Z2 = rng.normal(size=(40, 6, p * p * C))
    a, b = 2.5, -1.25
    o1, _, _, cnt = G.aggregate(Z1, idx, H, W, C, p)
    o2, _, _, _ = G.aggregate(Z2, idx, H, W, C, p)
    o12, _, _, _ = G.aggregate(a * Z1 + b * Z2, idx, H, W, C, p)
    assert np.allclose(o12, a * o1 + b * o2, rtol=1e-12, atol=1e-12)
    oc, _, _, _ = G.aggregate(np.full_like(Z1, 7.0), idx, H, W, C, p)
    assert np.allclose(oc[cnt > 0], 7.0) and np.all(oc[cnt == 0] == 0)
    ow, wsum, _, _ = G.aggregate(Z1, idx, H, W, C, p, weights=np.full((40, 6), 3.0))
    assert np.allclose(ow, o1, rtol=1e-12, atol=1e-12) and np.allclose(wsum, 3.0 * cnt)


def test_invalid_indices_are_zero_and_skipped():
    img = np.arange(5 * 6, dtype=np.float32).reshape(5, 6)
    p = 3
    # -1, past the end, and top-lefts whose patch would leave the image
    idx = np.array([[-1, 5 * 6, 4, 3 * 6 + 1, 2 * 6 + 3]], dtype=np.int32)
    g = G.gather_groups(img, p, idx)
    assert np.all(g[0, :4] == 0)
    assert np.array_equal(g[0, 4], img[2:5, 3:6].flatten())
    out, _, _, count = G.aggregate(np.ones((1, 5, 9)), idx, 5, 6, 1, p)
    assert count.sum() == 9 and np.all(count[2:5, 3:6] == 1)
