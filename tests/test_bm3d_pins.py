"""Pins for the 3-D block-matching oracle (oracle/bm3d.py), each against
something other than the oracle itself:

- depth = C (one channel offset) is ordinary multi-channel block matching
  (§IV's channel sum): equal to the C block-matching oracle, offsets times C;
- a hand-worked 2 x 2 x 3 case with patch 1, depth 1 (distances are squared
  value differences across pixels and channels);
- invariants: shift by a constant, symmetry d(r, j) = d(j, r), d >= 0 and
  sorted, self-distance 0 first;
- duplicated channels give a zero-distance match at the next channel offset.
"""
import numpy as np
import pytest

from oracle import bm3d as B3
from oracle import oracle as O
from paper_2006_13714_gb300 import synth


@pytest.mark.parametrize("dt", [np.uint8, np.float32])
def test_full_depth_equals_channel_sum_block_matching(dt):
    img = np.ascontiguousarray(np.stack([synth.gray(30, 28, 25.0, 40 + c, dt) for c in range(3)], axis=-1))
    i3, d3 = B3.match_3d(img, 4, 3, 9, 2, 10)
    i2, d2 = O.match(img, 4, 9, 2, 10)
    assert np.array_equal(i3, np.where(i2 >= 0, i2 * 3, -1))
    if dt == np.uint8:
        assert np.array_equal(d3, d2)
    else:
        assert np.allclose(d3, d2, rtol=1e-12, atol=1e-9)


def test_hand_worked_patch_one_depth_one():
    # pixel (0,0) = [0 10 20], (0,1) = [1 11 21], (1,0) = [5 15 25], (1,1) = [30 2 12];
    # offsets (y*2 + x)*3 + c.  Reference (0,0,c=0) holds 0; the candidates' values in
    # offset order are 0 10 20 1 11 21 5 15 25 30 2 12, squared differences
    # 0 100 400 1 121 441 25 225 625 900 4 144 -> nearest: offsets 0, 3, 10, 6.
    img = np.array([[[0, 10, 20], [1, 11, 21]], [[5, 15, 25], [30, 2, 12]]], dtype=np.uint8)
    idx, dist = B3.match_3d(img, 1, 1, 3, 1, 4, refs=[0])
    assert idx[0].tolist() == [0, 3, 10, 6] and dist[0].tolist() == [0, 1, 4, 25]
    # reference (1,1,c=1) holds 2: differences to 0 10 20 1 11 21 5 15 25 30 2 12 are
    # 2 8 18 1 9 19 3 13 23 28 0 10 -> offsets 10 (0), 3 (1), 0 (4), 6 (9)
    idx, dist = B3.match_3d(img, 1, 1, 3, 1, 4, refs=[(1 * 2 + 1) * 3 + 1])
    assert idx[0].tolist() == [10, 3, 0, 6] and dist[0].tolist() == [0, 1, 4, 9]


def test_invariants():
    img = np.ascontiguousarray(np.stack([synth.gray(26, 24, 25.0, 7 + c, np.uint8) for c in range(4)], axis=-1))
    p, d, win, s, K = 4, 2, 7, 3, 12
    idx, dist = B3.match_3d(img, p, d, win, s, K)
    idx2, dist2 = B3.match_3d((img.astype(np.float32) + 17.0), p, d, win, s, K)
    assert np.array_equal(idx, idx2) and np.allclose(dist, dist2)
    assert np.all(dist >= 0) and np.all(np.diff(dist, axis=1) >= 0)
    H, W, C = img.shape
    nc, nx = C - d + 1, (W - p) // s + 1
    for r in range(idx.shape[0]):
        rs, cr = divmod(r, nc)
        y, x = (rs // nx) * s, (rs % nx) * s
        assert dist[r, 0] == 0
    # symmetry: reference pairs that are candidates of each other
    full_i, full_d = B3.match_3d(img, p, d, win, s, 200)
    lut = {}
    for r in range(full_i.shape[0]):
        rs, cr = divmod(r, nc)
        y, x = (rs // nx) * s, (rs % nx) * s
        lut[((y * W + x) * C + cr)] = r
    checked = 0
    for r in range(full_i.shape[0]):
        rs, cr = divmod(r, nc)
        y, x = (rs // nx) * s, (rs % nx) * s
        me = (y * W + x) * C + cr
        for k in range(full_i.shape[1]):
            o = int(full_i[r, k])
            if o in lut:
                r2 = lut[o]
                j = np.nonzero(full_i[r2] == me)[0]
                if len(j):
                    assert full_d[r2, j[0]] == full_d[r, k]
                    checked += 1
    assert checked > 100


def test_duplicated_channels_match_at_the_next_offset():
    a = synth.gray(20, 20, 25.0, 3, np.uint8)
    img = np.ascontiguousarray(np.stack([a, a, a], axis=-1))
    idx, dist = B3.match_3d(img, 3, 1, 5, 4, 3, refs=[0])
    # reference (0,0,0): the same pixel at channel offsets 0, 1, 2 are all at distance 0
    assert idx[0].tolist() == [0, 1, 2] and dist[0].tolist() == [0, 0, 0]
