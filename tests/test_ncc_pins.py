"""Pins for the NCC block-matching oracle (oracle/ncc.py), each against something
other than the oracle itself:

- a hand-worked 3 x 3 case with an exact rational tie (10/sqrt(500) twice),
  broken by the smaller offset;
- scaled copies of a patch score exactly 1 (Cauchy-Schwarz equality);
- invariants: scale invariance of the ranking, scores in [0, 1] for
  non-negative images, the reference first unless an earlier offset holds a
  positive multiple of it, zero patches score 0;
- the exact uint8 ranking agrees with the float64 ranking of the same image
  wherever the float64 scores are not tied.
"""
import math

import numpy as np

from oracle import ncc as N
from paper_2006_13714_gb300 import synth


def test_hand_worked_with_exact_tie():
    img = np.array([[1, 2, 0], [2, 4, 0], [0, 0, 3]], dtype=np.uint8)
    # patches (2 x 2): (0,0)=[1 2;2 4] n=25, (0,1)=[2 0;4 0] n=20,
    # (1,0)=[2 4;0 0] n=20, (1,1)=[4 0;0 3] n=25; offsets y*3 + x = 0, 1, 3, 4
    idx, sc = N.match_ncc(img, 2, 3, 1, 4)
    # ref (0,0): a = 25, 10, 10, 16 -> 1, 10/sqrt(500), 10/sqrt(500), 16/25
    assert idx[0].tolist() == [0, 4, 1, 3]
    assert np.allclose(sc[0], [1.0, 0.64, 10 / math.sqrt(500), 10 / math.sqrt(500)], atol=1e-15)
    # ref (1,1): a = 16, 8, 8, 25 -> 16/25, 8/sqrt(500), 8/sqrt(500), 1
    assert idx[3].tolist() == [4, 0, 1, 3]
    assert np.allclose(sc[3], [1.0, 0.64, 8 / math.sqrt(500), 8 / math.sqrt(500)], atol=1e-15)


def test_scaled_copies_score_one():
    img = np.zeros((6, 9), dtype=np.uint8)
    img[1:3, 1:3] = [[10, 20], [30, 40]]
    img[1:3, 5:7] = [[20, 40], [60, 80]]       # 2 x the first patch
    idx, sc = N.match_ncc(img, 2, 9, 1, 3, refs=[1 * 8 + 5])  # reference at (1, 5)
    assert idx[0, 0] == 1 * 9 + 1 and idx[0, 1] == 1 * 9 + 5   # tie at 1.0: smaller offset first
    assert sc[0, 0] == 1.0 and sc[0, 1] == 1.0


def test_invariants():
    img = synth.gray(32, 30, 25.0, 21, np.float32)
    img = np.abs(img)  # non-negative
    i1, s1 = N.match_ncc(img, 5, 9, 3, 8)
    i2, s2 = N.match_ncc(img * 4.0, 5, 9, 3, 8)  # a power of two: exact in float32
    assert np.array_equal(i1, i2) and np.allclose(s1, s2, rtol=1e-12)
    assert np.all(s1 <= 1.0 + 1e-12) and np.all(s1 >= 0.0)
    assert np.all(np.diff(s1, axis=1) <= 1e-15)
    nx = (30 - 5) // 3 + 1
    self_off = np.array([(r // nx) * 3 * 30 + (r % nx) * 3 for r in range(i1.shape[0])])
    assert np.mean(i1[:, 0] == self_off) > 0.95
    z = np.zeros((12, 12), dtype=np.uint8)
    z[6:, 6:] = 50
    iz, sz = N.match_ncc(z, 3, 5, 3, 4, refs=[0])
    assert np.all(sz[0] == 0.0) and iz[0].tolist() == [0, 1, 2, 12]  # all zero: offset order


def test_exact_uint8_ranking_matches_float_where_untied():
    img = synth.gray(40, 38, 25.0, 5, np.uint8)
    ie, se = N.match_ncc(img, 4, 7, 2, 10)
    iff, sf = N.match_ncc(img.astype(np.float32), 4, 7, 2, 10)
    assert np.allclose(se, sf, rtol=0, atol=1e-12)
    diff = np.argwhere(ie != iff)
    for r, k in diff:  # only where the float64 scores coincide
        assert abs(se[r, k] - sf[r, k]) < 1e-12
