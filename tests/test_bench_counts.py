"""The work counts bench.py divides by (CPU): the clipped-window pair count
behind every algorithmic roofline figure, and the issued tensor-core FLOP of
the 512^2 float32 class.

- useful_pairs against brute force over every reference and window offset;
- the issued count against the tile geometry written out factor by factor
  (tiles, union columns, padded union rows, MMAs per column), and against
  its lower bound: every useful pair is computed by all three split products.
"""
import itertools
import math

import bench


def brute_pairs(H, W, p, win, s):
    h = (win - 1) // 2
    n = 0
    for ry, rx in itertools.product(range(0, H - p + 1, s), range(0, W - p + 1, s)):
        for dy, dx in itertools.product(range(-h, h + 1), repeat=2):
            y, x = ry + dy, rx + dx
            n += 0 <= y <= H - p and 0 <= x <= W - p
    return n


def test_useful_pairs_matches_brute_force():
    for H, W, p, win, s in [(20, 17, 4, 7, 3), (16, 16, 8, 9, 1), (13, 29, 5, 21, 2), (9, 9, 9, 3, 1)]:
        assert bench.useful_pairs(H, W, p, win, s) == brute_pairs(H, W, p, win, s)


def test_issued_flop_of_the_bench_class():
    H = W = 512
    p, win, s = 8, 39, 3
    got = bench.tc_issued_flop_per_image(H, W, p, win, s)
    n_ref = (H - p) // s + 1                       # 169 references per axis
    tiles = math.ceil(n_ref / 16) * math.ceil(n_ref / 8)     # 11 x 22
    union_rows = 15 * s + win                      # 84 candidate rows per tile
    union_cols = 7 * s + win                       # 60 candidate columns per tile
    rb = 96                                        # 84 + 7 rounded up to 16
    mmas = 3 * 4 + 1                               # 3 split products x 4 K-steps + norm step
    assert (union_rows + p - 1 + 15) // 16 * 16 == rb
    assert got == tiles * union_cols * mmas * (2 * 128 * rb * 16)
    useful = 2.0 * bench.useful_pairs(H, W, p, win, s) * p * p
    assert got >= 3 * useful
    assert 13.0 < got / useful < 15.0
