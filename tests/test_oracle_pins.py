"""Pins for the CPU oracle, each against something other than the oracle itself.

- hand-worked fixtures under tests/golden (derivations in their headers);
- closed forms: constant image, one bright pixel, p = 1;
- invariants: shift by a constant, symmetry d(r, j) = d(j, r), d >= 0,
  sorted output, self-distance 0 (footnote to §IV's patch-group equation),
  channel additivity of 3-D patch distances (§IV, Eq. equ:self-convMM);
- Lemma 2 (§III-B) evaluated on its own must equal the definition bit for
  bit on integer images;
- periodic images: exact zero-distance matches at every period multiple.
"""
import glob
import os

import numpy as np
import pytest

from conftest import load_golden
from oracle import oracle as O
from paper_2006_13714_gb300 import synth

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.txt")))


@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p) for p in GOLDEN])
@pytest.mark.parametrize("method", ["direct", "selfconv"])
def test_golden_fixture(path, method):
    img, prm, expect = load_golden(path)
    idx, dist = O.match(img, prm["patch"], prm["window"], prm["stride"], prm["K"], method=method)
    assert idx.shape == (len(expect), prm["K"])
    for r, row in enumerate(expect):
        assert [int(v) for v in idx[r]] == [o for o, _ in row]
        for k, (_, d) in enumerate(row):
            if img.dtype == np.uint8:
                assert int(dist[r, k]) == int(d)
            elif np.isinf(dist[r, k]):
                assert np.isinf(d)
            else:
                assert dist[r, k] == d


def _window_offsets(H, W, p, h, ry, rx):
    ys = range(max(0, ry - h), min(H - p, ry + h) + 1)
    xs = range(max(0, rx - h), min(W - p, rx + h) + 1)
    return [y * W + x for y in ys for x in xs]


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_constant_image_orders_by_offset(dtype):
    H, W, p, win, s = 13, 11, 3, 5, 2
    img = np.full((H, W), 42, dtype=dtype)
    K = win * win
    idx, dist = O.match(img, p, win, s, K)
    ny, nx = O.num_refs(H, W, p, s)
    for r in range(ny * nx):
        ry, rx = (r // nx) * s, (r % nx) * s
        offs = _window_offsets(H, W, p, (win - 1) // 2, ry, rx)
        got = [int(v) for v in idx[r] if v >= 0]
        assert got == offs
        assert np.all(dist[r, :len(offs)] == 0)
        assert np.all(idx[r, len(offs):] == -1)


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_single_bright_pixel_closed_form(dtype):
    # Zero image with one pixel of value v at P.  For two distinct patches the
    # squared distance is v^2 if exactly one covers P, 2 v^2 if both cover it
    # (at different in-patch positions), 0 if neither.
    H, W, p, win, s = 12, 12, 3, 7, 1
    v = 200.0
    P = (5, 6)
    img = np.zeros((H, W), dtype=dtype)
    img[P] = v
    K = win * win
    idx, dist = O.match(img, p, win, s, K)
    ny, nx = O.num_refs(H, W, p, s)

    def covers(y, x):
        return y <= P[0] < y + p and x <= P[1] < x + p

    for r in range(ny * nx):
        ry, rx = (r // nx) * s, (r % nx) * s
        for k in range(K):
            j = int(idx[r, k])
            if j < 0:
                continue
            jy, jx = divmod(j, W)
            if (jy, jx) == (ry, rx):
                want = 0.0
            else:
                want = v * v * (int(covers(ry, rx)) + int(covers(jy, jx)))
            assert float(dist[r, k]) == want


def test_patch_one_is_pixel_difference():
    # p = 1: the patch distance reduces to the squared pixel difference.
    rng = np.random.default_rng(7)
    H, W, win = 9, 10, 5
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    K = win * win
    idx, dist = O.match(img, 1, win, 1, K)
    h = win // 2
    for r in range(H * W):
        ry, rx = divmod(r, W)
        cands = []
        for y in range(max(0, ry - h), min(H - 1, ry + h) + 1):
            for x in range(max(0, rx - h), min(W - 1, rx + h) + 1):
                dd = (int(img[ry, rx]) - int(img[y, x])) ** 2
                cands.append((dd, y * W + x))
        cands.sort()
        n = len(cands)
        assert [int(v) for v in idx[r, :n]] == [o for _, o in cands]
        assert [int(v) for v in dist[r, :n]] == [d for d, _ in cands]


def test_shift_invariance_u8_and_f32():
    img = synth.gray(24, 20, 25, seed=11, dtype=np.uint8)
    img = (img // 2).astype(np.uint8)  # values <= 127, room for +100
    a = O.match(img, 4, 9, 2, 12)
    b = O.match((img + 100).astype(np.uint8), 4, 9, 2, 12)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    f = img.astype(np.float32)
    c = O.match(f, 4, 9, 2, 12)
    d = O.match(f - 1000.0, 4, 9, 2, 12)
    assert np.array_equal(c[0], d[0]) and np.array_equal(c[1], d[1])
    assert np.array_equal(c[0], a[0]) and np.array_equal(c[1].astype(np.int64), a[1])


def test_symmetry_and_basic_invariants():
    H, W, p, win = 16, 15, 3, 7
    img = synth.gray(H, W, 25, seed=5, dtype=np.uint8)
    K = win * win
    idx, dist = O.match(img, p, win, 1, K)
    nx = W - p + 1
    table = {}
    for r in range(idx.shape[0]):
        ry, rx = divmod(r, nx)
        roff = ry * W + rx
        valid = idx[r] >= 0
        d = dist[r][valid]
        o = idx[r][valid]
        assert np.all(d >= 0)
        keys = list(zip(d.tolist(), o.tolist()))
        assert keys == sorted(keys)
        assert d[0] == 0
        assert len(set(o.tolist())) == len(o)
        for dd, oo in keys:
            table[(roff, oo)] = dd
    checked = 0
    for (a, b), d_ab in table.items():
        if (b, a) in table:
            assert table[(b, a)] == d_ab
            checked += 1
    assert checked > 1000


def test_self_is_first_without_earlier_duplicates():
    img = synth.gray(20, 20, 25, seed=3, dtype=np.float32)
    idx, dist = O.match(img, 5, 9, 3, 8)
    ny, nx = O.num_refs(20, 20, 5, 3)
    for r in range(ny * nx):
        ry, rx = (r // nx) * 3, (r % nx) * 3
        assert dist[r, 0] == 0.0
        assert idx[r, 0] == ry * 20 + rx


def test_channel_additivity():
    # A C=4 distance equals the sum of the four single-channel distances.
    img = synth.rgbnir(18, 17, 20, seed=9)
    p, win, s = 4, 7, 2
    K = win * win
    idx4, d4 = O.match(img, p, win, s, K)
    per = [O.match(np.ascontiguousarray(img[:, :, c]), p, win, s, K) for c in range(4)]
    for r in range(idx4.shape[0]):
        total = {}
        for ic, dc in per:
            for o, d in zip(ic[r], dc[r]):
                if o >= 0:
                    total[int(o)] = total.get(int(o), 0) + int(d)
        got = {int(o): int(d) for o, d in zip(idx4[r], d4[r]) if o >= 0}
        assert got == total


@pytest.mark.parametrize("C", [1, 2, 4])
def test_lemma2_equals_definition_exactly_on_integers(C):
    rng = np.random.default_rng(100 + C)
    img = rng.integers(0, 256, size=(21, 19, C), dtype=np.uint8)
    a = O.match(img, 5, 9, 2, 30, method="direct")
    b = O.match(img, 5, 9, 2, 30, method="selfconv")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_lemma2_matches_definition_on_floats():
    img = synth.gray(22, 25, 25, seed=4, dtype=np.float32)
    a = O.match(img, 6, 11, 3, 40, method="direct")
    b = O.match(img, 6, 11, 3, 40, method="selfconv")
    fin = np.isfinite(a[1])
    assert np.array_equal(np.isfinite(b[1]), fin)
    scale = np.maximum(a[1][:, -1:], 1.0)
    # cancellation in ||X_j||^2 + ||X_r||^2 - 2 C_r(j): double rounding only
    assert np.all(np.abs(a[1][fin] - b[1][fin]) <= 1e-9 * np.broadcast_to(scale, a[1].shape)[fin])


def test_periodic_image_zero_matches():
    # Period T dividing the stride: every candidate at a multiple of T from the
    # reference is an exact copy (d = 0); nothing else is.
    T = 3
    rng = np.random.default_rng(1)
    tile = rng.integers(0, 256, size=(T, T), dtype=np.uint8)
    H, W, p, win, s = 18, 21, 4, 9, 3
    img = np.tile(tile, (H // T, W // T))
    K = win * win
    idx, dist = O.match(img, p, win, s, K)
    ny, nx = O.num_refs(H, W, p, s)
    h = win // 2
    for r in range(ny * nx):
        ry, rx = (r // nx) * s, (r % nx) * s
        want = sorted(y * W + x
                      for y in range(max(0, ry - h), min(H - p, ry + h) + 1)
                      for x in range(max(0, rx - h), min(W - p, rx + h) + 1)
                      if (y - ry) % T == 0 and (x - rx) % T == 0)
        zeros = [int(o) for o, d in zip(idx[r], dist[r]) if o >= 0 and d == 0]
        assert zeros == want


def test_reference_subset_rows_match_full_run():
    img = synth.gray(30, 30, 25, seed=8, dtype=np.uint8)
    full = O.match(img, 5, 9, 2, 10)
    refs = [0, 5, 17, 33, full[0].shape[0] - 1]
    sub = O.match(img, 5, 9, 2, 10, refs=refs, threads=2)
    assert np.array_equal(sub[0], full[0][refs]) and np.array_equal(sub[1], full[1][refs])


def test_pair_distance_matches_list():
    img = synth.gray(30, 30, 25, seed=8, dtype=np.float32)
    idx, dist = O.match(img, 5, 9, 2, 10)
    nx = O.num_refs(30, 30, 5, 2)[1]
    for r in (0, 7, 40):
        ry, rx = (r // nx) * 2, (r % nx) * 2
        for k in range(10):
            cy, cx = divmod(int(idx[r, k]), 30)
            assert O.pair_distance(img, 5, (ry, rx), (cy, cx)) == dist[r, k]


def test_invalid_arguments_rejected():
    img = np.zeros((8, 8), np.uint8)
    for args in [(9, 3, 1, 4), (2, 4, 1, 4), (2, 3, 0, 4), (2, 3, 1, 0)]:
        with pytest.raises(ValueError):
            O.match(img, *args)
