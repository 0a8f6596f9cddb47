"""GPU parity of 3-D block matching across channels (bm_match_3d, through the
C ABI) against the oracle (oracle/bm3d.py).

uint8: indices and distances identical (exact integer distances, fixed
tie-break).  float32: |d_gpu - d_oracle| <= 1e-4 max(d_oracle, 1), and where
indices differ the GPU's candidate is a near-tie of the oracle's at that rank
(the rule of float32 block matching).
"""
import numpy as np
import pytest

from oracle import bm3d as B3
from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth
from parity import sample_refs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.Context(0)
    yield c
    c.close()


def make_image(H, W, C, dt, seed):
    if C == 4 and dt == "u8":
        return synth.rgbnir(H, W, 20.0, seed)
    npdt = np.uint8 if dt == "u8" else np.float32
    return np.ascontiguousarray(np.stack([synth.gray(H, W, 25.0, seed * 10 + c, npdt)
                                          for c in range(C)], axis=-1))


def pair_d(img, p, d, a, b):
    (y1, x1, c1), (y2, x2, c2) = a, b
    A = img[y1:y1 + p, x1:x1 + p, c1:c1 + d].astype(np.float64)
    Bv = img[y2:y2 + p, x2:x2 + p, c2:c2 + d].astype(np.float64)
    return float(((A - Bv) ** 2).sum())


def check(ctx, img, p, d, win, s, K, refs=None):
    H, W, C = img.shape
    gi, gd = ctx.match_3d(torch.from_numpy(img).cuda(), p, d, win, s, K)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    oi, od = B3.match_3d(img, p, d, win, s, K, refs=refs)
    ids = list(range(gi.shape[0])) if refs is None else list(refs)
    gi, gd = gi[ids], gd[ids]
    if img.dtype == np.uint8:
        bad = np.argwhere((gi != oi) | (gd.astype(np.int64) != od))
        assert bad.size == 0, f"{len(bad)} mismatches, first {bad[:3].tolist()}"
        return
    pad = oi < 0
    assert np.array_equal(gi < 0, pad)
    err = np.abs(gd[~pad].astype(np.float64) - od[~pad])
    assert np.all(err <= 1e-4 * np.maximum(od[~pad], 1.0))
    nc, nx = C - d + 1, (W - p) // s + 1
    for r, k in np.argwhere((gi != oi) & ~pad):
        rs, cr = divmod(ids[r], nc)
        ref = ((rs // nx) * s, (rs % nx) * s, cr)
        o = int(gi[r, k])
        cand = (o // C // W, (o // C) % W, o % C)
        assert abs(pair_d(img, p, d, ref, cand) - od[r, k]) <= 1e-4 * max(od[r, k], 1.0)


CASES = [
    # name,        H,   W,  C, dtype, p, d, win, s,  K
    ("u8_c4_d2",   48,  44, 4, "u8",  8, 2, 15, 3, 16),
    ("u8_c3_d1",   40,  37, 3, "u8",  5, 1, 9,  2, 12),
    ("u8_c4_d4",   36,  33, 4, "u8",  4, 4, 11, 2, 8),
    ("u8_c2_d1_k", 20,  22, 2, "u8",  3, 1, 3,  2, 32),
    ("f32_c3_d2",  40,  42, 3, "f32", 4, 2, 13, 3, 16),
    ("f32_c2_d1",  44,  40, 2, "f32", 7, 1, 21, 4, 10),
    # uint8 with a patch side of 4 or 8 takes the integer (dp4a) kernel:
    # windows shorter than its 8-row candidate groups, one channel offset
    # (two-row tiles), ragged borders, K at its limit
    ("u8_c2_d1_p8_w7",  29, 35, 2, "u8", 8, 1, 7,  2, 20),
    ("u8_c1_d1_p4",     33, 30, 1, "u8", 4, 1, 13, 1, 32),
    ("u8_c4_d3_p4",     27, 38, 4, "u8", 4, 3, 17, 2, 32),
    ("u8_c3_d2_p8_s5",  45, 41, 3, "u8", 8, 2, 23, 5, 9),
    ("f32_c4_d2_p8",    36, 34, 4, "f32", 8, 2, 15, 3, 16),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_small_full_parity(ctx, case):
    name, H, W, C, dt, p, d, win, s, K = case
    check(ctx, make_image(H, W, C, dt, seed=H + W * 5 + C), p, d, win, s, K)


def test_saturated_values(ctx):
    # only 0 and 255: the largest squared differences (every partial sum of
    # the integer kernel near its top) and many equal distances, which the
    # offset must order
    rng = np.random.default_rng(77)
    img = np.ascontiguousarray((rng.random((30, 34, 3)) < 0.5).astype(np.uint8) * 255)
    check(ctx, img, 8, 2, 11, 2, 24)
    check(ctx, img, 4, 3, 9, 1, 32)


def test_full_size_sampled_parity(ctx):
    img = make_image(512, 512, 4, "u8", seed=4100)
    ny, nx = B.bm_num_refs(512, 512, 8, 3)
    refs = [r * 3 + c for r in sample_refs(ny, nx, 100, 4100) for c in range(3)]
    check(ctx, img, 8, 2, 39, 3, 16, refs=refs)


def test_invalid_and_unsupported(ctx):
    img = torch.zeros((32, 32, 4), dtype=torch.uint8, device="cuda")
    idx = torch.full((1000,), -7, dtype=torch.int32, device="cuda")
    h = ctx.handle
    rc = B.bm_match_3d(h, img.data_ptr(), 32, 32, 4, B.BM_U8, 4, 5, 5, 2, 8, idx.data_ptr(),
                       idx.data_ptr(), None)
    assert rc == B.BM_ERR_INVALID  # depth > C
    rc = B.bm_match_3d(h, img.data_ptr(), 32, 32, 4, B.BM_U8, 4, 2, 5, 2, 33, idx.data_ptr(),
                       idx.data_ptr(), None)
    assert rc == B.BM_ERR_UNSUPPORTED  # K > 32
    rc = B.bm_match_3d(h, img.data_ptr(), 32, 32, 4, B.BM_U8, 8, 3, 5, 2, 8, idx.data_ptr(),
                       idx.data_ptr(), None)
    assert rc == B.BM_ERR_UNSUPPORTED  # 8 * 8 * 3 > 128
    torch.cuda.synchronize()
    assert bool((idx == -7).all())
