"""GPU parity of NCC block matching (bm_match_ncc, through the C ABI) against
the oracle (oracle/ncc.py).

uint8: indices identical (the ranking is exact on both sides); scores within
2^-23 relative (the GPU rounds the exact quotient once, the oracle computes
it in float64).  float32: scores within 2e-5 of the float64 cosine (float32
sums of p*p*C products: relative error ~ (n + 2) 2^-24 in the cross term
and the norms); where the indices differ, the GPU's candidate must be a
near-tie of the oracle's at that rank (its exact cosine within 2e-5).
"""
import math

import numpy as np
import pytest

from oracle import ncc as N
from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth
from parity import sample_refs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_TOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.Context(0)
    yield c
    c.close()


def make_image(H, W, C, dt, seed):
    npdt = np.uint8 if dt == "u8" else np.float32
    if C == 1:
        return synth.gray(H, W, 25.0, seed, npdt)
    return np.ascontiguousarray(np.stack([synth.gray(H, W, 25.0, seed * 10 + c, npdt)
                                          for c in range(C)], axis=-1))


def cosine(img3, p, a_yx, b_yx):
    A = img3[a_yx[0]:a_yx[0] + p, a_yx[1]:a_yx[1] + p].astype(np.float64).reshape(-1)
    Bv = img3[b_yx[0]:b_yx[0] + p, b_yx[1]:b_yx[1] + p].astype(np.float64).reshape(-1)
    na, nb = A @ A, Bv @ Bv
    return 0.0 if na == 0 or nb == 0 else (A @ Bv) / math.sqrt(na * nb)


def check(ctx, img, p, win, s, K, refs=None):
    img3 = img if img.ndim == 3 else img[:, :, None]
    H, W, _ = img3.shape
    gi, gs = ctx.match_ncc(torch.from_numpy(img).cuda(), p, win, s, K)
    torch.cuda.synchronize()
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    oi, os_ = N.match_ncc(img, p, win, s, K, refs=refs)
    ids = list(range(gi.shape[0])) if refs is None else list(refs)
    gi, gs = gi[ids], gs[ids]
    pad = oi < 0
    assert np.array_equal(gi < 0, pad), "padding pattern differs"
    assert np.all(np.isinf(gs[pad])) and np.all(gs[pad] < 0)
    if img.dtype == np.uint8:
        bad = np.argwhere(gi != oi)
        assert bad.size == 0, f"{len(bad)} index mismatches, first {bad[:3].tolist()}"
        rel = np.abs(gs[~pad] - os_[~pad]) / np.maximum(np.abs(os_[~pad]), 1e-30)
        assert np.all((rel <= 2.0 ** -23) | (os_[~pad] == 0)), f"max rel {rel.max():.3e}"
        return
    assert np.all(np.abs(gs[~pad] - os_[~pad]) <= F32_TOL), f"max err {np.abs(gs[~pad] - os_[~pad]).max():.3e}"
    nx = (W - p) // s + 1
    for r, k in np.argwhere((gi != oi) & ~pad):
        rid = ids[r]
        ref = ((rid // nx) * s, (rid % nx) * s)
        cand = divmod(int(gi[r, k]), W)
        assert abs(cosine(img3, p, ref, cand) - os_[r, k]) <= F32_TOL, (rid, k)
    for r in range(gi.shape[0]):
        v = gi[r][gi[r] >= 0]
        assert len(set(v.tolist())) == len(v)


CASES = [
    # name,        H,   W,  C, dtype, p, win, s,  K
    ("u8_p8",      70,  66, 1, "u8",  8, 39, 3, 16),
    ("u8_c4",      50,  46, 4, "u8",  8, 15, 3, 32),
    ("u8_p5_c3",   40,  45, 3, "u8",  5, 9,  2, 12),
    ("u8_k_gt_win", 30, 30, 1, "u8",  4, 5,  3, 40),
    ("f32_p8",     70,  66, 1, "f32", 8, 39, 3, 16),
    ("f32_p7",     60,  57, 1, "f32", 7, 21, 4, 20),
    ("f32_c2_p4",  36,  33, 2, "f32", 4, 11, 2, 8),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_small_full_parity(ctx, case):
    name, H, W, C, dt, p, win, s, K = case
    check(ctx, make_image(H, W, C, dt, seed=H + 3 * W + C), p, win, s, K)


@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_full_size_sampled_parity(ctx, dt):
    img = make_image(512, 512, 1, dt, seed=2001)
    ny, nx = B.bm_num_refs(512, 512, 8, 3)
    check(ctx, img, 8, 39, 3, 16, refs=sample_refs(ny, nx, 200, 2001))


def test_constant_and_zero_images(ctx):
    const = np.full((24, 26), 77, dtype=np.uint8)
    check(ctx, const, 4, 7, 2, 10)       # every score 1: offset order
    zero = np.zeros((24, 26), dtype=np.uint8)
    check(ctx, zero, 4, 7, 2, 10)        # every score 0: offset order


def test_invalid_and_unsupported(ctx):
    img = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    idx = torch.full((15 * 15, 65), -7, dtype=torch.int32, device="cuda")
    sc = torch.full((15 * 15, 65), -7.0, dtype=torch.float32, device="cuda")
    h = ctx.handle
    rc = B.bm_match_ncc(h, img.data_ptr(), 32, 32, 1, B.BM_U8, 4, 5, 2, 65, idx.data_ptr(),
                        sc.data_ptr(), None)
    assert rc == B.BM_ERR_UNSUPPORTED
    rc = B.bm_match_ncc(h, img.data_ptr(), 32, 32, 1, B.BM_U8, 4, 6, 2, 8, idx.data_ptr(),
                        sc.data_ptr(), None)
    assert rc == B.BM_ERR_INVALID
    torch.cuda.synchronize()
    assert bool((idx == -7).all()) and bool((sc == -7.0).all())


@pytest.mark.parametrize("dt", ["u8"])
def test_tensor_core_form_is_used_and_agrees(dt):
    """bm_match_ncc runs its tensor-core form for a supported uint8 class
    (the tensor-core job counter moves) and agrees exactly with the
    CUDA-core kernels (BM_ALGO_DIRECT) and with the oracle."""
    img = make_image(130, 121, 1, dt, seed=77)
    tc = B.Context(0)
    cc = B.Context(0)
    cc.set_algo(B.BM_ALGO_DIRECT)
    t = torch.from_numpy(img).cuda()
    before = tc.stats()["tc_jobs"]
    a_idx, a_sc = tc.match_ncc(t, 8, 39, 3, 16)
    torch.cuda.synchronize()
    assert tc.stats()["tc_jobs"] == before + 1
    b_idx, b_sc = cc.match_ncc(t, 8, 39, 3, 16)
    torch.cuda.synchronize()
    assert cc.stats()["tc_jobs"] == 0
    assert torch.equal(a_idx, b_idx) and torch.equal(a_sc, b_sc)
    check(tc, img, 8, 39, 3, 16)
    for c in (tc, cc):
        c.close()
