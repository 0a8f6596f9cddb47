"""GPU parity of the patch-group gather and the reconstruction (through the C ABI)
against the numpy oracle (oracle/groups.py).

Gather is a copy: bit-exact.  Reconstruction sums in float32 in an
unspecified order (atomics): every pixel must lie within
(n + 1) * 2^-23 * sum|w Z| / |sum w| + 2^-23 |out| of the float64 oracle,
n the number of covering patches; unweighted coverage counts are exact.
The match indices come from the oracle's block matching (never from the
CUDA path), plus planted invalid entries.
"""
import glob
import os

import numpy as np
import pytest

from oracle import groups as G
from oracle import oracle as O
from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth
from parity import load_group_fixture

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIX = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "groups", "*.txt")))


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


def oracle_idx(img, p, win, s, K, plant_seed=None):
    idx, _ = O.match(img, p, win, s, K)
    idx = idx.astype(np.int32)
    if plant_seed is not None:
        rng = np.random.default_rng(plant_seed)
        H, W = img.shape[:2]
        n = idx.size
        pos = rng.choice(n, size=max(1, n // 50), replace=False)
        bad = np.array([-1, H * W, H * W + 7, (H - p + 1) * W, W - p + 1, -5], dtype=np.int64)
        idx.reshape(-1)[pos] = bad[np.arange(len(pos)) % len(bad)]
    return idx


def check_aggregate(ctx, Z, idx, H, W, C, p, ny, nx, weights=None):
    zt = torch.from_numpy(np.ascontiguousarray(Z, dtype=np.float32)).cuda()
    it = torch.from_numpy(idx).cuda()
    wt = None if weights is None else torch.from_numpy(weights.astype(np.float32)).cuda()
    out, wmap = ctx.aggregate(zt, it, H, W, C, p, ny, nx, weights=wt)
    torch.cuda.synchronize()
    out, wmap = out.cpu().numpy().astype(np.float64), wmap.cpu().numpy().astype(np.float64)
    w64 = None if weights is None else weights.astype(np.float32).astype(np.float64)
    o_out, o_w, o_abs, o_cnt = G.aggregate(Z.astype(np.float32).astype(np.float64), idx, H, W, C,
                                           p, weights=w64)
    u = 2.0 ** -23
    if weights is None:
        assert np.array_equal(wmap, o_cnt), "coverage counts differ"
    else:
        assert np.all(np.abs(wmap - o_w) <= (o_cnt + 1) * u * np.abs(o_w) + 1e-30)
    denom = np.where(o_w != 0, np.abs(o_w), 1.0)[..., None]
    tol = (o_cnt[..., None] + 1) * u * o_abs / denom + u * np.abs(o_out)
    err = np.abs(out - o_out)
    assert np.all(err <= tol + 1e-30), f"max err {err.max():.3e}, worst ratio {np.max(err / (tol + 1e-30)):.3f}"
    assert np.all(out[o_w == 0] == 0)


@pytest.mark.parametrize("path", FIX, ids=[os.path.basename(p) for p in FIX])
def test_group_fixture_on_gpu(ctx, path):
    f = load_group_fixture(path)
    img = f["image"].astype(np.float32)
    H, W, C = img.shape
    p, idx = f["patch"], f["idx"]
    nR, K = idx.shape
    g = ctx.gather_groups(torch.from_numpy(img).cuda(), p, torch.from_numpy(idx).cuda(), nR, 1)
    torch.cuda.synchronize()
    assert np.array_equal(g.cpu().numpy(), f["groups"].astype(np.float32))
    out, wmap = ctx.aggregate(torch.from_numpy(f["z"].astype(np.float32)).cuda(),
                              torch.from_numpy(idx).cuda(), H, W, C, p, nR, 1)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().reshape(H, -1), f["out"].astype(np.float32))
    assert np.array_equal(wmap.cpu().numpy(), f["weight"].astype(np.float32))


GATHER = [
    # name,          H,   W,  C, dtype, p, win, s,  K
    ("g_f32_p8",     90,  77, 1, "f32", 8, 39, 3, 16),
    ("g_u8_p8",      90,  77, 1, "u8",  8, 39, 3, 16),
    ("g_u8_c4",      60,  50, 4, "u8",  8, 15, 3, 32),
    ("g_f32_p7",     70,  66, 1, "f32", 7, 21, 4, 20),
    ("g_u8_p5_c3",   40,  45, 3, "u8",  5, 9,  2, 12),
    ("g_f32_p1",     20,  30, 1, "f32", 1, 5,  1, 25),
]


@pytest.mark.parametrize("case", GATHER, ids=[c[0] for c in GATHER])
def test_gather_bit_exact(ctx, case):
    name, H, W, C, dt, p, win, s, K = case
    img = make_image(H, W, C, dt, seed=len(name) * 31 + H)
    idx = oracle_idx(img, p, win, s, K, plant_seed=H + W)
    ny, nx = B.bm_num_refs(H, W, p, s)
    t = torch.from_numpy(img).cuda()
    g = ctx.gather_groups(t, p, torch.from_numpy(idx).cuda(), ny, nx)
    torch.cuda.synchronize()
    assert np.array_equal(g.cpu().numpy(), G.gather_groups(img, p, idx))


def test_gather_unaligned_output_buffer(ctx):
    img = make_image(50, 40, 1, "f32", seed=8)
    idx = oracle_idx(img, 8, 15, 3, 8)
    ny, nx = B.bm_num_refs(50, 40, 8, 3)
    n = ny * nx * 8 * 64
    buf = torch.full((n + 1,), -3.0, dtype=torch.float32, device="cuda")
    view = buf[1:].view(ny * nx, 8, 64)  # 4-byte aligned, not 16-byte
    ctx.gather_groups(torch.from_numpy(img).cuda(), 8, torch.from_numpy(idx).cuda(), ny, nx,
                      out=view)
    torch.cuda.synchronize()
    assert float(buf[0]) == -3.0
    assert np.array_equal(view.cpu().numpy(), G.gather_groups(img, 8, idx))


AGG = [
    # name,        H,   W,  C, p, win, s,  K, weighted
    ("a_p8",       90,  77, 1, 8, 39, 3, 16, False),
    ("a_p8_w4",    96,  88, 1, 8, 39, 3, 16, False),   # W % 4 == 0: quad reductions
    ("a_c4_w4",    64,  52, 4, 8, 15, 3, 32, True),
    ("a_p5_w4",    48,  44, 1, 5, 11, 2, 12, True),
    ("a_p8_w",     90,  77, 1, 8, 39, 3, 16, True),
    ("a_c4",       60,  50, 4, 8, 15, 3, 32, False),
    ("a_p7_w",     70,  66, 1, 7, 21, 4, 20, True),
    ("a_p5_c3",    40,  45, 3, 5, 9,  2, 12, False),
]


@pytest.mark.parametrize("case", AGG, ids=[c[0] for c in AGG])
def test_aggregate_within_bound(ctx, case):
    name, H, W, C, p, win, s, K, weighted = case
    img = make_image(H, W, C, "f32", seed=H * 3 + C)
    idx = oracle_idx(img, p, win, s, K, plant_seed=H * W)
    ny, nx = B.bm_num_refs(H, W, p, s)
    rng = np.random.default_rng(H + K)
    Z = G.gather_groups(img, p, idx).astype(np.float64) + rng.normal(0, 5.0, size=(ny * nx, K, p * p * C))
    w = rng.uniform(0.1, 2.0, size=(ny * nx, K)) if weighted else None
    check_aggregate(ctx, Z, idx, H, W, C, p, ny, nx, weights=w)


def test_aggregate_scattered_indices(ctx):
    # indices spread over the whole image, four channels: many patches of
    # different references overlap at random
    H, W, C, p = 300, 280, 4, 8
    rng = np.random.default_rng(9)
    ny, nx, K = 12, 10, 24
    ys = rng.integers(0, H - p + 1, size=(ny * nx, K))
    xs = rng.integers(0, W - p + 1, size=(ny * nx, K))
    idx = (ys * W + xs).astype(np.int32)
    Z = rng.normal(100, 30, size=(ny * nx, K, p * p * C))
    check_aggregate(ctx, Z, idx, H, W, C, p, ny, nx)


def test_identity_reconstruction_through_the_gpu_path(ctx):
    # groups gathered on the GPU from the GPU's own matches, aggregated on the
    # GPU: every covered pixel comes back (sums of n equal values / n)
    img = make_image(128, 120, 1, "f32", seed=77)
    t = torch.from_numpy(img).cuda()
    idx, _ = ctx.match(t, 8, 39, 3, 16)
    ny, nx = B.bm_num_refs(128, 120, 8, 3)
    g = ctx.gather_groups(t, 8, idx, ny, nx)
    out, wmap = ctx.aggregate(g, idx, 128, 120, 1, 8, ny, nx)
    torch.cuda.synchronize()
    out, wmap = out.cpu().numpy()[..., 0], wmap.cpu().numpy()
    cov = wmap > 0
    n = wmap[cov]
    assert np.all(np.abs(out[cov] - img[cov]) <= (n + 1) * 2.0 ** -23 * np.abs(img[cov]) * 2)


def test_empty_grid_and_invalid_arguments(ctx):
    img = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    idx = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    g = ctx.gather_groups(img, 4, idx, 0, 0)
    assert g.numel() == 0
    out, wmap = ctx.aggregate(torch.zeros((0, 4, 16), device="cuda"), idx, 16, 16, 1, 4, 0, 0)
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0 and float(wmap.abs().sum()) == 0.0
    h = ctx.handle
    for args in [(0, 16, 1, 4), (16, 16, 9, 4), (16, 16, 1, 0), (16, 16, 1, 17)]:
        H, W, C, p = args
        rc = B.bm_gather_groups(h, img.data_ptr(), H, W, C, B.BM_F32, p, idx.data_ptr(), 1, 1, 4,
                                img.data_ptr(), None)
        assert rc == B.BM_ERR_INVALID
    rc = B.bm_aggregate(h, img.data_ptr(), idx.data_ptr(), None, 1, 1, 4, 16, 16, 1, 4,
                        img.data_ptr(), None, None)
    assert rc == B.BM_ERR_INVALID
    # patch volume beyond 256 elements (9 * 9 * 4): unsupported, as for bm_match
    rc = B.bm_aggregate(h, img.data_ptr(), idx.data_ptr(), None, 1, 1, 4, 16, 16, 4, 9,
                        img.data_ptr(), img.data_ptr(), None)
    assert rc == B.BM_ERR_UNSUPPORTED
