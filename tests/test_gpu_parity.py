"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Small cases are compared in full (several tiles plus ragged tails); the
full-size workloads are compared on a seeded sample of references that
always includes the grid corners and edges.
"""
import zlib

import numpy as np
import pytest

from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth
from parity import compare, sample_refs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.Context(0)
    yield c
    c.close()


def make_image(H, W, C, dtype, seed, sigma=25.0):
    if C == 1:
        return synth.gray(H, W, sigma, seed, np.uint8 if dtype == "u8" else np.float32)
    if C == 4 and dtype == "u8":
        return synth.rgbnir(H, W, sigma, seed)
    planes = [synth.gray(H, W, sigma, seed * 10 + c, np.uint8 if dtype == "u8" else np.float32)
              for c in range(C)]
    return np.ascontiguousarray(np.stack(planes, axis=-1))


def run(ctx, img, p, win, s, K, algo):
    t = torch.from_numpy(img).cuda()
    fn = ctx.match if algo == "selfconv" else ctx.match_direct
    idx, dist = fn(t, p, win, s, K)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


SMALL = [
    # id,             H,   W,  C, dtype, p, win, s,  K
    ("cfg1_tiny",     64,  64, 1, "u8",  8, 21, 1, 16),
    ("cfg2_small",    96,  88, 1, "f32", 8, 39, 3, 16),
    ("cfg3_small",   150, 133, 1, "f32", 7, 61, 4, 70),
    ("cfg4_small",    80,  72, 4, "u8",  8, 39, 3, 32),
    ("cfg4_small_f",  70,  66, 4, "f32", 8, 39, 3, 32),
    ("ragged_u8",     45,  77, 1, "u8",  5,  9, 2, 10),
    ("c2_u8",         40,  50, 2, "u8",  6, 11, 2, 12),
    ("c3_f32",        37,  41, 3, "f32", 4,  7, 1,  8),
    ("p1_fullwin",    20,  30, 1, "u8",  1,  5, 1, 25),
    ("win1_pad",      20,  20, 1, "f32", 3,  1, 2,  4),
    ("k_gt_window",   30,  30, 1, "u8",  4,  5, 3, 40),
    ("p_eq_H",         8,  12, 1, "u8",  8,  7, 1,  5),
    ("p7_c4",         60,  50, 4, "u8",  7, 15, 3, 20),
    ("p16_f32",       50,  50, 1, "f32", 16, 9, 4,  8),
    ("stride5_f32",  101, 203, 1, "f32", 8, 39, 5, 16),
    ("tall_u8",      300,  40, 1, "u8",  8, 39, 3, 16),
    ("c8_u8",         40,  36, 8, "u8",  5,  9, 2, 12),   # the largest channel count
    ("c8_f32",        38,  35, 8, "f32", 4, 11, 3, 10),
]


@pytest.mark.parametrize("algo", ["selfconv", "direct"])
@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_small_full_parity(ctx, case, algo):
    name, H, W, C, dt, p, win, s, K = case
    img = make_image(H, W, C, dt, seed=zlib.crc32(name.encode()) % 10007)
    gidx, gdist = run(ctx, img, p, win, s, K, algo)
    compare(img, p, win, s, K, gidx, gdist)


@pytest.mark.parametrize("algo", ["selfconv", "direct"])
@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_constant_image_tie_break(ctx, algo, dt):
    img = np.full((40, 37), 77, dtype=np.uint8 if dt == "u8" else np.float32)
    gidx, gdist = run(ctx, img, 6, 9, 2, 30, algo)
    compare(img, 6, 9, 2, 30, gidx, gdist)


@pytest.mark.parametrize("sigma", [0.05, 0.0])
def test_float_band_overflow_matches_oracle(ctx, sigma):
    # binary texture: patch distances cluster at multiples of 255^2, so the
    # error band around the K-th pool score holds the whole pool and the
    # re-rank recomputes those windows (sigma 0: exact ties, broken by offset)
    rng = np.random.default_rng(321)
    img = (255.0 * (rng.random((56, 60)) < 0.5) +
           sigma * rng.standard_normal((56, 60))).astype(np.float32)
    before = ctx.stats()["rerank_overflow"]
    gidx, gdist = run(ctx, img, 8, 21, 2, 16, "selfconv")
    assert ctx.stats()["rerank_overflow"] > before
    compare(img, 8, 21, 2, 16, gidx, gdist)


FULL = [
    ("cfg2_512_f32", 512, 512, 1, "f32", 8, 39, 3, 16, 2000),
    ("cfg4_1024x4_u8", 1024, 1024, 4, "u8", 8, 39, 3, 32, 4000),
    ("cfg3_1024_f32", 1024, 1024, 1, "f32", 7, 61, 4, 70, 3000),
    ("cfg1_64_u8", 64, 64, 1, "u8", 8, 21, 1, 16, 1000),
    ("serve_2048_f32", 2048, 2048, 1, "f32", 8, 39, 3, 16, 5000),   # the largest serving side
]


@pytest.mark.parametrize("algo", ["selfconv", "direct"])
@pytest.mark.parametrize("case", FULL, ids=[c[0] for c in FULL])
def test_full_size_sampled_parity(ctx, case, algo):
    name, H, W, C, dt, p, win, s, K, seed = case
    img = make_image(H, W, C, dt, seed=seed, sigma=20.0 if C == 4 else 25.0)
    gidx, gdist = run(ctx, img, p, win, s, K, algo)
    ny, nx = B.bm_num_refs(H, W, p, s)
    refs = sample_refs(ny, nx, 300, seed)
    compare(img, p, win, s, K, gidx, gdist, refs=refs)


WHOLE = [
    # the headline image and one image of the four-channel workload, every
    # reference compared (the oracle on all host cores)
    ("cfg2_512_f32_whole", 512, 512, 1, "f32", 8, 39, 3, 16, 2001),
    ("cfg4_1024x4_u8_whole", 1024, 1024, 4, "u8", 8, 39, 3, 32, 4001),
]


@pytest.mark.parametrize("case", WHOLE, ids=[c[0] for c in WHOLE])
def test_full_size_whole_image_parity(ctx, case):
    name, H, W, C, dt, p, win, s, K, seed = case
    img = make_image(H, W, C, dt, seed=seed, sigma=20.0 if C == 4 else 25.0)
    gidx, gdist = run(ctx, img, p, win, s, K, "selfconv")
    compare(img, p, win, s, K, gidx, gdist, threads=0)


def test_uneven_batch_of_32_in_one_call(ctx):
    """The WNNM-shaped batch: 32 float32 images of seeded uneven sizes
    (256^2 .. 1024^2, sigma 15/25/50), patch 7, stride 4, window 61, K 70,
    in one bm_match_batch call (graph-captured persistent launches).  Every
    image equals its own bm_match bit for bit, and a seeded sample of each
    image's references (with the grid corners and edges) matches the oracle.
    """
    p, win, s, K = 7, 61, 4, 70
    sizes = synth.batch_sizes(32, 3032)
    imgs, outs, reqs, nps = [], [], [], []
    for i, (H, W, sigma) in enumerate(sizes):
        a = synth.gray(H, W, sigma, 3100 + i, np.float32)
        t = torch.from_numpy(a).cuda()
        idx, dist = ctx.outputs(t, p, s, K)
        nps.append(a)
        imgs.append(t)
        outs.append((idx, dist))
        reqs.append(B.Context.request(t, p, win, s, K, idx, dist))
    stream = torch.cuda.Stream()
    ctx.match_batch(reqs, stream=stream)
    torch.cuda.synchronize()
    for i, (a, t, (idx, dist)) in enumerate(zip(nps, imgs, outs)):
        ridx, rdist = ctx.match(t, p, win, s, K)
        torch.cuda.synchronize()
        assert torch.equal(ridx, idx) and torch.equal(rdist, dist), f"image {i}"
        ny, nx = B.bm_num_refs(a.shape[0], a.shape[1], p, s)
        refs = sample_refs(ny, nx, 60, 3200 + i)
        compare(a, p, win, s, K, idx.cpu().numpy(), dist.cpu().numpy(), refs=refs, threads=0)


DIRECT_SHAPES = [
    # the direct kernel's register-blocked shapes (staged union tile, or the
    # image through L1 for the 4-channel window-61 unions), ragged edges
    ("d_p7_c1_w39_f32", 130, 121, 1, "f32", 7, 39, 4, 32),
    ("d_p8_c1_w61_u8", 140, 133, 1, "u8", 8, 61, 3, 16),
    ("d_p7_c4_w39_u8", 120, 117, 4, "u8", 7, 39, 4, 70),
    ("d_p7_c4_w61_f32", 131, 125, 4, "f32", 7, 61, 4, 16),
    ("d_p8_c4_w61_u8", 129, 140, 4, "u8", 8, 61, 3, 70),
    ("d_p8_c4_w61_f32", 110, 97, 4, "f32", 8, 61, 3, 32),
]


@pytest.mark.parametrize("case", DIRECT_SHAPES, ids=[c[0] for c in DIRECT_SHAPES])
def test_direct_kernel_shapes(ctx, case):
    name, H, W, C, dt, p, win, s, K = case
    img = make_image(H, W, C, dt, seed=zlib.crc32(name.encode()) % 10007,
                     sigma=20.0 if C == 4 else 25.0)
    gidx, gdist = run(ctx, img, p, win, s, K, "direct")
    compare(img, p, win, s, K, gidx, gdist, threads=0)


SPLIT_CASES = [
    # jobs small enough that alone they split their windows (bm_window_split > 1)
    ("u8_64", 64, 64, 1, "u8", 8, 21, 1, 16),
    ("f32_96x88", 96, 88, 1, "f32", 8, 39, 3, 16),
    ("f32_k70", 150, 133, 1, "f32", 7, 61, 4, 70),
    ("u8_c4", 80, 72, 4, "u8", 8, 39, 3, 32),
]


@pytest.mark.parametrize("case", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_window_split_equals_unsplit(ctx, case):
    """A job alone splits each tile's window across CTAs and merges the
    parts' lists; the same job inside a batch large enough to occupy the GPU
    runs unsplit.  The two must agree bit for bit (uint8 outputs, float32
    outputs after the re-rank of the merged pool)."""
    name, H, W, C, dt, p, win, s, K = case
    code = B.BM_U8 if dt == "u8" else B.BM_F32
    assert B.bm_window_split(H, W, C, code, p, win, s, K) > 1
    ny, nx = B.bm_num_refs(H, W, p, s)
    n = min(64, -(-304 * 128 * 11 // 10 // (ny * nx)) + 1)  # tiles >= 152 x 2 slots
    imgs, outs, reqs = [], [], []
    for i in range(n):
        t = torch.from_numpy(make_image(H, W, C, dt, seed=600 + i)).cuda()
        idx, dist = ctx.outputs(t, p, s, K)
        imgs.append(t)
        outs.append((idx, dist))
        reqs.append(B.Context.request(t, p, win, s, K, idx, dist))
    ctx.match_batch(reqs, stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    for i in (0, n // 2, n - 1):
        a_idx, a_dist = ctx.match(imgs[i], p, win, s, K)  # alone: split
        torch.cuda.synchronize()
        assert torch.equal(a_idx, outs[i][0]) and torch.equal(a_dist, outs[i][1]), f"image {i}"
    img0 = make_image(H, W, C, dt, seed=600)
    a_idx, a_dist = ctx.match(imgs[0], p, win, s, K)
    torch.cuda.synchronize()
    compare(img0, p, win, s, K, a_idx.cpu().numpy(), a_dist.cpu().numpy())


TS_CASES = [
    # classes whose A operand lives in tensor memory (TS MMAs): the staged tile
    # plus a shared-memory A does not fit
    ("ts_f32_c4_p8", 96, 90, 4, "f32", 8, 39, 3, 16),
    ("ts_f32_c4_p7", 101, 93, 4, "f32", 7, 39, 4, 16),
    ("ts_u8_c4_p8_k70", 110, 97, 4, "u8", 8, 61, 3, 70),
    ("ts_u8_c4_p7_k70", 90, 99, 4, "u8", 7, 39, 4, 70),
    ("ts_f32_c4_p8_w61", 100, 96, 4, "f32", 8, 61, 3, 16),
    ("ts_f32_c4_k70_heap32", 104, 99, 4, "f32", 8, 39, 3, 70),   # 32-bit-key heap
]


@pytest.mark.parametrize("case", TS_CASES, ids=[c[0] for c in TS_CASES])
def test_tensor_memory_a_classes(ctx, case):
    name, H, W, C, dt, p, win, s, K = case
    code = B.BM_U8 if dt == "u8" else B.BM_F32
    assert B.bm_workspace_bytes(H, W, C, code, p, win, s, K) > 0  # the tensor-core path
    img = make_image(H, W, C, dt, seed=zlib.crc32(name.encode()) % 10007, sigma=20.0)
    before = ctx.stats()["tc_jobs"]
    gidx, gdist = run(ctx, img, p, win, s, K, "selfconv")
    assert ctx.stats()["tc_jobs"] == before + 1
    compare(img, p, win, s, K, gidx, gdist, threads=0)


COLUMN_PART_CASES = [
    # classes whose staged tile fits only when each tile's candidate columns
    # are split into contiguous parts, each staging its own columns (and A
    # read from global memory); id, shape, parts the class uses
    ("cp_f32_c4_p8_w61_k32", 110, 97, 4, "f32", 8, 61, 3, 32, 2),
    ("cp_f32_c4_p8_w61_k70", 104, 99, 4, "f32", 8, 61, 3, 70, 2),
    ("cp_f32_c4_p7_w61_k16", 131, 125, 4, "f32", 7, 61, 4, 16, 2),
    ("cp_f32_c4_p7_w61_k70", 120, 111, 4, "f32", 7, 61, 4, 70, 2),   # pool K + 24, 32-bit keys
    ("cp_f32_c4_w61_k128_heap32", 100, 96, 4, "f32", 8, 61, 3, 128, 2),   # 32-bit-key heap
    ("cp_f32_c4_w81_3parts", 90, 84, 4, "f32", 8, 81, 3, 32, 3),
    ("cp_one_column", 70, 8, 4, "f32", 8, 61, 3, 32, 2),   # one candidate column: a part is empty
    ("cp_narrow", 60, 12, 4, "f32", 7, 61, 4, 32, 2),
]


@pytest.mark.parametrize("case", COLUMN_PART_CASES, ids=[c[0] for c in COLUMN_PART_CASES])
def test_column_part_classes(ctx, case):
    name, H, W, C, dt, p, win, s, K, parts = case
    code = B.BM_U8 if dt == "u8" else B.BM_F32
    assert B.bm_workspace_bytes(H, W, C, code, p, win, s, K) > 0  # the tensor-core path
    assert B.bm_window_split(H, W, C, code, p, win, s, K) == parts
    img = make_image(H, W, C, dt, seed=zlib.crc32(name.encode()) % 10007, sigma=20.0)
    before = ctx.stats()["tc_jobs"]
    gidx, gdist = run(ctx, img, p, win, s, K, "selfconv")
    assert ctx.stats()["tc_jobs"] == before + 1
    compare(img, p, win, s, K, gidx, gdist, threads=0)


def test_column_parts_in_a_batch(ctx):
    """Jobs of a column-part class in one batch with others (uneven sizes):
    each equals the same job alone."""
    specs = [(110, 97, 4, "f32", 8, 61, 3, 32), (64, 70, 4, "f32", 8, 61, 3, 32),
             (100, 90, 1, "f32", 8, 39, 3, 16), (200, 41, 4, "f32", 8, 61, 3, 32),
             (96, 96, 4, "f32", 7, 61, 4, 70)]
    imgs, outs, reqs = [], [], []
    for i, (H, W, C, dt, p, win, s, K) in enumerate(specs):
        t = torch.from_numpy(make_image(H, W, C, dt, seed=700 + i, sigma=20.0)).cuda()
        idx, dist = ctx.outputs(t, p, s, K)
        imgs.append(t)
        outs.append((idx, dist))
        reqs.append(B.Context.request(t, p, win, s, K, idx, dist))
    ctx.match_batch(reqs, stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    for (H, W, C, dt, p, win, s, K), t, (idx, dist) in zip(specs, imgs, outs):
        a_idx, a_dist = ctx.match(t, p, win, s, K)
        torch.cuda.synchronize()
        assert torch.equal(a_idx, idx) and torch.equal(a_dist, dist)
    H, W, C, dt, p, win, s, K = specs[3]
    ny, nx = B.bm_num_refs(H, W, p, s)
    compare(make_image(H, W, C, dt, seed=703, sigma=20.0), p, win, s, K, outs[3][0].cpu().numpy(),
            outs[3][1].cpu().numpy(), refs=sample_refs(ny, nx, 80, 704))


def test_selfconv_equals_direct_bitwise_on_u8(ctx):
    img = make_image(200, 180, 1, "u8", seed=5)
    a = run(ctx, img, 8, 39, 3, 16, "selfconv")
    b = run(ctx, img, 8, 39, 3, 16, "direct")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("bad", [
    dict(p=0), dict(p=70), dict(win=4), dict(win=129), dict(s=0), dict(K=0), dict(K=129),
])
def test_invalid_arguments_write_nothing(ctx, bad):
    img = torch.from_numpy(make_image(64, 64, 1, "u8", seed=1)).cuda()
    args = dict(p=8, win=21, s=1, K=16)
    args.update(bad)
    idx = torch.full((57 * 57, 16), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((57 * 57, 16), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BMError) as e:
        ctx.match(img, args["p"], args["win"], args["s"], args["K"], out=(idx, dist))
    assert e.value.code == B.BM_ERR_INVALID
    torch.cuda.synchronize()
    assert bool((idx == -7).all()) and bool((dist == -7).all())


def test_unsupported_patch_volume(ctx):
    img = torch.zeros((64, 64, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.BMError) as e:
        ctx.match(img, 8, 5, 4, 4)
    assert e.value.code == B.BM_ERR_UNSUPPORTED


def test_host_path_equals_device_path(ctx):
    for dt in ("u8", "f32"):
        img = make_image(130, 120, 1, dt, seed=12)
        hidx, hdist = ctx.match_host(img, 8, 39, 3, 16)
        didx, ddist = run(ctx, img, 8, 39, 3, 16, "selfconv")
        assert np.array_equal(hidx, didx) and np.array_equal(hdist, ddist)


def test_batch_equals_single(ctx):
    specs = [(100, 90, 1, "f32", 8, 39, 3, 16), (64, 64, 1, "u8", 8, 21, 1, 16),
             (80, 72, 4, "u8", 8, 39, 3, 32), (150, 133, 1, "f32", 7, 61, 4, 70)]
    imgs, reqs, outs = [], [], []
    for i, (H, W, C, dt, p, win, s, K) in enumerate(specs):
        t = torch.from_numpy(make_image(H, W, C, dt, seed=70 + i)).cuda()
        idx, dist = ctx.outputs(t, p, s, K)
        imgs.append(t)
        outs.append((idx, dist))
        reqs.append(B.Context.request(t, p, win, s, K, idx, dist))
    ctx.match_batch(reqs)
    torch.cuda.synchronize()
    for (H, W, C, dt, p, win, s, K), t, (idx, dist) in zip(specs, imgs, outs):
        a, b = ctx.match(t, p, win, s, K)
        torch.cuda.synchronize()
        assert torch.equal(a, idx) and torch.equal(b, dist)


TC_CASES = [("cfg1", 64, 64, 1, "u8", 8, 21, 1, 16), ("cfg2", 96, 88, 1, "f32", 8, 39, 3, 16),
            ("cfg3", 150, 133, 1, "f32", 7, 61, 4, 70), ("cfg4", 80, 72, 4, "u8", 8, 39, 3, 32)]


@pytest.mark.parametrize("case", TC_CASES, ids=[c[0] for c in TC_CASES])
def test_tensor_core_path_is_used(ctx, case):
    name, H, W, C, dt, p, win, s, K = case
    before = ctx.stats()["tc_jobs"]
    run(ctx, make_image(H, W, C, dt, seed=3), p, win, s, K, "selfconv")
    assert ctx.stats()["tc_jobs"] == before + 1


def test_float_error_bound_never_violated(ctx):
    # every float32 pool entry's identity estimate stays inside eps (n_r + n_j)
    for i, (H, W, p, win, s, K) in enumerate([(200, 180, 8, 39, 3, 16), (160, 150, 7, 61, 4, 70)]):
        run(ctx, make_image(H, W, 1, "f32", seed=40 + i), p, win, s, K, "selfconv")
    st = ctx.stats()
    assert st["bound_violations"] == 0, st


def test_host_batch_equals_device_path(ctx):
    # 20 mixed jobs from page-locked host buffers: more than one chunk, both pipelines
    specs = [(100, 90, 1, "f32", 8, 39, 3, 16), (64, 64, 1, "u8", 8, 21, 1, 16),
             (80, 72, 4, "u8", 8, 39, 3, 32), (150, 133, 1, "f32", 7, 61, 4, 70)] * 5
    imgs, outs, reqs = [], [], []
    for i, (H, W, C, dt, p, win, s, K) in enumerate(specs):
        img = torch.from_numpy(make_image(H, W, C, dt, seed=90 + i)).pin_memory()
        ny, nx = B.bm_num_refs(H, W, p, s)
        idx = torch.full((ny * nx, K), -5, dtype=torch.int32).pin_memory()
        dist = torch.full((ny * nx, K), -5, dtype=torch.int32 if dt == "u8" else torch.float32).pin_memory()
        imgs.append(img)
        outs.append((idx, dist))
        reqs.append(B.Context.request(img, p, win, s, K, idx, dist))
    arr = (B.bm_request * len(reqs))(*reqs)
    assert B.bm_match_host_batch(ctx.handle, arr, len(reqs)) == B.BM_OK
    for (H, W, C, dt, p, win, s, K), img, (idx, dist) in zip(specs, imgs, outs):
        a, b = ctx.match(img.cuda(), p, win, s, K)
        torch.cuda.synchronize()
        assert torch.equal(a.cpu(), idx) and torch.equal(b.cpu(), dist)


@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_largest_window_and_k(ctx, dt):
    # window 127 (the largest odd window) with K = 128 (the largest K)
    img = make_image(150, 140, 1, dt, seed=127)
    gidx, gdist = run(ctx, img, 8, 127, 5, 128, "selfconv")
    compare(img, 8, 127, 5, 128, gidx, gdist)


def test_empty_batches(ctx):
    arr = (B.bm_request * 1)()
    assert B.bm_match_batch(ctx.handle, arr, 0, None) == B.BM_OK
    assert B.bm_match_host_batch(ctx.handle, arr, 0) == B.BM_OK
    assert B.bm_match_batch(ctx.handle, arr, -1, None) == B.BM_ERR_INVALID
