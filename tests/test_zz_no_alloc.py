"""bm_match_static, the entry point that allocates nothing, against bm_match.

Both are called through the C ABI (the binding's functions with the C
names).  The comparison uses the float32 tolerance of the other parity
tests (|d_a - d_b| <= 1e-4 * max(d_b, 1); where indices differ the two
candidates must be such a near-tie); uint8 must be identical.
"""
import numpy as np
import pytest

from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth

REL_TOL = 1e-4


def _agree(idx_a, dist_a, idx_b, dist_b, is_u8):
    if is_u8:
        assert np.array_equal(idx_a, idx_b)
        assert np.array_equal(dist_a, dist_b)
        return
    assert np.array_equal(idx_a < 0, idx_b < 0)
    fin = idx_b >= 0
    a = dist_a[fin].astype(np.float64)
    b = dist_b[fin].astype(np.float64)
    assert np.all(np.abs(a - b) <= REL_TOL * np.maximum(b, 1.0))
    # a differing index is a near-tie swap: inside the row it moved rank
    # among equal-within-tolerance distances, or it left the K-set at the
    # boundary (its distance within the tolerance of the K-th)
    for r in np.nonzero((fin & (idx_a != idx_b)).any(axis=1))[0]:
        kth = float(dist_b[r][fin[r]][-1])
        for j in np.nonzero(fin[r] & (idx_a[r] != idx_b[r]))[0]:
            if idx_a[r, j] in idx_b[r]:
                continue
            assert abs(float(dist_a[r, j]) - kth) <= REL_TOL * max(kth, 1.0)


def _static(img, p, win, s, K, idx, dist, stream):
    H, W = img.shape[0], img.shape[1]
    C = 1 if img.dim() == 2 else img.shape[2]
    import torch
    dt = B.BM_U8 if img.dtype == torch.uint8 else B.BM_F32
    return B.bm_match_static(img.data_ptr(), H, W, C, dt, p, win, s, K, idx.data_ptr(),
                             dist.data_ptr(), stream.cuda_stream)


def test_scratch_bytes_host_only():
    # 512 x 512 float32, p 8, s 3, window 39, K 16: planes + norms + pool
    n = B.bm_static_scratch_bytes(512, 512, 1, B.BM_F32, 8, 39, 3, 16)
    assert 0 < n <= B.BM_STATIC_SCRATCH_BYTES
    assert B.bm_static_scratch_bytes(2048, 2048, 1, B.BM_F32, 8, 39, 3, 16) > \
        B.BM_STATIC_SCRATCH_BYTES
    assert B.bm_static_scratch_bytes(64, 64, 1, B.BM_U8, 8, 38, 3, 16) == 0  # even window


@pytest.mark.gpu
def test_static_equals_bm_match_on_two_calls_in_a_row():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    jobs = [
        (synth.gray(512, 512, 20.0, 7001, np.float32), 8, 39, 3, 16),
        (synth.gray(300, 277, 15.0, 7002, np.uint8), 8, 39, 3, 16),
    ]
    ctx = B.Context(0)
    st = torch.cuda.current_stream()
    imgs, outs_static = [], []
    for img_np, p, win, s, K in jobs:
        img = torch.from_numpy(img_np).cuda()
        imgs.append(img)
        outs_static.append(ctx.outputs(img, p, s, K))
    torch.cuda.synchronize()
    # two calls in a row on one stream, sharing the static scratch
    for (img_np, p, win, s, K), img, (idx, dist) in zip(jobs, imgs, outs_static):
        H, W = img_np.shape
        dt = B.BM_U8 if img_np.dtype == np.uint8 else B.BM_F32
        rc = B.bm_match_static(img.data_ptr(), H, W, 1, dt, p, win, s, K, idx.data_ptr(),
                               dist.data_ptr(), st.cuda_stream)
        assert rc == B.BM_OK, B.bm_last_error()
    torch.cuda.synchronize()
    for (img_np, p, win, s, K), img, (idx, dist) in zip(jobs, imgs, outs_static):
        ridx, rdist = ctx.match(img, p, win, s, K)
        torch.cuda.synchronize()
        _agree(idx.cpu().numpy(), dist.cpu().numpy(), ridx.cpu().numpy(), rdist.cpu().numpy(),
               img_np.dtype == np.uint8)
    ctx.close()


@pytest.mark.gpu
def test_static_rejects_jobs_beyond_the_scratch():
    import torch

    H = W = 2048
    img = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    ry, rx = B.bm_num_refs(H, W, 8, 3)
    idx = torch.full((ry * rx, 16), 7, dtype=torch.int32, device="cuda")
    dist = torch.full((ry * rx, 16), 7.0, dtype=torch.float32, device="cuda")
    rc = B.bm_match_static(img.data_ptr(), H, W, 1, B.BM_F32, 8, 39, 3, 16, idx.data_ptr(),
                           dist.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == B.BM_ERR_TOO_LARGE
    assert "too large" in B.bm_last_error()
    torch.cuda.synchronize()
    assert bool((idx == 7).all()) and bool((dist == 7.0).all())


def test_direct_path_geometry_needs_only_the_header():
    # four channels at window 127 with K 128 are outside the tensor-core
    # kernel's tiling (even a quarter of the staged tile exceeds shared
    # memory): only the 256-byte header
    assert B.bm_static_scratch_bytes(160, 150, 4, B.BM_U8, 8, 127, 4, 128) == 256


@pytest.mark.gpu
def test_static_allocates_nothing_and_covers_direct_and_four_channels():
    """After a warm-up call, further calls leave free device memory unchanged.

    Covers a 4-channel uint8 job (tensor cores), a float32 job, a 4-channel
    float32 class that runs in column parts (part lists in the scratch, a
    merge launch) and a geometry that takes the direct kernel, each compared
    with bm_match.
    """
    import torch

    torch.cuda.set_device(0)
    assert B.bm_static_init() == B.BM_OK
    jobs = [
        (synth.rgbnir(200, 180, 20.0, 7101), 8, 39, 3, 32),            # u8, C 4
        (synth.gray(256, 240, 25.0, 7102, np.float32), 8, 39, 3, 16),  # f32, C 1
        (synth.rgbnir(160, 150, 20.0, 7103), 8, 127, 4, 128),            # direct kernel
        (np.stack([synth.gray(120, 110, 20.0, 7105 + c, np.float32) for c in range(4)], -1),
         8, 61, 3, 32),                                                  # f32, C 4, column parts
    ]
    assert B.bm_static_scratch_bytes(160, 150, 4, B.BM_U8, 8, 127, 4, 128) == 256
    assert B.bm_window_split(120, 110, 4, B.BM_F32, 8, 61, 3, 32) == 2
    ctx = B.Context(0)
    st = torch.cuda.current_stream()
    data = []
    for img_np, p, win, s, K in jobs:
        img = torch.from_numpy(np.ascontiguousarray(img_np)).cuda()
        idx, dist = ctx.outputs(img, p, s, K)
        data.append((img, idx, dist))
    torch.cuda.synchronize()
    # warm-up: loads every kernel module these calls use
    for (img_np, p, win, s, K), (img, idx, dist) in zip(jobs, data):
        assert _static(img, p, win, s, K, idx, dist, st) == B.BM_OK, B.bm_last_error()
    torch.cuda.synchronize()
    assert B.bm_static_check(st.cuda_stream) == B.BM_OK
    free0, _ = torch.cuda.mem_get_info()
    for (img_np, p, win, s, K), (img, idx, dist) in zip(jobs, data):
        assert _static(img, p, win, s, K, idx, dist, st) == B.BM_OK, B.bm_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert B.bm_static_check(st.cuda_stream) == B.BM_OK
    for (img_np, p, win, s, K), (img, idx, dist) in zip(jobs, data):
        ridx, rdist = ctx.match(img, p, win, s, K)
        torch.cuda.synchronize()
        _agree(idx.cpu().numpy(), dist.cpu().numpy(), ridx.cpu().numpy(), rdist.cpu().numpy(),
               img_np.dtype == np.uint8)
    ctx.close()


@pytest.mark.gpu
def test_static_timeout_is_reported_by_static_check():
    """A bounded wait that runs out inside bm_match_static is not silent.

    The test hook withholds one stage publication of the next call's
    tensor-core kernel; its wait runs out (a bounded wait, no GPU fault), the
    kernel records the site in the sticky static fault word, and
    bm_static_check returns BM_ERR_TIMEOUT once, then BM_OK.  The next call
    gives the right result.
    """
    import torch

    from oracle import oracle as O

    torch.cuda.set_device(0)
    img_np = synth.gray(64, 64, 25.0, 7104, np.uint8)
    img = torch.from_numpy(img_np).cuda()
    ry, rx = B.bm_num_refs(64, 64, 8, 1)
    idx = torch.empty((ry * rx, 16), dtype=torch.int32, device="cuda")
    dist = torch.empty((ry * rx, 16), dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    assert B.bm_static_check(st.cuda_stream) == B.BM_OK
    assert B.bm_static_set_fault_injection(7) == B.BM_ERR_INVALID
    assert B.bm_static_set_fault_injection(1) == B.BM_OK
    assert _static(img, 8, 21, 1, 16, idx, dist, st) == B.BM_OK
    rc = B.bm_static_check(st.cuda_stream)
    assert rc == B.BM_ERR_TIMEOUT, rc
    assert "ran out" in B.bm_last_error()
    assert B.bm_static_check(st.cuda_stream) == B.BM_OK
    assert _static(img, 8, 21, 1, 16, idx, dist, st) == B.BM_OK
    assert B.bm_static_check(st.cuda_stream) == B.BM_OK
    oi, od = O.match(img_np, 8, 21, 1, 16)
    assert np.array_equal(idx.cpu().numpy(), oi)
    assert np.array_equal(dist.cpu().numpy().astype(np.int64), od)
