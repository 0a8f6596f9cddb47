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
