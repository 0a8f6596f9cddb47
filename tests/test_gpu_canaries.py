"""Canary words around every output buffer (compute-sanitizer is not available
on this pool): each entry point writes its outputs into the middle of a
larger buffer whose margins hold a known pattern, and the margins must be
intact afterwards -- no kernel writes outside its output."""
import numpy as np
import pytest

from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 4096          # elements on each side
CANARY_I = -123456789
CANARY_F = -1.2345e30


def guarded(shape, dtype):
    n = int(np.prod(shape))
    fill = CANARY_I if dtype in (torch.int32, torch.uint8) else CANARY_F
    if dtype == torch.uint8:
        fill = 0xA5
    buf = torch.full((n + 2 * MARGIN,), fill, dtype=dtype, device="cuda")
    return buf, buf[MARGIN:MARGIN + n].view(*shape)


def intact(buf):
    torch.cuda.synchronize()
    head, tail = buf[:MARGIN], buf[-MARGIN:]
    fill = head[0].item()
    return bool((head == fill).all()) and bool((tail == fill).all())


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_match_and_direct_outputs_stay_in_bounds(ctx, dt):
    H, W, p, win, s, K = 90, 77, 8, 39, 3, 16
    img = torch.from_numpy(synth.gray(H, W, 25.0, 5, np.uint8 if dt == "u8" else np.float32)).cuda()
    ny, nx = B.bm_num_refs(H, W, p, s)
    for fn in (ctx.match, ctx.match_direct):
        bi, idx = guarded((ny * nx, K), torch.int32)
        bd, dist = guarded((ny * nx, K), torch.int32 if dt == "u8" else torch.float32)
        fn(img, p, win, s, K, out=(idx, dist))
        assert intact(bi) and intact(bd)
        assert bool((idx >= -1).all())


def test_extension_outputs_stay_in_bounds(ctx):
    H, W, p, win, s, K = 70, 66, 8, 39, 3, 16
    img = torch.from_numpy(synth.gray(H, W, 25.0, 6, np.float32)).cuda()
    ny, nx = B.bm_num_refs(H, W, p, s)
    idx, _ = ctx.match(img, p, win, s, K)
    bg, groups = guarded((ny * nx, K, p * p), torch.float32)
    ctx.gather_groups(img, p, idx, ny, nx, out=groups)
    assert intact(bg)
    bo, out = guarded((H, W, 1), torch.float32)
    bw, wmap = guarded((H, W), torch.float32)
    ctx.aggregate(groups, idx, H, W, 1, p, ny, nx, out=(out, wmap))
    assert intact(bo) and intact(bw)
    be, est = guarded((ny * nx, p * p), torch.float32)
    bt, theta = guarded((ny * nx,), torch.float32)
    ctx.nlm(img, p, win, s, 283.0, out=(est, theta))
    assert intact(be) and intact(bt)
    bi, nidx = guarded((ny * nx, K), torch.int32)
    bs, nsc = guarded((ny * nx, K), torch.float32)
    ctx.match_ncc(img, p, win, s, K, out=(nidx, nsc))
    assert intact(bi) and intact(bs)
    img4 = torch.from_numpy(synth.rgbnir(48, 44, 20.0, 7)).cuda()
    ny4, nx4 = B.bm_num_refs(48, 44, 8, 3)
    b3i, i3 = guarded((ny4 * nx4 * 3, 16), torch.int32)
    b3d, d3 = guarded((ny4 * nx4 * 3, 16), torch.int32)
    ctx.match_3d(img4, 8, 2, 15, 3, 16, out=(i3, d3))
    assert intact(b3i) and intact(b3d)
