"""GPU parity of non-local means (bm_nlm, through the C ABI) against the numpy
oracle (oracle/nlm.py, float64).

Tolerance, from the float32 arithmetic of the kernel: a distance of n = p*p*C
squared differences has relative error <= (n + 3) 2^-24; the weight
w = exp(-d/b^2) then has relative error <= (d/b^2)(n + 3) 2^-24 + 2^-22, and
sum_j w_j (d_j/b^2) / Theta stays below ln(#candidates) (about 7.3 for a 39^2
window), so the weights are off by at most ~3e-5 of Theta; with the float32
accumulation (candidates per lane + 5 butterfly levels) every estimate is
within ~3.4e-5 of the data range of the exact value and Theta within ~3.5e-5
relative.  Tested: 5e-5 of max|X| for the estimates, 5e-5 relative for Theta.
"""
import numpy as np
import pytest

from oracle import nlm as N
from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth
from parity import sample_refs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 5e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.Context(0)
    yield c
    c.close()


def make_image(H, W, C, dt, seed, sigma=25.0):
    npdt = np.uint8 if dt == "u8" else np.float32
    if C == 1:
        return synth.gray(H, W, sigma, seed, npdt)
    return np.ascontiguousarray(np.stack([synth.gray(H, W, sigma, seed * 10 + c, npdt)
                                          for c in range(C)], axis=-1))


def check(ctx, img, p, win, s, b, refs=None):
    t = torch.from_numpy(img).cuda()
    est, theta = ctx.nlm(t, p, win, s, b)
    torch.cuda.synchronize()
    est, theta = est.cpu().numpy().astype(np.float64), theta.cpu().numpy().astype(np.float64)
    o_est, o_theta, _ = N.nlm(img, p, win, s, b, refs=refs)
    if refs is not None:
        est, theta = est[refs], theta[refs]
    scale = float(np.abs(img.astype(np.float64)).max())
    err = np.abs(est - o_est)
    assert np.all(err <= TOL * scale), f"max err {err.max():.3e} vs {TOL * scale:.3e}"
    rel = np.abs(theta - o_theta) / o_theta
    assert np.all(rel <= TOL), f"max Theta rel err {rel.max():.3e}"
    assert np.all(theta >= 1.0 - 1e-6)


CASES = [
    # name,        H,   W,  C, dtype, p, win, s, b
    ("f32_p8",     70,  66, 1, "f32", 8, 39, 3, 283.0),
    ("u8_p8",      64,  64, 1, "u8",  8, 21, 1, 283.0),
    ("f32_p7",     60,  57, 1, "f32", 7, 61, 4, 250.0),
    ("f32_p5_sm",  40,  45, 1, "f32", 5, 9,  2, 60.0),
    ("u8_c4_p4",   48,  40, 4, "u8",  4, 15, 3, 200.0),
    ("f32_c3_p3",  37,  41, 3, "f32", 3, 7,  1, 90.0),
    ("f32_p1",     20,  30, 1, "f32", 1, 5,  1, 20.0),
    ("u8_c2_p5",   33,  29, 2, "u8",  5, 11, 2, 150.0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_small_full_parity(ctx, case):
    name, H, W, C, dt, p, win, s, b = case
    check(ctx, make_image(H, W, C, dt, seed=H * 7 + W + C), p, win, s, b)


def test_full_size_sampled_parity(ctx):
    img = make_image(512, 512, 1, "f32", seed=2000)
    ny, nx = B.bm_num_refs(512, 512, 8, 3)
    check(ctx, img, 8, 39, 3, 283.0, refs=sample_refs(ny, nx, 300, 2000))


def test_window_one_returns_the_reference():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with B.Context(0) as c:
        img = make_image(30, 28, 1, "f32", seed=3)
        est, theta = c.nlm(torch.from_numpy(img).cuda(), 6, 1, 4, 50.0)
        torch.cuda.synchronize()
        est, theta = est.cpu().numpy(), theta.cpu().numpy()
        nx = (28 - 6) // 4 + 1
        for r in range(est.shape[0]):
            y, x = (r // nx) * 4, (r % nx) * 4
            assert np.array_equal(est[r], img[y:y + 6, x:x + 6].reshape(-1))
        assert np.all(theta == 1.0)


def test_invalid_and_unsupported(ctx):
    img = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    out = torch.full((1000,), -7.0, device="cuda")
    h = ctx.handle
    for b in (0.0, -1.0, float("inf"), float("nan")):
        rc = B.bm_nlm(h, img.data_ptr(), 32, 32, 1, B.BM_F32, 4, 5, 2, b, out.data_ptr(), None, None)
        assert rc == B.BM_ERR_INVALID
    rc = B.bm_nlm(h, img.data_ptr(), 32, 32, 1, B.BM_F32, 4, 4, 2, 10.0, out.data_ptr(), None, None)
    assert rc == B.BM_ERR_INVALID  # even window
    img4 = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
    rc = B.bm_nlm(h, img4.data_ptr(), 32, 32, 4, B.BM_F32, 5, 5, 2, 10.0, out.data_ptr(), None, None)
    assert rc == B.BM_ERR_UNSUPPORTED  # 5 * 5 * 4 > 64
    torch.cuda.synchronize()
    assert bool((out == -7.0).all())
