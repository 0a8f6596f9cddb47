"""Host-side choice of the float32 pool size L (the candidates per reference
the tensor-core pass keeps for the boundary re-rank), read back through the
ABI's workspace query (no GPU): the workspace holds two [refs][L] pool arrays,
so L follows from bm_workspace_bytes and the workspace layout.

The rule: L = K + 8 rounded up to 8 by default; four or eight channels keep
K + 16 (K <= 40) or K + 24; one channel at windows of 45 or more keeps K + 16
for K <= 24 and for K > 40 -- each only when the larger pool leaves the
tensor-core geometry no worse (the config-3 class keeps K + 8).

Also host-only: every class of the serving mix has a tensor-core geometry
(column parts where the staged tile does not fit whole), and the static
entry point's scratch carries the same part lists as a context workspace.
"""
import pytest

from paper_2006_13714_gb300 import bm as B


def _ru(v, m):
    return (v + m - 1) // m * m


def _a256(v):
    return _ru(v, 256)


def _pool_from_workspace(H, W, C, p, win, s, K):
    """Solve the workspace layout for L (float32 jobs on the tensor-core path)."""
    Cp = 1 if C == 1 else 2 if C == 2 else 4 if C <= 4 else 8
    pw = (p * Cp + 7) // 8
    if pw > 1 and pw % 2:
        pw += 1
    p_eff = _ru(p, 2) if pw == 1 else p
    pitch = _ru(W * Cp + 8 * pw + 16, 8)
    plane = (H + p_eff + 8) * pitch * 2
    Hc, Wc = H - p + 1, W - p + 1
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    nR = ny * nx
    fixed = 2 * _a256(plane) + _a256(Hc * Wc * 4) + _a256(Hc * Wc * 16) + 256
    ws = B.bm_workspace_bytes(H, W, C, B.BM_F32, p, win, s, K)
    split = B.bm_window_split(H, W, C, B.BM_F32, p, win, s, K)
    assert ws > 0
    for L in range(8, 161, 8):
        total = fixed + 2 * _a256(nR * L * 4) + (2 * _a256(split * nR * L * 4) if split > 1 else 0)
        if total == ws:
            return L
    raise AssertionError(f"no pool size matches workspace {ws}")


@pytest.mark.parametrize("shape,K,expected", [
    ((512, 512, 1, 8, 39, 3), 16, 24),    # the 512^2 window-39 batch: K + 8
    ((512, 512, 1, 8, 61, 3), 16, 32),    # one channel, window 61, K <= 24: 32
    ((512, 512, 1, 8, 61, 3), 32, 40),    # one channel, 24 < K <= 40: K + 8
    ((512, 512, 1, 8, 61, 3), 70, 88),    # one channel, window 61, K > 40: K + 16
    ((512, 512, 1, 7, 61, 4), 70, 80),    # config-3 class: the larger pool's geometry is worse
    ((512, 512, 1, 8, 39, 3), 70, 80),    # window 39, one channel: K + 8
    ((512, 512, 4, 8, 61, 3), 70, 96),    # four channels, K > 40: K + 24
    ((512, 512, 4, 8, 39, 3), 32, 48),    # four channels, K <= 40: K + 16
    ((512, 512, 4, 8, 61, 3), 16, 32),    # four channels, K 16: 32
])
def test_pool_size_rule(shape, K, expected):
    H, W, C, p, win, s = shape
    assert _pool_from_workspace(H, W, C, p, win, s, K) == expected


def test_uint8_jobs_have_no_pool():
    # uint8 ranks exactly on the tensor cores: no pool, a smaller workspace
    a = B.bm_workspace_bytes(512, 512, 1, B.BM_U8, 8, 39, 3, 16)
    b = B.bm_workspace_bytes(512, 512, 1, B.BM_F32, 8, 39, 3, 16)
    assert 0 < a < b


def test_every_serving_class_runs_on_tensor_cores():
    """Every class of the serving mix (uint8 / float32, one or four channels,
    patch 8 at stride 3 or 7 at stride 4, window 39 or 61, K 16 / 32 / 70)
    has a tensor-core geometry (a workspace; the direct kernel needs none),
    at the mix's smallest and largest sides and an uneven one."""
    for dt in (B.BM_U8, B.BM_F32):
        for C in (1, 4):
            for p, s in ((8, 3), (7, 4)):
                for win in (39, 61):
                    for K in (16, 32, 70):
                        for H, W in ((128, 128), (2048, 2048), (1000, 333)):
                            assert B.bm_workspace_bytes(H, W, C, dt, p, win, s, K) > 0, (dt, C, p, win, K, H, W)
                            assert 1 <= B.bm_window_split(H, W, C, dt, p, win, s, K) <= 4


def test_column_part_lists_in_static_scratch():
    # a column-part class's static scratch holds its part lists on top of the pool
    parts = B.bm_window_split(512, 512, 4, B.BM_F32, 8, 61, 3, 32)
    assert parts == 2
    ws = B.bm_workspace_bytes(512, 512, 4, B.BM_F32, 8, 61, 3, 32)
    st = B.bm_static_scratch_bytes(512, 512, 4, B.BM_F32, 8, 61, 3, 32)
    # both layouts carry the same operand, norm, pool and part-list arrays
    assert abs(ws - st) <= 512
