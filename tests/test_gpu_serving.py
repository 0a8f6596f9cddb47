"""Serving (continuous batching), batch-graph replays and the autotuner.

Serving: requests submitted while others are on the GPU are admitted in
batches as memory and stream slots free up; every result must be the same
as the same request matched alone (and, sampled, the same as the oracle).
"""
import time

import numpy as np
import pytest

from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth
from parity import compare, sample_refs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _image(H, W, C, dt, seed):
    if C == 1:
        return synth.gray(H, W, 20.0, seed, np.uint8 if dt == "u8" else np.float32)
    planes = [synth.gray(H, W, 20.0, seed * 10 + c, np.uint8 if dt == "u8" else np.float32)
              for c in range(C)]
    return np.ascontiguousarray(np.stack(planes, axis=-1))


def _mixed_requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        dt = "u8" if rng.integers(0, 2) == 0 else "f32"
        C = int(rng.choice([1, 4]))
        H, W = int(rng.integers(48, 160)), int(rng.integers(48, 160))
        p = int(rng.choice([7, 8]))
        win = int(rng.choice([15, 21, 39]))
        s = 3 if p == 8 else 4
        K = int(rng.choice([8, 16, 32]))
        out.append((_image(H, W, C, dt, 5000 + i), p, win, s, K))
    return out


def _poll_all(ctx, tickets, timeout_s=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for t in tickets:
            if t in done:
                continue
            d, st = ctx.poll(t)
            if d:
                done[t] = st
        assert time.time() - t0 < timeout_s, "serving did not finish"
        time.sleep(0.0005)
    return done


def test_mixed_stream_equals_each_request_alone():
    ctx = B.Context(0)
    reqs = _mixed_requests(24, 77)
    bufs, tickets = [], []
    for img, p, win, s, K in reqs:
        t = torch.from_numpy(img).cuda()
        idx, dist = ctx.outputs(t, p, s, K)
        bufs.append((t, idx, dist))
    torch.cuda.synchronize()
    for (img, p, win, s, K), (t, idx, dist) in zip(reqs, bufs):
        tickets.append(ctx.submit(ctx.request(t, p, win, s, K, idx, dist)))
    status = _poll_all(ctx, tickets)
    assert all(v == B.BM_OK for v in status.values())
    for (img, p, win, s, K), (t, idx, dist) in zip(reqs, bufs):
        a_idx, a_dist = ctx.match(t, p, win, s, K)  # the same request alone
        torch.cuda.synchronize()
        assert np.array_equal(idx.cpu().numpy(), a_idx.cpu().numpy())
        assert np.array_equal(dist.cpu().numpy(), a_dist.cpu().numpy())
    # and the mix against the oracle on a sample of references
    for i in (0, 5, 11):
        img, p, win, s, K = reqs[i]
        ry, rx = B.bm_num_refs(img.shape[0], img.shape[1], p, s)
        refs = sample_refs(ry, rx, 40, 900 + i)
        compare(img, p, win, s, K, bufs[i][1].cpu().numpy(), bufs[i][2].cpu().numpy(), refs=refs)
    ctx.close()


def test_budget_admission_and_errors():
    img = _image(96, 96, 1, "f32", 11)
    t = torch.from_numpy(img).cuda()
    # a budget that holds about two of these jobs at a time
    probe = B.Context(0)
    need = B.bm_workspace_bytes(96, 96, 1, B.BM_F32, 8, 39, 3, 16)
    probe.close()
    ctx = B.Context(0, mem_budget_bytes=int(2.5 * need))
    outs = [ctx.outputs(t, 8, 3, 16) for _ in range(6)]
    tickets = [ctx.submit(ctx.request(t, 8, 39, 3, 16, o[0], o[1])) for o in outs]
    status = _poll_all(ctx, tickets)
    assert all(v == B.BM_OK for v in status.values())
    ref_idx, ref_dist = ctx.match(t, 8, 39, 3, 16)
    torch.cuda.synchronize()
    for o in outs:
        assert np.array_equal(o[0].cpu().numpy(), ref_idx.cpu().numpy())
    # a request larger than the whole budget is refused; unknown tickets are reported
    big = _image(400, 400, 1, "f32", 12)
    tb = torch.from_numpy(big).cuda()
    bi, bd = ctx.outputs(tb, 8, 3, 16)
    with pytest.raises(B.BMError) as e:
        ctx.submit(ctx.request(tb, 8, 39, 3, 16, bi, bd))
    assert e.value.code == B.BM_ERR_BUSY
    with pytest.raises(B.BMError) as e:
        ctx.poll(123456789)
    assert e.value.code == B.BM_ERR_NOT_FOUND
    ctx.close()


def test_batch_graph_replay_reads_current_inputs():
    ctx = B.Context(0)
    st = torch.cuda.Stream()
    imgs = [torch.from_numpy(_image(80, 90, 1, "f32", 31 + i)).cuda() for i in range(3)]
    outs = [ctx.outputs(t, 8, 3, 16) for t in imgs]
    reqs = [ctx.request(t, 8, 39, 3, 16, o[0], o[1]) for t, o in zip(imgs, outs)]
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        ctx.match_batch(reqs, stream=st)  # captured
        ctx.match_batch(reqs, stream=st)  # replayed
    st.synchronize()
    first = [o[0].cpu().numpy().copy() for o in outs]
    # new pixels in the same buffers: the replay must see them
    new = [_image(80, 90, 1, "f32", 61 + i) for i in range(3)]
    for t, a in zip(imgs, new):
        t.copy_(torch.from_numpy(a))
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        ctx.match_batch(reqs, stream=st)
    st.synchronize()
    for i, (a, o) in enumerate(zip(new, outs)):
        single_idx, single_dist = ctx.match(imgs[i], 8, 39, 3, 16)
        torch.cuda.synchronize()
        assert np.array_equal(o[0].cpu().numpy(), single_idx.cpu().numpy())
        assert np.array_equal(o[1].cpu().numpy(), single_dist.cpu().numpy())
        assert not np.array_equal(o[0].cpu().numpy(), first[i])
        ry, rx = B.bm_num_refs(80, 90, 8, 3)
        compare(a, 8, 39, 3, 16, o[0].cpu().numpy(), o[1].cpu().numpy(),
                refs=sample_refs(ry, rx, 30, 70 + i))
    ctx.close()


@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_autotuner_picks_a_configuration_with_identical_results(tmp_path, dt):
    cache = str(tmp_path / "tune.txt")
    img = _image(128, 120, 1, dt, 41)
    t = torch.from_numpy(img).cuda()
    plain = B.Context(0)
    p_idx, p_dist = plain.match(t, 8, 39, 3, 16)
    torch.cuda.synchronize()
    tuned = B.Context(0, tune_cache=cache)
    t_idx, t_dist = tuned.match(t, 8, 39, 3, 16)  # tunes the class, then matches
    torch.cuda.synchronize()
    assert np.array_equal(p_idx.cpu().numpy(), t_idx.cpu().numpy())
    assert np.array_equal(p_dist.cpu().numpy(), t_dist.cpu().numpy())
    lines = open(cache).read().split("\n")
    assert any(line.startswith("tc2_dtype") for line in lines)
    # a second context reads the table instead of tuning again
    again = B.Context(0, tune_cache=cache)
    a_idx, a_dist = again.match(t, 8, 39, 3, 16)
    torch.cuda.synchronize()
    assert np.array_equal(p_idx.cpu().numpy(), a_idx.cpu().numpy())
    for c in (plain, tuned, again):
        c.close()


def test_mixed_class_batch_graph_replay():
    """Several classes in one bm_match_batch (one of them on the direct
    kernel): their launches run on parallel branches of one captured graph.
    Replays with new pixels give what each job gives alone."""
    ctx = B.Context(0)
    st = torch.cuda.Stream()
    specs = [(100, 90, 1, "f32", 8, 39, 3, 16), (64, 64, 1, "u8", 8, 21, 1, 16),
             (80, 72, 4, "u8", 8, 39, 3, 32), (150, 133, 1, "f32", 7, 61, 4, 70),
             (96, 96, 1, "u8", 7, 39, 4, 32),
             (90, 84, 4, "f32", 8, 127, 3, 128)]  # a direct-kernel class: its own branch
    imgs, outs, reqs = [], [], []
    for i, (H, W, C, dt, p, win, s, K) in enumerate(specs):
        t = torch.from_numpy(_image(H, W, C, dt, 300 + i)).cuda()
        o = ctx.outputs(t, p, s, K)
        imgs.append(t)
        outs.append(o)
        reqs.append(ctx.request(t, p, win, s, K, o[0], o[1]))
    assert B.bm_workspace_bytes(90, 84, 4, B.BM_F32, 8, 127, 3, 128) == 0  # direct kernel
    torch.cuda.synchronize()
    for rnd in range(2):
        if rnd == 1:
            for i, (t, (H, W, C, dt, p, win, s, K)) in enumerate(zip(imgs, specs)):
                t.copy_(torch.from_numpy(_image(H, W, C, dt, 400 + i)))
            torch.cuda.synchronize()
        with torch.cuda.stream(st):
            ctx.match_batch(reqs, stream=st)  # first call captures, then replays
            ctx.match_batch(reqs, stream=st)
        st.synchronize()
        for (H, W, C, dt, p, win, s, K), t, o in zip(specs, imgs, outs):
            a_idx, a_dist = ctx.match(t, p, win, s, K)
            torch.cuda.synchronize()
            assert torch.equal(a_idx, o[0]) and torch.equal(a_dist, o[1])
    ctx.close()


def test_autotuner_window_split_choice_is_exact(tmp_path):
    """The tuner's choices include the window split (1, 2 or 4 parts); a job
    that splits alone gets a recorded pick whose results equal the
    heuristic's, for uint8 (exact) and float32 (pool re-ranked)."""
    cache = str(tmp_path / "tune.txt")
    for dt in ("u8", "f32"):
        img = _image(96, 90, 1, dt, 45)
        code = B.BM_U8 if dt == "u8" else B.BM_F32
        assert B.bm_window_split(96, 90, 1, code, 8, 39, 3, 16) > 1
        t = torch.from_numpy(img).cuda()
        plain = B.Context(0)
        p_idx, p_dist = plain.match(t, 8, 39, 3, 16)
        tuned = B.Context(0, tune_cache=cache)
        t_idx, t_dist = tuned.match(t, 8, 39, 3, 16)
        torch.cuda.synchronize()
        assert torch.equal(p_idx, t_idx) and torch.equal(p_dist, t_dist)
        for c in (plain, tuned):
            c.close()
    picks = [ln.split() for ln in open(cache).read().split("\n") if ln.strip()]
    assert len(picks) == 2 and all(int(p[1]) >= -1 for p in picks)
