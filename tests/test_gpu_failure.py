"""Failure detection on the GPU without a GPU fault.

The tensor-core kernel's waits are bounded; a test hook makes one CTA's
producer withhold a stage publication, so the MMA warp's wait runs out after
its limit.  The CTA then takes its abort path (drains its copies and MMAs,
frees its tensor memory, records the wait site), the kernel ends, and the
host reports BM_ERR_TIMEOUT through bm_check.  The context must stay usable:
the next call returns correct results and a clean check.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2006_13714_gb300 import bm as B
from paper_2006_13714_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    img = synth.gray(64, 64, 25.0, 321, np.uint8)
    t = torch.from_numpy(img).cuda()
    with B.Context(0) as ctx:
        st = torch.cuda.current_stream()
        assert B.bm_check(ctx.handle, st.cuda_stream) == B.BM_OK
        assert B.bm_set_fault_injection(ctx.handle, 1) == B.BM_OK
        ctx.match(t, 8, 21, 1, 16)
        rc = B.bm_check(ctx.handle, st.cuda_stream)
        assert rc == B.BM_ERR_TIMEOUT, rc
        # the first wait to run out is the MMA warp's (stage filled) or the
        # epilogue's (accumulator filled): both wait on the withheld stage
        msg = B.bm_last_error(ctx.handle)
        assert "ran out" in msg and ("stage filled" in msg or "accumulator filled" in msg), msg
        # the word was cleared and the context still works
        assert B.bm_check(ctx.handle, st.cuda_stream) == B.BM_OK
        idx, dist = ctx.match(t, 8, 21, 1, 16)
        assert B.bm_check(ctx.handle, st.cuda_stream) == B.BM_OK
        oi, od = O.match(img, 8, 21, 1, 16)
        assert np.array_equal(idx.cpu().numpy(), oi)
        assert np.array_equal(dist.cpu().numpy().astype(np.int64), od)


def test_invalid_injection_mode():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with B.Context(0) as ctx:
        assert B.bm_set_fault_injection(ctx.handle, 7) == B.BM_ERR_INVALID
        assert B.bm_check(None, None) == B.BM_ERR_INVALID


def _wait_done(ctx, ticket, limit_s=60.0):
    import time
    t0 = time.time()
    while True:
        done, status = ctx.poll(ticket)
        if done:
            return status
        assert time.time() - t0 < limit_s, "served request did not finish"
        time.sleep(0.002)


def test_served_request_reports_timeout():
    """A served request whose kernel ran out of a bounded wait is not BM_OK.

    The serving thread copies every job's error word to the host after the
    batch and fails the ticket with BM_ERR_TIMEOUT; the poll that reports it
    sets the polling thread's bm_last_error to the wait site.  The next
    request on the same context is served correctly.
    """
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    img = synth.gray(64, 64, 25.0, 322, np.uint8)
    t = torch.from_numpy(img).cuda()
    with B.Context(0) as ctx:
        idx, dist = ctx.outputs(t, 8, 1, 16)
        torch.cuda.synchronize()
        assert B.bm_set_fault_injection(ctx.handle, 1) == B.BM_OK
        tk = ctx.submit(B.Context.request(t, 8, 21, 1, 16, idx, dist))
        status = _wait_done(ctx, tk)
        assert status == B.BM_ERR_TIMEOUT, status
        msg = B.bm_last_error(ctx.handle)
        assert "ran out" in msg, msg
        # the context-wide sticky word saw it too; bm_check clears it
        st = torch.cuda.current_stream()
        assert B.bm_check(ctx.handle, st.cuda_stream) == B.BM_ERR_TIMEOUT
        assert B.bm_check(ctx.handle, st.cuda_stream) == B.BM_OK
        idx2, dist2 = ctx.outputs(t, 8, 1, 16)
        torch.cuda.synchronize()
        tk2 = ctx.submit(B.Context.request(t, 8, 21, 1, 16, idx2, dist2))
        assert _wait_done(ctx, tk2) == B.BM_OK
        oi, od = O.match(img, 8, 21, 1, 16)
        assert np.array_equal(idx2.cpu().numpy(), oi)
        assert np.array_equal(dist2.cpu().numpy().astype(np.int64), od)
