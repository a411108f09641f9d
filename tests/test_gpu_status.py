"""Asynchronous device errors, made on purpose with a wait that runs out.

The level-0 look-back scan waits, with a bound, for the running total of the
tile before it.  The test hook ls_debug_set_wait keeps the first tile from
ever publishing its total (a flag that nothing sets) and shortens the bound to
a few thousand polls, so the waits of the following tiles give up: the call
records LS_ERR_TIMEOUT in its own status block, its later kernels do nothing
(the keys are left unspecified, every access in bounds), and the error reaches
the stream's status word and no other.  Nothing here faults or traps the GPU.
"""
import numpy as np
import pytest

import lsgen
import oracle

torch = pytest.importorskip("torch")
import paper_2107_03290_gb300 as ls  # noqa: E402

pytestmark = pytest.mark.gpu

LS_OK, LS_ERR_TIMEOUT = 0, 4
SHORT = 1 << 12   # polls before a wait gives up (a few milliseconds)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ls.build()
    ls.load()
    torch.cuda.init()
    yield


def _same(got: torch.Tensor, keys: np.ndarray) -> bool:
    want = oracle.reference_sort(keys)
    return np.array_equal(got.cpu().numpy().view(np.uint8), want.view(np.uint8))


def test_stalled_scan_times_out_on_its_stream_only():
    keys = lsgen.normal_f64(300_000, 1)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    t1 = torch.from_numpy(keys.copy()).cuda()
    t2 = torch.from_numpy(keys.copy()).cuda()
    torch.cuda.synchronize()
    ls.debug_set_wait(stall=1, spin_limit=SHORT, stream=s1)
    try:
        ls.sort_(t1, stream=s1)     # its level-0 waits run out
        ls.sort_(t2, stream=s2)     # concurrent call on another stream
        assert ls.stream_status(s1) == LS_ERR_TIMEOUT
        assert ls.stream_status(s2) == LS_OK
        assert ls.stream_status(s1) == LS_OK   # read and cleared
    finally:
        ls.debug_set_wait(0, 0, stream=s1)
    assert _same(t2, keys)
    # the next call on the failed stream is clean and correct
    t1.copy_(torch.from_numpy(keys))
    torch.cuda.synchronize()
    ls.sort_(t1, stream=s1)
    assert ls.stream_status(s1) == LS_OK
    assert _same(t1, keys)


def test_unread_error_does_not_stop_later_calls():
    """Every call clears its own block: an error left unread on a stream is
    still reported, but the calls after it sort correctly."""
    keys = lsgen.zipf_lognormal_f64(200_000, 3, k=2000)
    s = torch.cuda.Stream()
    t = torch.from_numpy(keys.copy()).cuda()
    ls.debug_set_wait(stall=1, spin_limit=SHORT, stream=s)
    ls.sort_(t, stream=s)
    ls.debug_set_wait(0, 0, stream=s)
    s.synchronize()
    t.copy_(torch.from_numpy(keys))
    torch.cuda.synchronize()
    ls.sort_(t, stream=s)
    s.synchronize()
    assert _same(t, keys)
    assert ls.stream_status(s) == LS_ERR_TIMEOUT   # the first call's error
    assert ls.stream_status(s) == LS_OK


def test_server_request_times_out_alone():
    """A large request (full learned sort) whose waits run out fails with
    LS_ERR_TIMEOUT; batched requests in flight with it, and later requests,
    finish LS_OK with the right result."""
    big = lsgen.exponential_f32((1 << 24) + 4097, 5)
    small = [lsgen.normal_f64(50_000, 9), lsgen.uniform_u64(70_000, 2)]
    srv = ls.Server(hbm_budget_bytes=8 << 30, max_inflight=8, streams=3, debug_stall=1,
                    debug_spin_limit=SHORT)
    try:
        tb = torch.from_numpy(big.copy()).cuda()
        ts = [torch.from_numpy(a.copy()).cuda() for a in small]
        torch.cuda.synchronize()
        kb = srv.submit(tb)
        ks = [srv.submit(t) for t in ts]
        assert srv.wait(kb, check=False)["status"] == LS_ERR_TIMEOUT
        for k, t, a in zip(ks, ts, small):
            assert srv.wait(k, check=False)["status"] == LS_OK
            assert _same(t, a)
    finally:
        srv.close()
    srv = ls.Server(hbm_budget_bytes=8 << 30, max_inflight=8, streams=3)
    try:
        tb.copy_(torch.from_numpy(big))
        torch.cuda.synchronize()
        assert srv.wait(srv.submit(tb), check=False)["status"] == LS_OK
        assert _same(tb, big)
    finally:
        srv.close()
