"""Inputs past 2^32 keys (the largest single arrays the planner accepts on this
GPU's memory): every position, count and offset that could wrap at 32 bits is
exercised.  The oracle cannot sort these on the host in seconds, so the checks
are properties that hold at any size: the output is non-decreasing and holds
the same multiset (exact per-chunk sums of the values and a histogram of the
top byte, before and after)."""
import numpy as np
import pytest
import torch

import paper_2107_03290_gb300 as ls  # noqa: E402

pytestmark = pytest.mark.gpu

CH = 1 << 28  # keys per checking chunk


def _u32_as_i64(x):
    return x.view(torch.int32).to(torch.int64) & 0xFFFFFFFF


def _signature(t):
    """Exact sum and top-byte histogram of uint32 keys, chunk by chunk."""
    s = 0
    h = torch.zeros(256, dtype=torch.int64, device=t.device)
    for a in range(0, t.numel(), CH):
        v = _u32_as_i64(t[a:a + CH])
        s += int(v.sum().item())
        h += torch.bincount(v >> 24, minlength=256)
    return s, h.cpu().numpy()


def _non_decreasing(t):
    prev = None
    for a in range(0, t.numel(), CH):
        v = _u32_as_i64(t[a:a + CH])
        if not bool(torch.all(v[1:] >= v[:-1]).item()):
            return False
        if prev is not None and int(v[0].item()) < prev:
            return False
        prev = int(v[-1].item())
    return True


def test_sort_u32_past_2_32_keys():
    """Uniform keys, then 1000 distinct values (equality slots and fills carry
    most keys), in one buffer so that the second sort reuses the workspace."""
    n = (1 << 32) + 12_345
    free, _ = torch.cuda.mem_get_info()
    if free < 120 << 30:  # keys 17 GB, workspace (scratch, ids, job lists) about 70 GB
        pytest.skip("needs about 120 GB of free device memory")
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    t = torch.empty(n, dtype=torch.int32, device="cuda")
    u = t.view(torch.uint32)
    for dist in ("uniform", "duplicates"):
        for a in range(0, n, CH):
            m = min(CH, n - a)
            if dist == "uniform":
                t[a:a + m] = torch.randint(-2**31, 2**31 - 1, (m,), dtype=torch.int32,
                                           device="cuda", generator=g)
            else:
                t[a:a + m] = torch.randint(0, 1000, (m,), dtype=torch.int32, device="cuda",
                                           generator=g) * 4_000_000
        before = _signature(u)
        ls.sort_(u)
        torch.cuda.synchronize()
        assert ls.stream_status() == 0, dist
        assert _non_decreasing(u), dist
        after = _signature(u)
        assert before[0] == after[0], dist
        assert np.array_equal(before[1], after[1]), dist


def test_sort_f64_past_2_32_keys_zipf():
    """2^32 + 12,345 f64 keys drawn with Zipf(1.1) weights from 100,000
    lognormal values: the heavy-value table, compaction into scratch and the
    sample sort of the 43M-key training sample at full scale."""
    n = (1 << 32) + 12_345
    free, _ = torch.cuda.mem_get_info()
    if free < 160 << 30:  # keys 34 GB, workspace about 80 GB
        pytest.skip("needs about 160 GB of free device memory")
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    k = 100_000
    vals = torch.exp(2.0 * torch.randn(k, dtype=torch.float64, device="cuda", generator=g))
    w = torch.arange(1, k + 1, dtype=torch.float64, device="cuda") ** -1.1
    cdf = torch.cumsum(w / w.sum(), 0)
    t = torch.empty(n, dtype=torch.float64, device="cuda")
    for a in range(0, n, CH):
        m = min(CH, n - a)
        r = torch.rand(m, dtype=torch.float64, device="cuda", generator=g)
        t[a:a + m] = vals[torch.searchsorted(cdf, r).clamp_(max=k - 1)]
    bits = t.view(torch.int64)

    def signature():
        s, h = 0, torch.zeros(4096, dtype=torch.int64, device="cuda")
        for a in range(0, n, CH):
            v = bits[a:a + CH]
            s = (s + int(v.sum().item())) & ((1 << 64) - 1)  # exact modulo 2^64
            h += torch.bincount((v >> 52) & 4095, minlength=4096)
        return s, h.cpu().numpy()

    before = signature()
    ls.sort_(t)
    torch.cuda.synchronize()
    assert ls.stream_status() == 0
    prev = None
    for a in range(0, n, CH):  # non-decreasing (positive finite values)
        v = t[a:a + CH]
        assert bool(torch.all(v[1:] >= v[:-1]).item())
        assert prev is None or float(v[0].item()) >= prev
        prev = float(v[-1].item())
    after = signature()
    assert before[0] == after[0]
    assert np.array_equal(before[1], after[1])
