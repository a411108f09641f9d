"""The allocation-free radix sort entry point (ls_radix_sort_u64_noalloc).

Callers that cannot allocate device memory when they sort (a framework whose
caching allocator owns the GPU's memory, a latency-bound loop that must stay out
of the driver's allocator) use this variant; its scratch is a static device
array inside the library.  This file is collected last on purpose: if it fails,
a run that stops at the first failure has already run every other test.  It
passes alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2107_03290_gb300 as ls  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    ls.build()
    return ls.load()


def _sorted_both(lib, a: np.ndarray):
    """Sort copies of `a` with the allocating and the allocation-free entry
    points, both through the C ABI; return the two results."""
    t1 = torch.from_numpy(a.copy()).cuda()
    t2 = torch.from_numpy(a.copy()).cuda()
    st = torch.cuda.current_stream().cuda_stream
    assert lib.ls_radix_sort_u64(t1.data_ptr(), t1.numel(), st) == 0
    assert lib.ls_radix_sort_u64_noalloc(t2.data_ptr(), t2.numel(), st) == 0
    torch.cuda.synchronize()
    return t1.cpu().numpy(), t2.cpu().numpy()


def test_noalloc_matches_allocating_entry_point(lib):
    rng = np.random.default_rng(2024)
    # two calls in a row: the second is smaller, so stale scratch contents of
    # the first must not leak into it
    for n in (ls.NOALLOC_RADIX_MAX, 300_001):
        a = rng.integers(0, 2**64 - 1, n, dtype=np.uint64)
        a[: n // 7] = a[n // 3]  # duplicates
        ref, got = _sorted_both(lib, a)
        assert np.array_equal(got, ref)                  # integer keys: exact
        assert np.array_equal(got, np.sort(a))


def test_noalloc_rejects_oversized_input(lib):
    n = ls.NOALLOC_RADIX_MAX + 1
    a = np.arange(n, 0, -1, dtype=np.uint64)
    t = torch.from_numpy(a.copy()).cuda()
    rc = lib.ls_radix_sort_u64_noalloc(t.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    assert rc == 1  # LS_ERR_INVALID
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), a)
    assert lib.ls_stream_status(None) == 0
