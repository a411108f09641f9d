"""Argsort and key-value sort (ls_argsort, ls_sort_pairs) against the oracle.

The stable argsort is unique (equal keys keep their input order), so the GPU
permutation is compared element for element with the oracle's plain
definition (std::stable_sort of the positions by total order); the sorted keys
with the oracle's sort, and the values with the input values gathered through
the oracle's permutation."""
import numpy as np
import pytest

import lsgen
import oracle

torch = pytest.importorskip("torch")
import paper_2107_03290_gb300 as ls  # noqa: E402
from test_gpu_parity import make  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ls.build()
    ls.load()
    torch.cuda.init()
    yield
    assert ls.stream_status() == 0


DISTS = ["normal", "zipf_lognormal", "uniform_u64", "timestamp_u32", "exponential_f32",
         "twodups", "all_equal", "two_values", "signed_zeros", "f64_specials", "f32_specials",
         "u64_extremes", "sorted", "reverse"]


@pytest.mark.parametrize("n", [0, 1, 2, 17, 1000, 65_537, 1_000_003])
@pytest.mark.parametrize("dist", DISTS)
def test_argsort_matches_oracle(dist, n):
    keys = make(dist, n) if n else make(dist, 2)[:0]
    t = torch.from_numpy(keys.copy()).cuda()
    perm = ls.argsort(t)
    torch.cuda.synchronize()
    got = perm.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.reference_argsort(keys))
    assert np.array_equal(t.cpu().numpy().view(np.uint8), keys.view(np.uint8))  # keys untouched


@pytest.mark.parametrize("vdt", [np.uint32, np.float64])
@pytest.mark.parametrize("dist", ["normal", "zipf_lognormal", "uniform_u64", "timestamp_u32",
                                  "exponential_f32", "f32_specials", "two_values"])
def test_sort_pairs_matches_oracle(dist, vdt):
    keys = make(dist, 300_001)
    n = keys.size
    vals = (np.arange(n, dtype=np.uint64) * np.uint64(2654435761)).astype(vdt) if vdt == np.uint32 \
        else lsgen.normal_f64(n, 99)
    tk, tv = torch.from_numpy(keys.copy()).cuda(), torch.from_numpy(vals.copy()).cuda()
    ls.sort_pairs_(tk, tv)
    torch.cuda.synchronize()
    perm = oracle.reference_argsort(keys).astype(np.int64)
    want_k = oracle.reference_sort(keys)
    assert np.array_equal(tk.cpu().numpy().view(np.uint8), want_k.view(np.uint8))
    assert np.array_equal(tv.cpu().numpy().view(np.uint8), vals[perm].view(np.uint8))


def test_argsort_rejects_bad_arguments():
    lib = ls.load()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert lib.ls_argsort(t.data_ptr(), None, 8, 0, None) == 1
    assert lib.ls_argsort(t.data_ptr(), p.data_ptr() + 2, 8, 0, None) == 1
    assert lib.ls_argsort(t.data_ptr(), p.data_ptr(), 1 << 32, 0, None) == 1
    assert lib.ls_sort_pairs(t.data_ptr(), p.data_ptr(), 8, 0, 2, None) == 1
