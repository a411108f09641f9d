"""Bit-exact parity at the benchmarked sizes.

Every benchmarked configuration is sorted through the C ABI exactly as
``bench.py`` sorts it (same generator, seed, size and parameters) and compared
byte for byte with the oracle's plain definition of the result (std::sort by
IEEE total order).  Alg. 2 ends with an insertion sort that leaves the keys
monotonically ordered (Sec. 4.2), so the sorted output is unique and no sum,
norm or histogram stands in for the comparison.

* the 1M-key N(0,1) latency case, with the paper's setting (fan-out 1000,
  1000 leaves, 1% sample; Sec. 6.1) and with the planner's fan-out;
* the five 200M-key single-array workloads (Zipf-lognormal f64, uniform u64,
  Gaussian-mixture f64, timestamp-like u32, exponential f32);
* every one of the 4,096 arrays of the batched workload;
* every request input of the serving workload, through the server.

The oracle's std::sort runs in a host thread while the GPU sorts.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import lsgen
import oracle

torch = pytest.importorskip("torch")
import paper_2107_03290_gb300 as ls  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ls.build()
    ls.load()
    torch.cuda.init()
    yield
    torch.cuda.empty_cache()


def _first_diff(got: np.ndarray, want: np.ndarray) -> str:
    w = got.view(np.uint64 if got.itemsize == 8 else np.uint32)
    v = want.view(np.uint64 if want.itemsize == 8 else np.uint32)
    d = np.flatnonzero(w != v)
    return f"{d.size} of {got.size} positions differ, first {d[:5]}"


def assert_bytes_equal(got: np.ndarray, want: np.ndarray):
    assert got.dtype == want.dtype and got.shape == want.shape
    if not np.array_equal(got.view(np.uint8), want.view(np.uint8)):
        raise AssertionError(_first_diff(got, want))


def sort_on_gpu(keys: np.ndarray, params=None) -> np.ndarray:
    t = torch.from_numpy(keys).cuda()
    ls.sort_(t, params)
    torch.cuda.synchronize()
    assert ls.stream_status() == 0
    out = t.cpu().numpy()
    del t
    return out


@pytest.mark.parametrize("cfg", [dict(fanout=1000, leaves=1000), dict()],
                         ids=["fanout1000-leaves1000", "planner"])
def test_normal_1m_matches_oracle(cfg):
    dt, n, fn = lsgen.WORKLOADS["normal_1m_f64"]
    keys = fn(n)
    got = sort_on_gpu(keys, ls.default_params(**cfg))
    assert_bytes_equal(got, oracle.reference_sort(keys))


@pytest.mark.parametrize("workload", ["zipf_lognormal_200m_f64", "uniform_200m_u64",
                                      "gauss_mix_200m_f64", "timestamp_200m_u32",
                                      "exponential_200m_f32"])
def test_200m_workload_matches_oracle(workload):
    dt, n, fn = lsgen.WORKLOADS[workload]
    keys = fn(n)
    with ThreadPoolExecutor(1) as ex:
        want = ex.submit(oracle.reference_sort, keys)
        got = sort_on_gpu(keys)
        want = want.result()
    assert_bytes_equal(got, want)


def test_batched_workload_every_array_matches_oracle():
    arrays = lsgen.batch_arrays(4096, seed=6)
    sizes = np.array([a.size for a in arrays], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    flat = np.concatenate(arrays)
    with ThreadPoolExecutor(16) as ex:
        wants = list(ex.map(oracle.reference_sort, arrays))
    work = torch.from_numpy(flat).cuda()
    views = [work[offs[i]:offs[i + 1]] for i in range(len(arrays))]
    ls.sort_batch_(views)
    torch.cuda.synchronize()
    assert ls.stream_status() == 0
    res = work.cpu().numpy()
    bad = [i for i in range(len(arrays))
           if not np.array_equal(res[offs[i]:offs[i + 1]].view(np.uint8), wants[i].view(np.uint8))]
    assert not bad, f"{len(bad)} of {len(arrays)} arrays differ, first {bad[:5]}"


def test_serving_inputs_match_oracle():
    """The serving workload's 64 request inputs (10K to 64M keys, three key
    types, 30% heavy), submitted together so that small ones are batched and
    large ones take the full sort, each compared with the oracle."""
    pool = lsgen.serving_pool(64)
    with ThreadPoolExecutor(16) as ex:
        wants = list(ex.map(oracle.reference_sort, pool))
    srcs = [torch.from_numpy(a).cuda() for a in pool]
    dsts = [torch.empty_like(x) for x in srcs]
    torch.cuda.synchronize()
    srv = ls.Server(hbm_budget_bytes=120 << 30, max_inflight=64, streams=8)
    tickets = [srv.submit(d, src=x) for d, x in zip(dsts, srcs)]
    for k in tickets:
        srv.wait(k)
    srv.close()
    bad = [i for i, (d, w) in enumerate(zip(dsts, wants))
           if not np.array_equal(d.cpu().numpy().view(np.uint8), w.view(np.uint8))]
    assert not bad, f"{len(bad)} of {len(pool)} requests differ, first {bad[:5]}"
