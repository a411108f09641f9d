"""GPU parity of the in-place variant (LS_FLAG_IN_PLACE; Sec. 4.2, Alg. 1's
fragment flush over read positions and Defragment): every output compared
byte for byte with the oracle's sorted array, as for the regular path, plus
the workspace it saves.

The cases force each in-place step: level 0 with and without heavy values
(equality keys counted, never moved), the model's level-1 split of buckets
with heavy values (sub-buckets laid out around the equality ranges), the
key-range levels, and the in-place radix fallback; unaligned starts take the
scalar block moves, and sizes that are not a multiple of the 128-byte block
take the partial last slot.
"""
import numpy as np
import pytest

import lsgen
import oracle
from test_gpu_parity import DISTS, assert_same, make

torch = pytest.importorskip("torch")
import paper_2107_03290_gb300 as ls  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ls.build()
    ls.load()
    torch.cuda.init()
    yield
    assert ls.stream_status() == 0, "device status word set"


def ip_params(**kw):
    flags = kw.pop("flags", 0) | ls.FLAG_IN_PLACE
    return ls.default_params(flags=flags, **kw)


def ip_sort(keys: np.ndarray, params=None, misalign: int = 0, stats: bool = False):
    dt = torch.from_numpy(keys[:0]).dtype
    if misalign:
        base = torch.empty(keys.size + misalign, dtype=dt, device="cuda")
        t = base[misalign:]
        t.copy_(torch.from_numpy(keys))
    else:
        t = torch.from_numpy(keys.copy()).cuda()
    st = ls.sort_(t, params if params is not None else ip_params(), stats=stats)
    torch.cuda.synchronize()
    return (t.cpu().numpy(), st) if stats else t.cpu().numpy()


SIZES = [2, 3, 17, 1000, 4097, 65_537, 1_000_003]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dist", DISTS)
def test_inplace_matches_oracle(dist, n):
    keys = make(dist, n)
    assert_same(ip_sort(keys), keys)


@pytest.mark.parametrize("dist", ["normal", "zipf_lognormal", "uniform_u64", "timestamp_u32",
                                  "exponential_f32", "f32_specials", "f64_specials", "rootdups"])
@pytest.mark.parametrize("cfg", [
    dict(fanout=1, leaves=1), dict(fanout=4, leaves=8), dict(fanout=16, leaves=64),
    dict(fanout=3000, leaves=2000), dict(flags=ls.FLAG_NO_HEAVY), dict(heavy_per_bucket=15),
    dict(fanout=512, heavy_per_bucket=4), dict(fanout=64, heavy_per_bucket=15),
    dict(sample_div=1000, sample_max=500)], ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_inplace_params(dist, cfg):
    """Small fan-outs push most keys through the in-place refinement levels and
    the in-place fallback; fan-out 3000 is capped at the in-place maximum."""
    keys = make(dist, 300_001)
    assert_same(ip_sort(keys, ip_params(**cfg)), keys)


@pytest.mark.parametrize("dist", ["normal", "exponential_f32", "timestamp_u32", "uniform_u64",
                                  "zipf_lognormal"])
@pytest.mark.parametrize("mis", [1, 2, 3])
def test_inplace_misaligned(dist, mis):
    for n in (5, 4099, 200_003, 1_000_001):
        keys = make(dist, n)
        assert_same(ip_sort(keys, misalign=mis), keys)


def test_inplace_fallback_path():
    """Two adjacent values the model cannot separate, equality buckets off:
    the key-range levels leave a segment above the in-bucket limit, which the
    in-place radix fallback splits by its lowest differing byte."""
    a = np.concatenate([np.full(150_000, 3.0), np.full(150_000, np.nextafter(3.0, 4.0)),
                        lsgen.normal_f64(10_000, 3)])
    np.random.default_rng(0).shuffle(a)
    got, st = ip_sort(a, ip_params(flags=ls.FLAG_NO_HEAVY), stats=True)
    assert st["n_fallback"] + st["n_fill"] >= 1
    assert_same(got, a)


def test_inplace_fallback_many_bytes():
    """Keys clustered on a geometric ladder: every key-range split leaves one
    large piece, so the fallback recurses over several bytes in place."""
    rng = np.random.default_rng(11)
    ladder = np.array([2.0 ** k for k in range(-40, 40)], np.float64)
    a = rng.choice(ladder, 400_000) * (1.0 + rng.integers(0, 64, 400_000) * 2.0 ** -52)
    got, st = ip_sort(a, ip_params(flags=ls.FLAG_NO_HEAVY, fanout=2, leaves=1), stats=True)
    assert_same(got, a)


@pytest.mark.parametrize("code,dt", [(0, np.float64), (3, np.uint32)])
def test_inplace_workspace(code, dt):
    """The in-place workspace drops the regular path's n-key scratch and its
    per-key ids (what is left: per-level tables, job lists and a few bytes per
    128-byte block); the call reports what it allocated."""
    n = 20_000_000
    w = np.dtype(dt).itemsize
    ip = ls.workspace_bytes(n, code, ip_params())
    reg = ls.workspace_bytes(n, code, ls.default_params())
    assert reg - ip >= n * (w + 4), (reg, ip)
    assert ip < reg // 2, (reg, ip)
    keys = lsgen.uniform_u32(n, 5) if dt == np.uint32 else lsgen.normal_f64(n, 5)
    got, st = ip_sort(keys, stats=True)
    assert st["workspace_bytes"] == ip
    assert_same(got, keys)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["zipf_lognormal_200m_f64", "uniform_200m_u64"])
def test_inplace_full_size(name):
    """The benchmarked 200M-key workloads, in place, against the oracle."""
    keys = lsgen.workload(name)
    got = ip_sort(keys)
    assert_same(got, keys)


def test_inplace_server_request():
    """A server configured in place sorts its large requests in place and
    charges less workspace for them at admission."""
    n = (1 << 24) + 12_345
    keys = lsgen.uniform_u64(n, 21)
    t = torch.from_numpy(keys.copy()).cuda()
    srv = ls.Server(hbm_budget_bytes=n * 8 + ls.workspace_bytes(n, 1, ip_params()) + (1 << 20),
                    in_place=True)
    try:
        tk = srv.submit(t)
        st = srv.wait(tk)
        assert st["status"] == 0
    finally:
        srv.close()
    assert_same(t.cpu().numpy(), keys)
