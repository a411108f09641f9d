"""GPU parity: the CUDA learned sort (called through the C ABI) against the
CPU oracle.  The sorted output is unique under the total order, so every
comparison of final outputs is bit-exact.  Stage tests compare the training
step and the level-0 histogram with the oracle's spec functions."""
import numpy as np
import pytest

import lsgen
import oracle

torch = pytest.importorskip("torch")
import paper_2107_03290_gb300 as ls  # noqa: E402

pytestmark = pytest.mark.gpu

NPT = {"f64": np.float64, "u64": np.uint64, "f32": np.float32, "u32": np.uint32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ls.build()
    ls.load()
    torch.cuda.init()
    yield
    assert ls.stream_status() == 0, "device status word set"


def gpu_sort(keys: np.ndarray, params=None, misalign: int = 0) -> np.ndarray:
    if misalign:
        base = torch.empty(keys.size + misalign, dtype=torch.from_numpy(keys[:0]).dtype,
                           device="cuda")
        t = base[misalign:]
        t.copy_(torch.from_numpy(keys))
    else:
        t = torch.from_numpy(keys.copy()).cuda()
    ls.sort_(t, params)
    torch.cuda.synchronize()
    return t.cpu().numpy()


def assert_same(got: np.ndarray, keys: np.ndarray):
    want = oracle.reference_sort(keys)
    assert got.dtype == want.dtype and got.shape == want.shape
    if not np.array_equal(got.view(np.uint8), want.view(np.uint8)):
        bad = np.flatnonzero(got.view(np.uint8).reshape(got.size, -1).any(1)
                             != want.view(np.uint8).reshape(got.size, -1).any(1))
        w = got.view(np.uint64 if got.itemsize == 8 else np.uint32)
        v = want.view(np.uint64 if got.itemsize == 8 else np.uint32)
        diff = np.flatnonzero(w != v)
        raise AssertionError(f"{diff.size} of {got.size} positions differ, first {diff[:5]}")


def _specials(dt, n, rng):
    if dt == np.float64:
        pool = np.array([-np.inf, -1e300, -1.0, -5e-324, -0.0, 0.0, 5e-324, 1.0, 2.0, 1e300,
                         np.inf, np.nan, -np.nan], np.float64)
    else:
        pool = np.array([-np.inf, -3e38, -1.0, -1e-45, -0.0, 0.0, 1e-45, 1.0, 2.0, 3e38, np.inf,
                         np.nan, -np.nan], np.float32)
    return rng.choice(pool, n)


def make(dist: str, n: int) -> np.ndarray:
    rng = np.random.default_rng(n * 7 + len(dist))
    if dist == "normal":
        return lsgen.normal_f64(n, 1)
    if dist == "zipf_lognormal":
        return lsgen.zipf_lognormal_f64(n, 2, k=max(10, n // 20))
    if dist == "uniform_u64":
        return lsgen.uniform_u64(n, 3)
    if dist == "gauss_mix":
        return lsgen.gauss_mix_f64(n, 4)
    if dist == "timestamp_u32":
        m = max(1000, (n // 1000) * 1000)
        return lsgen.timestamp_u32(m, 5)[:n].copy()
    if dist == "exponential_f32":
        return lsgen.exponential_f32(n, 6)
    if dist == "rootdups":
        return lsgen.rootdups_f64(n)
    if dist == "twodups":
        return lsgen.twodups_f64(n)
    if dist == "sorted":
        return np.sort(lsgen.normal_f64(n, 7))
    if dist == "reverse":
        return np.sort(lsgen.normal_f64(n, 8))[::-1].copy()
    if dist == "all_equal":
        return np.full(n, 3.25)
    if dist == "two_values":
        return rng.choice(np.array([1.0, 7.0]), n)
    if dist == "signed_zeros":
        return rng.choice(np.array([-0.0, 0.0]), n)
    if dist == "heavy_99.99":
        a = np.full(n, 42.0)
        a[rng.integers(0, n, max(1, n // 10000))] = rng.normal(size=max(1, n // 10000))
        return a
    if dist == "u32_small_range":
        return lsgen.uniform_u32(n, 9, bits=4)
    if dist == "u64_extremes":
        return rng.choice(np.array([0, 1, 2**63 - 1, 2**63, 2**64 - 1], np.uint64), n)
    if dist == "f64_specials":
        return _specials(np.float64, n, rng)
    if dist == "f32_specials":
        return _specials(np.float32, n, rng)
    raise KeyError(dist)


DISTS = ["normal", "zipf_lognormal", "uniform_u64", "gauss_mix", "timestamp_u32",
         "exponential_f32", "rootdups", "twodups", "sorted", "reverse", "all_equal", "two_values",
         "signed_zeros", "heavy_99.99", "u32_small_range", "u64_extremes", "f64_specials",
         "f32_specials"]
SIZES = [2, 3, 17, 1000, 4097, 65_537, 1_000_003]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dist", DISTS)
def test_sort_matches_oracle(dist, n):
    keys = make(dist, n)
    assert_same(gpu_sort(keys), keys)


@pytest.mark.parametrize("dist", ["normal", "zipf_lognormal", "uniform_u64", "timestamp_u32",
                                  "exponential_f32", "f32_specials", "f64_specials"])
@pytest.mark.parametrize("cfg", [
    dict(fanout=1, leaves=1), dict(fanout=4, leaves=8), dict(fanout=16, leaves=64),
    dict(fanout=3000, leaves=2000), dict(flags=ls.FLAG_NO_HEAVY), dict(heavy_per_bucket=8),
    dict(fanout=1000, heavy_per_bucket=4), dict(fanout=64, heavy_per_bucket=15),
    dict(sample_div=1000, sample_max=500)], ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_sort_params(dist, cfg):
    """Small fan-outs force level-1 re-partitions and the radix fallback."""
    keys = make(dist, 300_001)
    assert_same(gpu_sort(keys, ls.default_params(**cfg)), keys)


@pytest.mark.parametrize("dist", ["normal", "exponential_f32", "timestamp_u32", "uniform_u64",
                                  "zipf_lognormal"])
@pytest.mark.parametrize("mis", [1, 2, 3])
def test_sort_misaligned(dist, mis):
    """Unaligned starts exercise the TMA head/tail path (bulk copies need 16 B);
    zipf_lognormal also takes the compaction of the non-equality keys."""
    for n in (5, 4099, 200_003):
        keys = make(dist, n)
        assert_same(gpu_sort(keys, misalign=mis), keys)


def test_sort_fallback_path():
    """Two distinct values the model cannot separate, equality buckets off:
    the level-1 split cannot shrink the bucket, so the radix fallback sorts it."""
    a = np.concatenate([np.full(150_000, 3.0), np.full(150_000, np.nextafter(3.0, 4.0)),
                        lsgen.normal_f64(10_000, 3)])
    np.random.default_rng(0).shuffle(a)
    p = ls.default_params(flags=ls.FLAG_NO_HEAVY)
    t = torch.from_numpy(a.copy()).cuda()
    st = ls.sort_(t, p, stats=True)
    assert st["n_fallback"] + st["n_fill"] >= 1
    assert_same(t.cpu().numpy(), a)


@pytest.mark.parametrize("dist", ["normal", "zipf_lognormal", "gauss_mix", "uniform_u64",
                                  "exponential_f32", "timestamp_u32"])
def test_train_matches_oracle(dist):
    n = 400_000
    keys = make(dist, n)
    p = ls.default_params(leaves=256, fanout=256, heavy_per_bucket=4)
    m = ls.train(torch.from_numpy(keys).cuda(), p, with_sample=True)
    op = oracle.params(leaves=256, fanout=256)
    # sample: stratified offsets, sorted by total order -- exact
    s = oracle.sample_size(n, op)
    assert m["sample_size"] == s
    idx = oracle.sample_indices(n, s, 0).astype(np.int64)
    want_tk = np.sort(oracle.total_order_keys(keys[idx]))
    assert np.array_equal(m["sorted_sample_tk"], want_tk)
    # FP64 fit: same definition, different reduction order
    fm = oracle.train(keys, op)
    assert m["sample_finite"] == fm.m.s_fin
    np.testing.assert_allclose(m["root"], fm.root, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(m["leaf"][:, 3:], fm.leaf[:, 3:], rtol=0, atol=0)  # lo, hi exact
    np.testing.assert_allclose(m["leaf"][:, :3], fm.leaf[:, :3], rtol=1e-9, atol=1e-12)
    # the level-0 map evaluated on the GPU's FP64 model
    gm = oracle.FittedModel(256)
    gm.m.root[0], gm.m.root[1], gm.m.root[2] = m["root"]
    gm.leaf[:] = m["leaf"]
    ev = oracle.EvalParams(gm, 256)
    smp = keys[idx]
    # level-0 thresholds: bisection of the FP64 bucket map over the total order
    thr, pmax = oracle.spec_thresholds(oracle.EvalParams(gm, 256), oracle.dtype_name(keys))
    assert np.array_equal(m["thr"], thr)
    assert m["pos_max"] == pmax
    # heavy set from the sorted sample
    sorted_smp = np.sort(smp)
    fin = sorted_smp[np.isfinite(sorted_smp.astype(np.float64))] if sorted_smp.dtype.kind == "f" \
        else sorted_smp
    fin = oracle.reference_sort(fin)
    h = oracle.spec_heavy(fin, int(m["tau"]), 4, ev)
    assert np.array_equal(h, m["heavy_tk"])


@pytest.mark.parametrize("dist", ["normal", "zipf_lognormal", "uniform_u64"])
def test_train_large_sample_matches_oracle(dist):
    """20M keys: a 200K-key sample of 8-byte keys, sorted by the sample sort
    whose splitters the sampling kernel draws (smaller samples and 4-byte keys
    take the radix sort); sorted sample exact, fit within rtol 1e-9, and the
    whole sort bit-exact."""
    n = 20_000_000
    keys = make(dist, n)
    p = ls.default_params(leaves=1000, fanout=256)
    m = ls.train(torch.from_numpy(keys).cuda(), p, with_sample=True)
    op = oracle.params(leaves=1000, fanout=256)
    s = oracle.sample_size(n, op)
    assert m["sample_size"] == s and s > (1 << 17)
    idx = oracle.sample_indices(n, s, 0).astype(np.int64)
    want_tk = np.sort(oracle.total_order_keys(keys[idx]))
    assert np.array_equal(m["sorted_sample_tk"], want_tk)
    fm = oracle.train(keys, op)
    np.testing.assert_allclose(m["root"], fm.root, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(m["leaf"][:, 3:], fm.leaf[:, 3:], rtol=0, atol=0)
    np.testing.assert_allclose(m["leaf"][:, :3], fm.leaf[:, :3], rtol=1e-9, atol=1e-12)
    assert_same(gpu_sort(keys), keys)


@pytest.mark.parametrize("dist", ["normal", "zipf_lognormal", "two_values", "timestamp_u32",
                                  "exponential_f32", "f64_specials"])
def test_level0_histogram_matches_spec(dist):
    n = 300_000
    keys = make(dist, n)
    p = ls.default_params(leaves=128, fanout=200, heavy_per_bucket=4)
    t = torch.from_numpy(keys).cuda()
    h = ls.level0_histogram(t, p)
    m = ls.train(t, p)
    ev = oracle.EvalParams.from_export(m, 128, 200)
    hs = oracle.spec_ext_histogram(ev, keys, m["heavy_tk"])
    assert h.sum() == n
    assert np.array_equal(h, hs)


def _colliding_heavy(n: int, seed: int) -> np.ndarray:
    """Heavy values that share slots of the level-0 heavy table (the key's
    bits, halves folded by xor, 32-bit Fibonacci hashing to 13 bits): six
    values in each of four slots, with decreasing frequencies, so that most of
    them lose their slot and must be recognised by the full lookup; 30% normal
    background."""
    rng = np.random.default_rng(seed)
    cand = np.unique(rng.lognormal(0.0, 2.0, 200_000))
    bits = cand.view(np.uint64)
    fold = ((bits ^ (bits >> np.uint64(32))) & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    slot = (((fold * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)) >> np.uint64(19)).astype(np.int64)
    vals = []
    for sl in np.flatnonzero(np.bincount(slot, minlength=8192) >= 6)[:4]:
        vals.extend(cand[slot == sl][:6])
    vals = np.array(vals)
    w = 1.0 / np.arange(1, vals.size + 1)
    cnt = np.floor(0.7 * n * w / w.sum()).astype(np.int64)
    keys = np.concatenate([np.repeat(vals, cnt), rng.normal(0.0, 3.0, n - cnt.sum())])
    return keys[rng.permutation(n)]


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("lim", [1e30, 1e300])
@pytest.mark.parametrize("n", [3_000, 300_001])
def test_keys_across_binades(dt, lim, n):
    """Log-uniform magnitudes of both signs (every binade from 1/lim to lim,
    zeros and denormals mixed in), so that segments span many binades: the
    in-bucket slot map through the keys' FP32 images, and (beyond the FP32
    range) the fallback to the total-order map."""
    rng = np.random.default_rng(n + int(np.log10(lim)))
    hi = min(np.log(lim), np.log(np.finfo(dt).max) - 1)
    mag = np.exp(rng.uniform(-hi, hi, n))
    keys = (np.where(rng.random(n) < 0.5, -mag, mag)).astype(dt)
    k = max(1, n // 100)
    keys[rng.integers(0, n, k)] = np.array([0.0, -0.0, np.finfo(dt).tiny / 4], dt)[rng.integers(0, 3, k)]
    assert_same(gpu_sort(keys), keys)


@pytest.mark.parametrize("n", [300_000, 3_000_001])
def test_heavy_slot_collisions(n):
    keys = _colliding_heavy(n, n)
    assert_same(gpu_sort(keys), keys)
    if n == 300_000:  # level-0 counts against the spec
        p = ls.default_params(leaves=128, fanout=200, heavy_per_bucket=4)
        t = torch.from_numpy(keys).cuda()
        h = ls.level0_histogram(t, p)
        m = ls.train(t, p)
        ev = oracle.EvalParams.from_export(m, 128, 200)
        assert np.array_equal(h, oracle.spec_ext_histogram(ev, keys, m["heavy_tk"]))


@pytest.mark.parametrize("n", [1, 2, 100, 4095, 4096, 4097, 100_000, 1_000_000])
def test_radix_sort_u64(n):
    rng = np.random.default_rng(n)
    for a in (rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2),
              rng.integers(0, 300, n, dtype=np.uint64) << np.uint64(40)):
        t = torch.from_numpy(a.copy()).cuda()
        ls.radix_sort_u64_(t)
        assert np.array_equal(t.cpu().numpy(), np.sort(a))


@pytest.mark.parametrize("n", [2, 3, 100, 8191, 8192, 8193, 100_000, 2_000_000])
def test_sample_sort_u64(n):
    """The training sample's sample sort: random keys, few distinct values
    (splitters repeat, their keys skip the sort), presorted and reversed runs."""
    rng = np.random.default_rng(n + 1)
    r = rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    for a in (r, rng.integers(0, 300, n, dtype=np.uint64) << np.uint64(40), np.sort(r),
              np.sort(r)[::-1].copy(), np.full(n, 2**64 - 1, dtype=np.uint64)):
        t = torch.from_numpy(a.copy()).cuda()
        ls.sample_sort_u64_(t)
        assert np.array_equal(t.cpu().numpy(), np.sort(a))


@pytest.mark.parametrize("n", [20_000, 300_001])
def test_sample_sort_u64_oversized_gap(n):
    """Oversample positions (i * n / 8192) hold widely spread keys and every
    other position a small distinct key, so one gap holds almost every key:
    the chunk-sort-and-merge path."""
    rng = np.random.default_rng(n)
    a = rng.permutation(np.arange(1, n + 1, dtype=np.uint64))
    pos = (np.arange(8192, dtype=np.uint64) * np.uint64(n)) // np.uint64(8192)
    a[pos.astype(np.int64)] = (np.arange(8192, dtype=np.uint64) + np.uint64(1)) << np.uint64(50)
    t = torch.from_numpy(a.copy()).cuda()
    ls.sample_sort_u64_(t)
    assert np.array_equal(t.cpu().numpy(), np.sort(a))


def test_empty_and_one():
    for dt in (torch.float64, torch.float32):
        for n in (0, 1):
            t = torch.ones(n, dtype=dt, device="cuda")
            ls.sort_(t)
            assert t.cpu().tolist() == [1.0] * n


def test_invalid_arguments():
    lib = ls.load()
    assert lib.ls_sort(None, 5, 0, None) == 1
    assert lib.ls_sort(None, 0, 0, None) == 0
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert lib.ls_sort(t.data_ptr(), 8, 7, None) == 1
    assert lib.ls_sort(t.data_ptr() + 1, 4, 0, None) == 1       # misaligned for f64


def test_sort_host_e2e():
    a = lsgen.zipf_lognormal_f64(500_000, 11, k=1000)
    b = a.copy()
    ls.sort_host(b)
    assert_same(b, a)


@pytest.mark.parametrize("off", [0, 1, 3])
@pytest.mark.parametrize("dist", ["zipf_lognormal", "uniform_u64", "exponential_f32"])
def test_sort_host_pinned(dist, off):
    """ls_sort_host on a pinned host buffer (copied by the SMs over the link),
    at an offset that leaves it unaligned to 16 bytes."""
    keys = make(dist, 300_001)
    dt = torch.from_numpy(keys[:0]).dtype
    h = torch.empty(keys.size + off, dtype=dt).pin_memory()
    v = h[off:]
    v.copy_(torch.from_numpy(keys))
    code = {8: 0 if keys.dtype == np.float64 else 1, 4: 2 if keys.dtype == np.float32 else 3}[keys.itemsize]
    ls.sort_host_ptr(v.data_ptr(), keys.size, code)
    assert_same(v.numpy().copy(), keys)


def test_sort_batch():
    arrays = lsgen.batch_arrays(64, seed=6, scale=0.02)
    ts = [torch.from_numpy(a.copy()).cuda() for a in arrays]
    ls.sort_batch_(ts)
    torch.cuda.synchronize()
    for a, t in zip(arrays, ts):
        assert_same(t.cpu().numpy(), a)


BATCH_MIX = [("normal", 0), ("normal", 1), ("uniform_u64", 2), ("two_values", 3),
             ("normal", 2047), ("zipf_lognormal", 2048), ("normal", 2049), ("uniform_u64", 4096),
             ("exponential_f32", 4097), ("f64_specials", 8192), ("f32_specials", 8193),
             ("heavy_99.99", 50_000), ("zipf_lognormal", 300_001), ("timestamp_u32", 200_000),
             ("uniform_u64", 1_000_003), ("gauss_mix", 777_777)]


@pytest.mark.parametrize("dt", [np.float64, np.uint64, np.float32, np.uint32])
def test_sort_batch_mixed_sizes(dt):
    """Arrays of every size class (in-bucket jobs, key-range levels) in one call."""
    arrays = []
    for d, n in BATCH_MIX:
        a = make(d, n)
        if a.dtype != dt:  # re-type the distribution's values for this dtype
            a = a.astype(np.float64)
            if np.dtype(dt).kind == "u":
                a = np.nan_to_num(a, nan=0.0, posinf=1e18, neginf=0.0)
                a = np.abs(a) * (1 << 20)
                a = np.minimum(a, float(np.iinfo(dt).max) / 2)
            a = a.astype(dt)
        arrays.append(a)
    ts = [torch.from_numpy(a.copy()).cuda() for a in arrays]
    ls.sort_batch_(ts)
    torch.cuda.synchronize()
    assert ls.stream_status() == 0
    for a, t in zip(arrays, ts):
        assert_same(t.cpu().numpy(), a)


def test_server_alone_equals_mix():
    """Each request's result is the same alone and in a concurrent mix."""
    arrays = [make(d, n) for d, n in [("normal", 300_000), ("zipf_lognormal", 1_000_000),
                                      ("uniform_u64", 200_000), ("exponential_f32", 700_000),
                                      ("heavy_99.99", 50_000), ("normal", 10_000)]]
    alone = []
    for a in arrays:
        t = torch.from_numpy(a.copy()).cuda()
        ls.sort_(t)
        alone.append(t.cpu().numpy())
    srv = ls.Server(hbm_budget_bytes=8 << 30, max_inflight=4, streams=3)
    ts = [torch.from_numpy(a.copy()).cuda() for a in arrays]
    torch.cuda.synchronize()
    tickets = [srv.submit(t) for t in ts]
    stats = [srv.wait(k) for k in tickets]
    srv.close()
    for a, t, al, st in zip(arrays, ts, alone, stats):
        got = t.cpu().numpy()
        assert np.array_equal(got.view(np.uint8), al.view(np.uint8))
        assert_same(got, a)
        assert st["total_ms"] >= st["device_ms"] >= 0


def test_server_batched_mix_from_sources():
    """Requests admitted together go through one batched launch per key type
    (large ones through the full sort); inputs copied on the server's stream."""
    specs = [("normal", 1_000), ("zipf_lognormal", 300_000), ("uniform_u64", 50_000),
             ("exponential_f32", 20_000), ("normal", 4_500_000), ("two_values", 9_000),
             ("uniform_u64", 2_000_000), ("timestamp_u32", 100_000), ("gauss_mix", 123_457),
             ("normal", 17_000_000)]  # above the batching limit (2^24 keys): the full sort
    arrays = [make(d, n) for d, n in specs]
    srcs = [torch.from_numpy(a).cuda() for a in arrays]
    dsts = [torch.empty_like(x) for x in srcs]
    torch.cuda.synchronize()
    srv = ls.Server(hbm_budget_bytes=16 << 30, max_inflight=16, streams=2)
    tickets = [srv.submit(d, src=x) for d, x in zip(dsts, srcs)]
    stats = [srv.wait(k) for k in tickets]
    srv.close()
    for a, d, x, st in zip(arrays, dsts, srcs, stats):
        assert_same(d.cpu().numpy(), a)
        assert np.array_equal(x.cpu().numpy().view(np.uint8), a.view(np.uint8))  # source intact
        assert st["total_ms"] >= st["device_ms"] >= 0


def test_server_admission():
    srv = ls.Server(hbm_budget_bytes=1 << 20, max_inflight=2, streams=1)
    t = torch.zeros(1_000_000, dtype=torch.float64, device="cuda")
    with pytest.raises(ls.LsError) as e:
        srv.submit(t)
    assert e.value.code == 5
    srv.close()
