"""Pins for the CPU oracle (no GPU).  Each test checks the oracle against
something other than itself: the plain definition of the result (sorted order,
computed by numpy on the total-order integer keys), published constants,
closed forms and hand-worked examples of Alg. 1 / Alg. 2."""
import itertools
import math
import struct

import numpy as np
import pytest

import lsgen
import oracle
from conftest import read_golden


def tk_numpy(a: np.ndarray) -> np.ndarray:
    """Total-order integer key computed with numpy bit ops (independent of the oracle)."""
    if a.dtype == np.float64:
        u = a.view(np.uint64)
        neg = (u >> np.uint64(63)) != 0
        return np.where(neg, ~u, u | np.uint64(1 << 63))
    if a.dtype == np.float32:
        u = a.view(np.uint32).astype(np.uint64)
        neg = (u >> np.uint64(31)) != 0
        return np.where(neg, (~u) & np.uint64(0xFFFFFFFF), u | np.uint64(0x80000000))
    return a.astype(np.uint64)


def assert_sorted_permutation(out: np.ndarray, inp: np.ndarray):
    """Invariants: non-decreasing by total order; same multiset of bit patterns."""
    t_out, t_in = tk_numpy(out), tk_numpy(inp)
    assert np.all(t_out[1:] >= t_out[:-1]), "not non-decreasing"
    assert np.array_equal(t_out, np.sort(t_in)), "not a permutation of the input"


def test_default_params_match_paper():
    g = {r[0]: int(r[1]) for r in read_golden("paper_params.txt")}
    p = oracle.params()
    assert p.leaves == g["leaves"]
    assert p.fanout == g["fanout"]
    assert p.frag_cap == g["frag_cap"]
    assert 100 // p.sample_div == g["sample_percent"]


@pytest.mark.parametrize("fname,dt,fmt", [("total_order_f64.txt", np.float64, "<Q"),
                                          ("total_order_f32.txt", np.float32, "<I")])
def test_total_order_golden(fname, dt, fmt):
    rows = read_golden(fname)
    bits = [int(r[0], 16) for r in rows]
    keys = np.array([struct.unpack("<d" if dt == np.float64 else "<f",
                                   struct.pack(fmt, b))[0] for b in bits], dtype=dt)
    tk = oracle.total_order_keys(keys)
    assert np.all(tk[1:] > tk[:-1])
    rng = np.random.default_rng(0)
    for _ in range(20):
        perm = rng.permutation(len(keys))
        got = oracle.reference_sort(keys[perm])
        assert got.view(np.uint64 if dt == np.float64 else np.uint32).tolist() == bits
        got2 = oracle.learned_sort(keys[perm], oracle.params(n_small=0, fanout=4, leaves=2))
        assert got2.view(np.uint64 if dt == np.float64 else np.uint32).tolist() == bits


def test_splitmix64_published_vector():
    g = {r[0]: int(r[1], 16) for r in read_golden("splitmix64.txt")}
    # s = 1 sample over n = 2^63 keys: offset = mix64(seed ^ 0) mod 2^63.
    assert int(oracle.sample_indices(1 << 63, 1, 0)[0]) == g["output0"] % (1 << 63)
    # the second output of the generator is mix64 of its second state
    st = 0x9E3779B97F4A7C15
    assert int(oracle.sample_indices(1 << 63, 1, st)[0]) == g["output1"] % (1 << 63)


@pytest.mark.parametrize("n,s", [(1000, 10), (1000, 1000), (12345, 678), (10**9, 10**5),
                                 (7, 3), (1, 1)])
def test_sample_indices_stratified(n, s):
    idx = oracle.sample_indices(n, s, 7).astype(np.int64)
    k = np.arange(s, dtype=object)
    lo = np.array([kk * n // s for kk in k], dtype=np.int64)
    stride = max(1, n // s)
    assert np.all(idx >= lo) and np.all(idx < lo + stride)
    assert np.all(idx < n) and np.all(np.diff(idx) > 0)
    if s == n:
        assert np.array_equal(idx, np.arange(n))


def test_sample_size_rule():
    p = oracle.params()
    assert oracle.sample_size(1_000_000, p) == 10_000          # 1% (Sec. 6.1)
    assert oracle.sample_size(200_000_000, p) == 2_000_000
    assert oracle.sample_size(1000, p) == 1000                 # at least min(n, 2L)
    assert oracle.sample_size(0, p) == 0
    assert oracle.sample_size(10**9, oracle.params(sample_max=12345)) == 12345


def test_fit_closed_form_line():
    # keys 0..m-1: eCDF y_k = k/m, so least squares is exact: slope 1/m.
    m = 4096
    xs = np.arange(m, dtype=np.float64)
    fm = oracle.fit_sorted(xs, 1)
    a, c, b = fm.root
    assert a == pytest.approx(1.0 / m, rel=1e-12)
    assert c == pytest.approx((m - 1) / 2, rel=1e-12)
    assert b == pytest.approx((m - 1) / (2 * m), rel=1e-12)
    la, lc, lb, lo, hi = fm.leaf[0]
    assert la == pytest.approx(1.0 / m, rel=1e-12)
    assert (lo, hi) == (0.0, 1.0)
    # L leaves over a uniform grid: leaf l holds keys [l k, (l+1) k).
    L = 16
    fm = oracle.fit_sorted(xs, L)
    k = m // L
    for l in range(L):
        la, lc, lb, lo, hi = fm.leaf[l]
        assert la == pytest.approx(1.0 / m, rel=1e-9)
        assert lc == pytest.approx(l * k + (k - 1) / 2, rel=1e-12)
        assert lo == pytest.approx(l / L, abs=1e-15)
        assert hi == pytest.approx((l + 1) / L, abs=1e-15)
        # F reproduces the eCDF at every key of the leaf
        for x in (l * k, l * k + k // 2, (l + 1) * k - 1):
            assert fm.predict(float(x)) == pytest.approx(x / m, abs=1e-12)


def test_fit_closed_form_degenerate():
    fm = oracle.fit_sorted(np.full(100, 3.5), 4)          # all equal: eCDF 0 everywhere
    assert fm.root[0] == 0.0 and fm.root[2] == 0.0
    assert fm.predict(3.5) == 0.0
    fm = oracle.fit_sorted(np.array([0.0] * 50 + [1.0] * 50), 1)   # two values
    a, c, b = fm.root
    assert a == pytest.approx(0.5) and c == pytest.approx(0.5) and b == pytest.approx(0.25)
    assert fm.predict(0.0) == pytest.approx(0.0) and fm.predict(1.0) == pytest.approx(0.5)
    fm = oracle.fit_sorted(np.zeros(0), 8)                 # no finite sample
    assert 0.0 <= fm.predict(1.0) <= 1.0
    # zero variance takes slope 0 even when the FP64 mean of the equal keys
    # does not round back to the key (35 copies of a value with a long mantissa)
    # (one key, six copies of x, ten keys: the six copies form a leaf, and
    # their centred FP64 sums are tiny but not zero)
    x = 104.66245874
    fm = oracle.fit_sorted(np.array([1.0] * 1 + [x] * 6 + [300.0] * 10), 64)
    own = [l for l in range(64) if abs(fm.leaf[l, 1] - x) < 1e-6]
    assert own, "the 35 copies should have a leaf of their own"
    assert all(fm.leaf[l, 0] == 0.0 for l in own)


@pytest.mark.parametrize("gen", ["normal", "zipf", "mix", "uniform_u64"])
def test_model_monotone_and_bounded(gen):
    n = 200_000
    a = {"normal": lambda: lsgen.normal_f64(n, 11),
         "zipf": lambda: lsgen.zipf_lognormal_f64(n, 12, k=1000),
         "mix": lambda: lsgen.gauss_mix_f64(n, 13),
         "uniform_u64": lambda: lsgen.uniform_u64(n, 14).astype(np.float64)}[gen]()
    fm = oracle.train(a, oracle.params(leaves=256))
    xs = np.sort(np.concatenate([a[:5000], [-np.inf, np.inf, -1e300, 1e300, 0.0, -0.0]]))
    F = np.array([fm.predict(float(x)) for x in xs])
    assert np.all(F >= 0) and np.all(F <= 1)
    assert np.all(np.diff(F) >= 0)
    # across every leaf boundary
    for l in range(1, 256):
        c = fm.leaf[l][1]
        if fm.leaf[l][0] == 0:
            continue
        x0 = np.nextafter(c, -np.inf)
        assert fm.predict(float(x0)) <= fm.predict(float(c)) <= fm.predict(float(np.nextafter(c, np.inf)))


def test_partition_worked_example():
    g = {r[0]: r[1:] for r in read_golden("partition_example.txt")}
    inp = np.array([float(v) for v in g["input"]])
    fm = oracle.FittedModel(1)
    fm.m.root[0], fm.m.root[1], fm.m.root[2] = 0.0, 0.0, 0.0      # all keys to leaf 0
    fm.leaf[0] = [1.0, 0.0, 0.0, 0.0, 1.0]                         # F(x) = x
    after, sizes, owners, fsz = oracle.partition(inp, fm, 0, 4, 2)
    assert after.tolist() == [float(v) for v in g["after_partition"]]
    assert sizes.tolist() == [int(v) for v in g["bucket_sizes"]]
    frags = [tuple(int(t) for t in v.split(":")) for v in g["fragments"]]
    assert list(zip(owners.tolist(), fsz.tolist())) == frags
    dfr = oracle.defragment(after, 4, sizes, owners, fsz)
    assert dfr.tolist() == [float(v) for v in g["after_defragment"]]


def test_partition_invariants():
    n, f, c = 50_000, 64, 100
    a = lsgen.normal_f64(n, 21)
    fm = oracle.train(a, oracle.params(leaves=128))
    after, sizes, owners, fsz = oracle.partition(a, fm, 0, f, c)
    assert int(sizes.sum()) == n and int(fsz.sum()) == n
    nfull = len(owners) - f
    assert np.all(fsz[:nfull] == c)            # flushed inside the loop: exactly c
    assert np.all(fsz[nfull:] < c)             # leftovers: one per bucket, < c
    assert owners[nfull:].tolist() == list(range(f))
    bucket = lambda x: min(f - 1, max(0, math.floor(fm.predict(float(x)) * f)))
    pos = 0
    for o, s in zip(owners.tolist(), fsz.tolist()):
        assert all(bucket(x) == o for x in after[pos:pos + s])
        pos += s
    dfr = oracle.defragment(after, f, sizes, owners, fsz)
    starts = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    expect = np.array([bucket(x) for x in a])
    for i in range(f):
        seg = dfr[starts[i]:starts[i + 1]]
        assert np.array_equal(np.sort(seg), np.sort(a[expect == i]))
    # level 1 with the monotone model: sub-buckets of bucket i are ordered
    i = int(np.argmax(sizes))
    seg = dfr[starts[i]:starts[i + 1]]
    after1, sizes1, own1, fsz1 = oracle.partition(seg, fm, 1, f, c, parent=i)
    d1 = oracle.defragment(after1, f, sizes1, own1, fsz1)
    st1 = np.concatenate([[0], np.cumsum(sizes1)]).astype(np.int64)
    nonempty = [j for j in range(f) if sizes1[j]]
    for j0, j1 in zip(nonempty, nonempty[1:]):
        assert d1[st1[j0]:st1[j0 + 1]].max() <= d1[st1[j1]:st1[j1 + 1]].min()


def _inputs():
    n = 60_000
    rng = np.random.default_rng(5)
    yield "normal", lsgen.normal_f64(n, 1)
    yield "uniform", lsgen.uniform_f64(n, 2)
    yield "zipf_lognormal", lsgen.zipf_lognormal_f64(n, 3, k=2000)
    yield "gauss_mix", lsgen.gauss_mix_f64(n, 4)
    yield "u64", lsgen.uniform_u64(n, 5)
    yield "u32_timestamp", lsgen.timestamp_u32(n, 6)
    yield "f32_exponential", lsgen.exponential_f32(n, 7)
    yield "rootdups", lsgen.rootdups_f64(n)
    yield "twodups", lsgen.twodups_f64(n)
    yield "sorted", np.sort(lsgen.normal_f64(n, 8))
    yield "reverse", np.sort(lsgen.normal_f64(n, 9))[::-1].copy()
    yield "all_equal", np.full(n, 2.5)
    yield "two_values", rng.choice([1.0, 7.0], n)
    yield "signed_zeros", rng.choice([-0.0, 0.0], n)
    heavy = np.full(n, 42.0)
    heavy[rng.integers(0, n, 3)] = rng.normal(size=3)
    yield "one_heavy_99.99", heavy
    yield "u32_small_range", lsgen.uniform_u32(n, 10, bits=4)
    yield "f32_specials", rng.choice(np.array([-np.inf, -1.0, -0.0, 0.0, 1e-45, 3.0, np.inf],
                                              np.float32), n)


@pytest.mark.parametrize("name,keys", list(_inputs()), ids=[x[0] for x in _inputs()])
@pytest.mark.parametrize("cfg", [dict(), dict(fanout=16, leaves=8, frag_cap=4, n_small=0)],
                         ids=["paper", "small_fanout"])
def test_learned_sort_equals_definition(name, keys, cfg):
    out = oracle.learned_sort(keys, oracle.params(**cfg))
    assert_sorted_permutation(out, keys)
    ref = oracle.reference_sort(keys)
    assert np.array_equal(out.view(np.uint8), ref.view(np.uint8))


def test_reference_sort_is_numpy_sort():
    for a in (lsgen.normal_f64(10_000, 3), lsgen.uniform_u64(10_000, 4),
              lsgen.exponential_f32(10_000, 5)):
        out = oracle.reference_sort(a)
        assert np.array_equal(tk_numpy(out), np.sort(tk_numpy(a)))


F64_SPECIALS = [-np.inf, -1.0, -0.0, 0.0, 1.0, 1.0, 2.0, np.inf, 5e-324, 1.7976931348623157e308]


@pytest.mark.parametrize("vals,dt", [
    (F64_SPECIALS[:8], np.float64),
    ([F64_SPECIALS[i] for i in (1, 2, 3, 8, 9, 4, 4, 0)], np.float64),
    ([0, 2**32 - 1, 5, 5, 0, 7, 2**31, 1], np.uint32),
    ([0, 2**64 - 1, 2**63, 3, 3, 3, 2**63 - 1, 12], np.uint64),
    ([-np.inf, -0.0, 0.0, 1e-45, 1.0, np.inf, np.nan, -np.nan], np.float32),
])
def test_exhaustive_permutations(vals, dt):
    """Every permutation of an 8-key multiset; the model path is forced (n_small = 0)."""
    base = np.array(vals, dtype=dt)
    expect = oracle.reference_sort(base)
    assert np.array_equal(tk_numpy(expect), np.sort(tk_numpy(base)))
    p = oracle.params(n_small=0, fanout=4, leaves=2, frag_cap=2)
    seen = set()
    for perm in itertools.permutations(range(len(base))):
        key = tuple(base[list(perm)].view(np.uint8).tolist())
        if key in seen:
            continue
        seen.add(key)
        out = oracle.learned_sort(base[list(perm)], p)
        assert np.array_equal(out.view(np.uint8), expect.view(np.uint8)), perm


def test_tiny_sizes():
    p = oracle.params(n_small=0)
    for n in range(0, 20):
        a = lsgen.normal_f64(n, 100 + n) if n else np.zeros(0)
        out = oracle.learned_sort(a, p)
        assert np.array_equal(out, oracle.reference_sort(a))


def test_model_quality_bounds_touch_up_work():
    """A wrong fit (dropped term, wrong sign) still sorts -- the insertion sort
    fixes it -- but leaves far more work to the touch-up.  Bound that work."""
    a = lsgen.uniform_f64(400_000, 31)
    out, tr = oracle.learned_sort(a, trace=True)
    assert tr["insertion_moves"] < 40 * a.size
    assert tr["max_bucket"] < 4 * a.size / 1000
    assert tr["sample_size"] == 4000 and tr["l1_partitions"] > 900


def _one_leaf_model(a: float) -> "oracle.FittedModel":
    """Root sends every key to leaf 0; the leaf is F(x) = clamp(a x, 0, 1)."""
    fm = oracle.FittedModel(1)
    fm.m.root[0], fm.m.root[1], fm.m.root[2] = 0.0, 0.0, 0.0
    fm.leaf[0] = [a, 0.0, 0.0, 0.0, 1.0]
    return fm


def test_counting_sort_worked_example():
    """Alg. 2's level-1 Partition, per-sub-bucket adj, paper-scale slots, running
    totals and pre-decrement placement, worked by hand on 10 keys."""
    g = {r[0]: r[1:] for r in read_golden("alg2_example.txt")}
    inp = np.array([float(v) for v in g["input"]])
    p = oracle.params(fanout=2, leaves=1, frag_cap=2, n_small=0)
    fm = _one_leaf_model(0.125)
    before, _ = oracle.sort_stages(inp, p, fm, touch_up=False)
    assert before.tolist() == [float(v) for v in g["before_touch_up"]]
    after, tr = oracle.sort_stages(inp, p, fm, touch_up=True)
    assert after.tolist() == [float(v) for v in g["sorted"]]
    assert tr["insertion_moves"] == int(g["insertion_moves"][0])
    assert tr["l1_partitions"] == 2 and tr["counting_sorts"] == 4


@pytest.mark.parametrize("f", [2, 4, 16])
def test_counting_sort_exact_under_exact_model(f):
    """Distinct keys k / N on a grid with the exact eCDF F(x) = x: level 0
    puts key k in bucket floor(f k / N), level 1 in sub-bucket floor(f^2 k / N)
    - i f, and the counting sort's slot (F - adj) N = k - (i f + j) N / f^2 is
    then the key's exact rank inside its sub-bucket, so the keys come out
    sorted before the touch-up and the insertion sort moves nothing."""
    N = 4096
    k = np.random.default_rng(f).permutation(N)
    keys = k.astype(np.float64) / N
    p = oracle.params(fanout=f, leaves=1, frag_cap=7, n_small=0)
    before, tr = oracle.sort_stages(keys, p, _one_leaf_model(1.0), touch_up=False)
    assert np.array_equal(before, np.arange(N) / N)
    assert tr["counting_sorts"] == f * f
    _, tr = oracle.sort_stages(keys, p, _one_leaf_model(1.0), touch_up=True)
    assert tr["insertion_moves"] == 0


def test_counting_sort_orders_all_but_shared_slots():
    """Before the touch-up, with a trained model and a small fan-out (large
    sub-buckets, so that the counting sort does the ordering): the keys run in
    (bucket, sub-bucket, slot) order, and a key is above its successor only
    when both share all three (the insertion sort's only work)."""
    a = lsgen.uniform_f64(40_000, 33)
    f, N = 4, a.size
    p = oracle.params(fanout=f, leaves=64, n_small=0)
    fm = oracle.train(a, p)
    before, tr = oracle.sort_stages(a, p, fm, touch_up=False)
    assert np.array_equal(np.sort(before), np.sort(a))
    assert tr["counting_sorts"] == f * f
    F = np.array([fm.predict(float(x)) for x in before])
    i = np.clip(np.floor(F * f), 0, f - 1)
    j = np.clip(np.floor(F * f * f) - i * f, 0, f - 1)
    sub = (i * f + j).astype(np.int64)
    n1 = np.bincount(sub, minlength=f * f)[sub]
    slot = np.clip(np.floor((F - sub / (f * f)) * N), 0, n1 - 1).astype(np.int64)
    key = sub * N + slot                              # (bucket, sub-bucket, slot)
    assert np.all(np.diff(key) >= 0)
    desc = np.flatnonzero(before[1:] < before[:-1])
    assert desc.size > 0 and np.all(key[desc] == key[desc + 1])
    out, tr = oracle.sort_stages(a, p, fm, touch_up=True)
    assert np.array_equal(out, np.sort(a))


# --------------------------------------------------------------------- spec functions
def _eval_for(a, L=128, f0=1000):
    fm = oracle.train(a, oracle.params(leaves=L))
    smp = a[oracle.sample_indices(a.size, oracle.sample_size(a.size, oracle.params(leaves=L)))
            .astype(np.int64)].astype(np.float64)
    smp = np.sort(smp[np.isfinite(smp)])
    return fm, smp, oracle.EvalParams(fm, f0)


@pytest.mark.parametrize("gen", ["normal", "gauss_mix", "zipf"])
def test_spec_bucket_monotone_and_thresholds(gen):
    a = {"normal": lambda: lsgen.normal_f64(100_000, 41),
         "gauss_mix": lambda: lsgen.gauss_mix_f64(100_000, 43),
         "zipf": lambda: lsgen.zipf_lognormal_f64(100_000, 44, k=3000)}[gen]()
    fm, smp, ev = _eval_for(a)
    xs = np.sort(np.concatenate([a[:4000], [-np.inf, np.inf, 0.0, -0.0, np.nan, -np.nan]]))
    xs = oracle.reference_sort(xs)
    b = oracle.spec_buckets(ev, xs).astype(np.int64)
    assert np.all(np.diff(b) >= 0) and b.min() >= 0 and b.max() <= 999
    # NaNs go to the end buckets by sign
    tk = oracle.total_order_keys(xs)
    assert b[0] == 0 and b[-1] == 999
    # the bucket is the number of thresholds at or below the key (bisection
    # over the total order agrees with the per-key evaluation)
    thr, pmax = oracle.spec_thresholds(ev, "f64")
    assert thr[0] == 0 and np.all(np.diff(thr.astype(object)) >= 0)
    cnt = np.searchsorted(thr[1:], tk, side="right")
    assert np.array_equal(np.minimum(cnt, pmax), b)
    # just below each finite threshold the bucket is smaller
    for bb in range(1, 1000, 97):
        t = int(thr[bb])
        key = lambda u: np.array([u], np.uint64).view(np.float64)
        x_at = key(t & 0x7FFFFFFFFFFFFFFF if t >> 63 else (~t) & (2**64 - 1))
        x_below = key((t - 1) & 0x7FFFFFFFFFFFFFFF if (t - 1) >> 63 else (~(t - 1)) & (2**64 - 1))
        assert oracle.spec_buckets(ev, x_at)[0] >= bb > oracle.spec_buckets(ev, x_below)[0]
    # Alg. 1 (Partition, level 0) puts the same number of keys in every bucket
    part, sizes, _, _ = oracle.partition(a, fm, 0, 1000, 100)
    allb = np.bincount(oracle.spec_buckets(ev, a).astype(np.int64), minlength=1000)
    assert np.array_equal(sizes.astype(np.int64), allb)


@pytest.mark.parametrize("dt", ["f32", "u32", "u64"])
def test_spec_thresholds_other_dtypes(dt):
    n = 50_000
    a = {"f32": lambda: lsgen.exponential_f32(n, 7),
         "u32": lambda: lsgen.timestamp_u32(n, 8),
         "u64": lambda: lsgen.uniform_u64(n, 9)}[dt]()
    L = 64
    fm = oracle.train(a, oracle.params(leaves=L))
    ev = oracle.EvalParams(fm, 100)
    thr, pmax = oracle.spec_thresholds(ev, dt)
    xs = oracle.reference_sort(a[:3000])
    b = oracle.spec_buckets(ev, xs).astype(np.int64)
    assert np.all(np.diff(b) >= 0)
    cnt = np.searchsorted(thr[1:], oracle.total_order_keys(xs), side="right")
    assert np.array_equal(np.minimum(cnt, pmax), b)
    if dt != "u64":
        assert int(thr.max()) <= 2**32


def test_spec_heavy_and_ext_histogram():
    keys = np.array([1.0] * 5 + [2.0] + [3.0] * 3 + [4.0] * 4, np.float64)
    fm = oracle.fit_sorted(keys, 2)
    ev = oracle.EvalParams(fm, 4)
    h = oracle.spec_heavy(keys, 3, 8, ev)
    assert h.tolist() == oracle.total_order_keys(np.array([1.0, 3.0, 4.0])).tolist()
    ev1 = oracle.EvalParams(fm, 1)
    h1 = oracle.spec_heavy(keys, 3, 1, ev1)          # one bucket, keep the longest run
    assert h1.tolist() == oracle.total_order_keys(np.array([1.0])).tolist()
    hist = oracle.spec_ext_histogram(ev1, keys, h)
    # one bucket owning heavies 1 < 3 < 4: slots <1, =1, (1,3), =3, (3,4), =4, >4
    assert hist.tolist() == [0, 5, 1, 3, 0, 4, 0]


# --------------------------------------------------------------------- argsort
def test_reference_argsort_small_example():
    """Total order with ties in input order: -inf < -0.0 < +0.0 < 1 < 2 = 2 < NaN."""
    keys = np.array([2.0, -0.0, 1.0, 0.0, 2.0, np.nan, -np.inf])
    assert oracle.reference_argsort(keys).tolist() == [6, 1, 3, 2, 0, 4, 5]


@pytest.mark.parametrize("dt", [np.float64, np.uint64, np.float32, np.uint32])
def test_reference_argsort_is_numpy_stable_argsort(dt):
    rng = np.random.default_rng(7)
    if np.dtype(dt).kind == "f":
        a = rng.choice(np.array([-np.inf, -2.5, -0.0, 0.0, 1e-30, 3.0, np.inf, np.nan], dt), 5000)
        a[:2000] = rng.normal(size=2000).astype(dt)
    else:
        a = rng.integers(0, 50, 5000).astype(dt)
    want = np.argsort(oracle.total_order_keys(a), kind="stable").astype(np.uint32)
    assert np.array_equal(oracle.reference_argsort(a), want)
