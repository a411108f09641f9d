"""Benchmark of the GB300 learned sort (one JSON line on stdout, rank 0).

Default workload: 200,000,000 float64 keys, each one of 100,000 distinct
lognormal(0,2) values chosen by Zipf(1.1) rank (the high-duplicate plain
single-array sort), seed 1.  A step is one full ls_sort of the workload
(train, level 0, level 1, in-bucket sorts), inputs resident in HBM; the input
is restored from a pristine device copy before every step, outside the timed
interval.  The inputs (1.6 GB) are larger than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--n N]

--impl reference times the CPU oracle (test infrastructure) on bounded samples
of the same workload on the host cores.  Multi-GPU runs are independent
replicas (the sort does not shard across GPUs here): every rank sorts its own
copy; value = keys over all ranks / max time.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lsgen  # noqa: E402

METRIC = "keys/s & HBM GB/s vs roofline, 1 GB300; batched/served vs plain; p50/p99 ms"
L2_BYTES = 129 * 1000 * 1000  # GB300 L2
NPT = {"f64": np.float64, "u64": np.uint64, "f32": np.float32, "u32": np.uint32}
WIDTH = {"f64": 8, "u64": 8, "f32": 4, "u32": 4}


def total_order_keys(a: np.ndarray) -> np.ndarray:
    """IEEE totalOrder keys of float arrays (unsigned order for integers), as
    unsigned integers of the same width: an order-preserving bijection."""
    w = a.dtype.itemsize
    u = a.view(np.uint64 if w == 8 else np.uint32)
    if a.dtype.kind != "f":
        return u
    sgn = (u >> np.array(8 * w - 1, u.dtype)).astype(bool)
    top = np.array(1 << (8 * w - 1), u.dtype)
    return np.where(sgn, ~u, u | top)


def order_keys_torch(torch, t):
    """The total order as signed 64-bit keys of a CUDA tensor (floats by IEEE
    totalOrder, unsigned integers by value), for a check by a library sort."""
    if t.element_size() == 8:
        u = t.view(torch.int64)
        if t.dtype == torch.float64:
            return torch.where(u < 0, u ^ 0x7FFFFFFFFFFFFFFF, u)
        return u ^ (-(1 << 63))
    b = t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    if t.dtype == torch.float32:
        return torch.where(b >= (1 << 31), (~b) & 0xFFFFFFFF, b | (1 << 31))
    return b


def run_configs(ls, torch, names, steps: int, warmup: int, peak: float):
    """The other benchmarked single-array workloads, each timed like the main
    line (CUDA events around every ls_sort call, input restored outside them)
    and checked element for element against a library sort of its keys."""
    out = []
    stream = torch.cuda.current_stream()
    for name in names:
        dt, keys = make_workload(name, 0)
        n, w = keys.size, WIDTH[dt]
        pristine = torch.from_numpy(keys).cuda()
        del keys
        work = torch.empty_like(pristine)
        prm = ls.default_params(leaves=1000)
        for _ in range(warmup):
            work.copy_(pristine)
            ls.sort_(work, prm)
        torch.cuda.synchronize()
        want = torch.sort(order_keys_torch(torch, pristine)).values
        exact = bool(torch.equal(order_keys_torch(torch, work), want))
        del want
        ms = []
        for _ in range(steps):
            work.copy_(pristine)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ls.sort_(work, prm)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = float(np.mean(ms))
        out.append({"workload": name, "n": int(n), "dtype": dt, "ms_per_sort": m,
                    "keys_per_s": n / (m / 1e3), "frac_4nw": 4 * n * w / (m / 1e3) / 1e9 / peak,
                    "steps": steps, "exact": exact,
                    "check": "torch.sort of the total-order keys (a library sort), element for element"})
        del pristine, work
        torch.cuda.empty_cache()
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def kernel_algorithmic_bytes(st: dict, n: int, w: int) -> dict:
    """Algorithmic bytes per launch of each timed kernel: K2 reads every key
    once (n*w); K4 reads every key and writes the non-equality ones."""
    eq = st["n_eq_keys"]
    return {
        "k_l0_hist": n * w,                        # read every key once
        "k_l0_scatter": n * w + (n - eq) * w,      # read every key, write non-equality keys
        "k_bucket_sort": None,                     # reported through the whole-sort figure
    }


def _region_sha(path: str, begin: str, end: str) -> str:
    text = open(path, "rb").read()
    a = text.index(begin.encode())
    b = text.index(end.encode(), a)
    return hashlib.sha256(text[a:b]).hexdigest()[:16]


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source (the region of its file between two markers) is still the one the
    counters were taken on (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}@{workload}")
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2107_03290_gb300", "csrc", e["source"])
    try:
        h = _region_sha(src, e["begin"], e["end"])
    except (OSError, ValueError, KeyError):
        return None
    return e["bytes_per_launch"] if h == e["source_sha"] else None


def replica_throughput(dev_ms: float, n: int, dist=None, device: str = "cuda"):
    """Whole-job keys/s of independent replicas (one per rank, each sorting its
    own n keys; nothing is exchanged): all ranks' keys over the slowest rank's
    time.  Returns (keys/s, slowest ms)."""
    import torch
    tmax, world = dev_ms, 1
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([dev_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax = float(t.item())
    return n * world / (tmax / 1000.0), tmax


def make_workload(name: str, n: int):
    dt, n0, fn = lsgen.WORKLOADS[name]
    return dt, fn(n if n else n0)


def run_reference(args, rank: int):
    import oracle
    if rank != 0:
        return
    dt, keys = make_workload(args.workload, args.n)
    sample = min(keys.size, args.ref_sample)
    # warmup + timed steps, each a bounded sample of the workload
    for i in range(args.warmup):
        oracle.learned_sort(keys[:sample])
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.learned_sort(keys[:sample])
    t = time.perf_counter() - t0
    v = sample * args.steps / t
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "keys/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000 * t / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dt, "data": "synthetic",
           "config": {"workload": args.workload, "n": int(keys.size), "dtype": dt,
                      "l2": "host memory (the oracle runs on one host core)",
                      "parallelism": "single"},
           "cpu_baseline": {"value": v, "unit": "keys/s", "cores": 1, "kind": "oracle",
                            "sample": f"first {sample} keys of the workload per step"},
           "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched(ls, torch, count: int, steps: int, warmup: int, with_loop: bool = True):
    """Batched workload: `count` float64 arrays (lognormal sizes, median 64K,
    clipped to [1K, 4M]; N(0,1) / U[0,1) / Zipf(1.1) over 10^4 values), sorted
    by one ls_sort_batch call per step; baseline: ls_sort on each array in turn
    on the same stream.  Inputs restored from a device copy outside the timing."""
    arrays = lsgen.batch_arrays(count, seed=6)
    sizes = [a.size for a in arrays]
    total = int(sum(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    host = torch.from_numpy(np.concatenate(arrays))
    pristine = host.to("cuda")
    work = torch.empty_like(pristine)
    views = [work[offs[i]:offs[i + 1]] for i in range(count)]
    st = torch.cuda.current_stream()

    def timed(fn, k):
        ms = []
        for _ in range(k):
            work.copy_(pristine)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    batch = lambda: ls.sort_batch_(views)
    loop = lambda: [ls.sort_(v) for v in views]
    timed(batch, warmup)
    mb = timed(batch, steps)
    ok = True
    res = work.cpu().numpy()
    for i in (0, count // 2, count - 1):
        seg = res[offs[i]:offs[i + 1]]
        ok = ok and bool(np.all(seg[1:] >= seg[:-1]))
    big = sum(1 for x in sizes if x > 8192)
    out = {"workload": f"batch_{count}_f64", "arrays": count, "keys": total,
           "model": (f"{big} arrays above 8192 keys split by a line through their own key range "
                     "(a one-leaf model; split targets per size class from csrc/ls_tuned.h), "
                     f"{count - big} sorted directly in one segment; no sampled RMI per array"),
           "batched_ms": float(np.median(mb)), "batched_keys_per_s": total / (np.median(mb) / 1e3),
           "steps": steps, "warmup": warmup, "sorted_sampled": ok}
    if with_loop:
        timed(loop, 1)
        ml = timed(loop, max(1, steps // 2))
        out.update(loop_ms=float(np.median(ml)), loop_keys_per_s=total / (np.median(ml) / 1e3),
                   batched_vs_loop=float(np.median(ml) / np.median(mb)))
    del pristine, work, views
    torch.cuda.empty_cache()
    return out


def run_serving(ls, torch, rates, seconds: float, pool_size: int = 64,
                budget_bytes: int = 120 << 30, client_bytes: int = 48 << 30, streams: int = 8,
                p99_bound_ms: float = 100.0):
    """Serving workload: Poisson arrivals of sort requests (each copies one
    device-resident pool array into its own buffer on the server's stream,
    outside the device time), admission by an HBM budget; reports p50/p99 of
    arrival -> completion and keys/s against sorting the same requests one at
    a time with the plain entry point in arrival order."""
    import threading
    pool = lsgen.serving_pool(pool_size)
    dev = [torch.from_numpy(a).cuda() for a in pool]
    rng = np.random.default_rng(11)
    out = []
    svc = None
    for rate in rates:
        n_req = max(1, int(rate * seconds))
        gaps = rng.exponential(1.0 / rate, n_req)
        picks = rng.integers(0, pool_size, n_req)
        srv = ls.Server(hbm_budget_bytes=budget_bytes, max_inflight=64, streams=streams)
        lat, done_t = [], []
        outstanding = []
        cv = threading.Condition()
        in_bytes = [0]

        def waiter():
            while True:
                with cv:
                    while not outstanding:
                        cv.wait()
                    item = outstanding.pop(0)
                if item is None:
                    return
                tk, buf, nb = item
                st = srv.wait(tk)
                lat.append(st["total_ms"])
                done_t.append(time.perf_counter())
                with cv:
                    in_bytes[0] -= nb
                    cv.notify_all()
                del buf

        th = threading.Thread(target=waiter)
        th.start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt = t0
        keys = 0
        for i in range(n_req):
            nxt += gaps[i]
            d = time.perf_counter() - nxt
            if d < 0:
                time.sleep(-d)
            src = dev[picks[i]]
            nb = src.numel() * src.element_size()
            with cv:  # the client keeps at most client_bytes of request buffers
                while in_bytes[0] + nb > client_bytes:
                    cv.wait()
                in_bytes[0] += nb
            buf = torch.empty_like(src)
            tk = srv.submit(buf, src=src)
            keys += src.numel()
            with cv:
                outstanding.append((tk, buf, nb))
                cv.notify_all()
        with cv:
            outstanding.append(None)
            cv.notify_all()
        th.join()
        wall = max(done_t) - t0
        srv.close()
        # one at a time: the same requests, in arrival order, each sorted by
        # the plain entry point on one stream.  Its device time depends only on
        # the pool array, so each array's plain sort is timed (median of 3) and
        # a single-stream queue is replayed on the arrival times.
        if svc is None:
            svc = plain_service_ms(ls, torch, dev)
        arr = np.cumsum(gaps)
        done, c = np.empty(n_req), 0.0
        for i in range(n_req):
            c = max(arr[i], c) + svc[picks[i]] / 1e3
            done[i] = c
        lat1 = (done - arr) * 1e3
        wall1 = done[-1]
        out.append({"rate_req_s": rate, "requests": n_req, "seconds": seconds, "keys": int(keys),
                    "offered_keys_per_s": keys / arr[-1],
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "served_keys_per_s": keys / wall,
                    "one_at_a_time": {"p50_ms": float(np.percentile(lat1, 50)),
                                      "p99_ms": float(np.percentile(lat1, 99)),
                                      "keys_per_s": keys / wall1},
                    "served_vs_one_at_a_time": (keys / wall) / (keys / wall1)})
        torch.cuda.empty_cache()
    # capacity: the highest rate whose p99 stays within the bound, and the
    # plain loop's device rate on the same mix (requests back to back)
    ok = [r for r in out if r["p99_ms"] <= p99_bound_ms]
    device_rate = sum(a.numel() for a in dev) / (sum(svc) / 1e3)
    cap = max(ok, key=lambda r: r["rate_req_s"]) if ok else None
    del dev
    torch.cuda.empty_cache()
    return {"workload": "serving_poisson", "pool": pool_size, "hbm_budget_gb": budget_bytes >> 30,
            "seconds_per_rate": seconds, "rates": out, "p99_bound_ms": p99_bound_ms,
            "one_at_a_time_device_keys_per_s": device_rate,
            "capacity": None if cap is None else {
                "rate_req_s": cap["rate_req_s"], "p99_ms": cap["p99_ms"],
                "served_keys_per_s": cap["served_keys_per_s"],
                "vs_one_at_a_time_device_rate": cap["served_keys_per_s"] / device_rate}}


def plain_service_ms(ls, torch, dev, reps: int = 3):
    """Device time (ms) of one plain ls_sort of each pool array (median of reps)."""
    st = torch.cuda.current_stream()
    out = []
    for src in dev:
        ms = []
        for _ in range(reps + 1):
            buf = src.clone()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ls.sort_(buf)
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            del buf
        out.append(float(np.median(ms[1:])))
    return out


def host_sorted_tk(a: np.ndarray, threads: int = 16) -> np.ndarray:
    """Total-order keys of `a`, sorted on the host: chunks sorted in threads,
    then merged by a stable sort (which merges sorted runs)."""
    from concurrent.futures import ThreadPoolExecutor
    tk = total_order_keys(a)
    parts = np.array_split(tk, threads)
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(np.sort, parts))
    return np.sort(np.concatenate(parts), kind="stable")


def run_suite(ls, torch, names, steps: int, warmup: int, peak: float):
    """The paper's synthetic suite: one JSON line per workload with keys/s,
    the fraction of the 4*n*w roofline, the realized duplicate ratio and the
    element-wise check of the GPU output against a host sort."""
    stream = torch.cuda.current_stream()
    for name in names:
        dt, n0, fn = lsgen.WORKLOADS[name]
        keys = fn(n0)
        n, w = keys.size, keys.dtype.itemsize
        pristine = torch.from_numpy(keys).cuda()
        work = torch.empty_like(pristine)
        ms = []
        for i in range(warmup + steps):
            work.copy_(pristine)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ls.sort_(work)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                ms.append(e0.elapsed_time(e1))
        got = total_order_keys(work.cpu().numpy())
        want = host_sorted_tk(keys)
        ok = bool(np.array_equal(got, want))
        distinct = int(1 + np.count_nonzero(want[1:] != want[:-1]))
        # keys whose value occurs at least twice
        starts = np.flatnonzero(np.concatenate([[True], want[1:] != want[:-1]]))
        runs = np.diff(np.concatenate([starts, [n]]))
        in_dups = int(runs[runs >= 2].sum())
        t = float(np.median(ms))
        print(json.dumps({"suite": name, "n": n, "dtype": dt, "ms_p50": t, "ms_min": float(np.min(ms)),
                          "keys_per_s": n / (t / 1e3),
                          "frac_4nw": 4 * n * w / (t / 1e3) / 1e9 / peak,
                          "dup_ratio": 1.0 - distinct / n, "frac_keys_repeated": in_dups / n,
                          "parity": "bit-exact" if ok else "MISMATCH", "steps": steps}), flush=True)
        del pristine, work, got, want, keys
        torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="zipf_lognormal_200m_f64", choices=list(lsgen.WORKLOADS))
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--fanout", type=int, default=None,
                    help="level-0 fan-out (default: 1000 for normal_1m_f64, else the planner's)")
    ap.add_argument("--leaves", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=10_000_000)
    ap.add_argument("--ref-sample", type=int, default=2_000_000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", type=int, default=4096, help="arrays of the batched line (0: skip)")
    ap.add_argument("--configs", default="uniform_200m_u64,gauss_mix_200m_f64,timestamp_200m_u32,exponential_200m_f32",
                    help="other workloads timed and checked in the same run (empty: none)")
    ap.add_argument("--latency-steps", type=int, default=50,
                    help="timed calls of the 1M-key latency case (fan-out 1000, 1000 leaves; 0: skip)")
    ap.add_argument("--inplace-steps", type=int, default=10,
                    help="timed sorts of the workload with LS_FLAG_IN_PLACE (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="seconds per arrival rate of the serving line (0: skip)")
    ap.add_argument("--suite", default="",
                    help="'paper' (or a comma list of workloads): the synthetic suite, one JSON "
                         "line per workload, instead of the benchmark line")
    ap.add_argument("--serve-rates", default="200,500,1000,2000,5000",
                    help="arrival rates (requests/s) of the serving line")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_2107_03290_gb300 as ls

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    ls.build()
    ls.load()

    if args.suite:
        names = list(lsgen.SUITE) if args.suite == "paper" else args.suite.split(",")
        run_suite(ls, torch, names, args.steps, args.warmup, load_peaks()[0])
        return

    dt, keys = make_workload(args.workload, args.n)
    n = keys.size
    w = WIDTH[dt]
    host = torch.from_numpy(keys).pin_memory()
    pristine = host.to("cuda", non_blocking=True)
    work = torch.empty_like(pristine)
    stream = torch.cuda.current_stream()

    # the 1M-key latency case runs with the stated configuration (fan-out 1000,
    # 1000 leaves, 1% sample; Sec. 6.1); the 200M-key workloads with the
    # planner's fan-out unless --fanout is given
    fanout = args.fanout if args.fanout is not None else (1000 if args.workload == "normal_1m_f64" else 0)
    prm = ls.default_params(fanout=fanout, leaves=args.leaves)

    def step(stats=True):
        work.copy_(pristine)
        return ls.sort_(work, prm, stats=stats)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # correctness of the benchmarked path, outside the timed region: the GPU's
    # output equals, element for element, a host sort of the pristine keys by
    # their total-order keys (the ordering contract; the sorted output is unique)
    ok = bool(np.array_equal(total_order_keys(work.cpu().numpy()),
                             np.sort(total_order_keys(keys))))

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # timed steps: CUDA events on the launching stream around each ls_sort call
    # (no per-phase events inside the call); the input is restored before each
    # step, outside the events
    step_ms = []
    l_before = ls.kernel_launches()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            work.copy_(pristine)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ls.sort_(work, prm)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
    launches = ls.kernel_launches() - l_before
    dev_ms = float(np.mean(step_ms))
    value, tmax = replica_throughput(dev_ms, n, dist, "cuda")
    # per-phase times from separate, untimed calls with statistics (events
    # between the phases)
    per = [step() for _ in range(max(3, min(10, args.steps)))]
    torch.cuda.synchronize()

    # per-kernel times and the roofline of the dominant kernel
    ks = ["ms_train", "ms_hist", "ms_scan", "ms_scatter", "ms_classify", "ms_level1", "ms_fill",
          "ms_sort_small", "ms_sort_large", "ms_fallback"]
    kms = {k: float(np.mean([s[k] for s in per])) for k in ks}
    peak, peak_kind = load_peaks()
    names = {"ms_hist": "k_l0_hist", "ms_scatter": "k_l0_scatter"}
    alg = kernel_algorithmic_bytes(per[-1], n, w)
    dom = max(("ms_hist", "ms_scatter"), key=lambda k: kms[k])
    kname = names[dom]
    ach = alg[kname] / (kms[dom] / 1e3) / 1e9
    whole = 4 * n * w / (dev_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_kind": peak_kind,
            "traffic": traffic_for(kname, args.workload),
            "share": kms[dom] / dev_ms,
            "sort_4nw": {"achieved": whole, "frac": whole / peak,
                         "note": "4*n*w bytes (2-pass read+write) / whole-sort time"}}

    # end to end through ls_sort_host: pinned host buffer, copies timed
    e2e = None
    if args.e2e_steps > 0:
        hb = torch.empty_like(host).pin_memory()
        ptr, code = hb.data_ptr(), {"f64": 0, "u64": 1, "f32": 2, "u32": 3}[dt]
        hb.copy_(host)
        ls.sort_host_ptr(ptr, n, code)
        tot = 0.0
        for _ in range(args.e2e_steps):
            hb.copy_(host)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ls.sort_host_ptr(ptr, n, code)
            tot += time.perf_counter() - t1
        e2e = {"value": n * world / (tot / args.e2e_steps), "unit": "keys/s",
               "h2d_bytes_per_step": n * w, "d2h_bytes_per_step": n * w}
        del hb

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        smp = min(n, args.cpu_sample)
        t1 = time.perf_counter()
        oracle.learned_sort(keys[:smp])
        tc = time.perf_counter() - t1
        cpu = {"value": smp / tc, "unit": "keys/s", "cores": 1, "kind": "oracle",
               "sample": f"first {smp} keys of the workload, one oracle LearnedSort 2.0 call"}

    # the 1M-key latency case with the paper's setting (fan-out 1000, 1000 leaves,
    # 1% sample; Sec. 6.1), L2-resident: per-call device time, p50 and p99
    latency = None
    if args.latency_steps > 0 and rank == 0 and args.workload != "normal_1m_f64":
        ldt, lkeys = make_workload("normal_1m_f64", 0)
        lpr = torch.from_numpy(lkeys).cuda()
        lwk = torch.empty_like(lpr)
        lprm = ls.default_params(fanout=1000, leaves=1000)
        for _ in range(5):
            lwk.copy_(lpr)
            ls.sort_(lwk, lprm)
        torch.cuda.synchronize()
        l_ok = bool(np.array_equal(total_order_keys(lwk.cpu().numpy()),
                                   np.sort(total_order_keys(lkeys))))
        lms = []
        for _ in range(args.latency_steps):
            lwk.copy_(lpr)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ls.sort_(lwk, lprm)
            e1.record(stream)
            e1.synchronize()
            lms.append(e0.elapsed_time(e1))
        lwk.copy_(lpr)
        lst = ls.sort_(lwk, lprm, stats=True)
        torch.cuda.synchronize()
        latency = {"workload": "normal_1m_f64", "n": int(lkeys.size), "fanout": 1000, "leaves": 1000,
                   "p50_ms": float(np.percentile(lms, 50)), "p99_ms": float(np.percentile(lms, 99)),
                   "mean_ms": float(np.mean(lms)), "steps": args.latency_steps, "exact": l_ok,
                   "train_ms": lst["ms_train"], "launches": int(lst["n_launches"])}
        del lpr, lwk

    # the in-place variant on the same workload: its own timed sorts (CUDA
    # events around each call), its exactness, and the workspace it allocates
    inplace = None
    if args.inplace_steps > 0 and rank == 0:
        pip = ls.default_params(fanout=fanout, leaves=args.leaves, flags=ls.FLAG_IN_PLACE)
        code = {"f64": 0, "u64": 1, "f32": 2, "u32": 3}[dt]
        for _ in range(2):
            work.copy_(pristine)
            ls.sort_(work, pip)
        torch.cuda.synchronize()
        ip_ok = bool(np.array_equal(total_order_keys(work.cpu().numpy()),
                                    np.sort(total_order_keys(keys))))
        ip_ms = []
        for _ in range(args.inplace_steps):
            work.copy_(pristine)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ls.sort_(work, pip)
            e1.record(stream)
            e1.synchronize()
            ip_ms.append(e0.elapsed_time(e1))
        work.copy_(pristine)
        ip_st = ls.sort_(work, pip, stats=True)
        torch.cuda.synchronize()
        ipm = float(np.mean(ip_ms))
        inplace = {"ms_per_sort": ipm, "keys_per_s": n / (ipm / 1e3), "steps": args.inplace_steps,
                   "exact": ip_ok,
                   "workspace_bytes": ls.workspace_bytes(n, code, pip),
                   "workspace_bytes_regular": ls.workspace_bytes(n, code, prm),
                   "phase_ms": {k: ip_st[k] for k in ("ms_train", "ms_hist", "ms_scan", "ms_scatter",
                                                      "ms_classify", "ms_level1", "ms_fill",
                                                      "ms_sort_small", "ms_sort_large",
                                                      "ms_fallback")},
                   "note": ("LS_FLAG_IN_PLACE: level 0 by fragment flush over read positions, "
                            "device defragment and cleanup; refinement levels and fallback "
                            "split in place per CTA; no n-key scratch")}

    configs = None
    if args.configs and rank == 0 and world == 1:
        names = [c for c in args.configs.split(",") if c and c != args.workload]
        configs = run_configs(ls, torch, names, steps=10, warmup=3, peak=load_peaks()[0])

    batched = None
    if args.batch > 0 and rank == 0:
        batched = run_batched(ls, torch, args.batch, steps=5, warmup=2)
    serving = None
    if args.serve_seconds > 0 and rank == 0:
        rates = [int(r) for r in args.serve_rates.split(",")]
        serving = run_serving(ls, torch, rates, args.serve_seconds)

    if rank == 0:
        last = per[-1]
        out = {"metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dt,
               "data": "synthetic",
               "config": {"workload": args.workload, "n": n, "dtype": dt,
                          "l2": ("inputs larger than L2 (restored from a device copy each step)"
                                 if n * w > L2_BYTES else
                                 "inputs fit in L2 (latency case; restored from a device copy each step)"),
                          "parallelism": "replicas" if world > 1 else "single",
                          "fanout": per[-1]["fanout"], "leaves": per[-1]["leaves"],
                          "sample": per[-1]["sample_size"]},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(launches), "clocks": clk.summary(),
               "wall_ms_per_step": 1000 * wall / args.steps, "correct": ok,
               "ms_p50": float(np.median(step_ms)),
               "ms_min": float(np.min(step_ms)),
               "ms_with_phase_events": float(np.mean([x["ms_total"] for x in per])),
               "kernels_ms": kms, "latency": latency, "configs": configs, "in_place": inplace,
               "batched": batched,
               "serving": serving,
               "path": {k: last[k] for k in ("n_heavy", "n_ext", "max_bucket", "n_eq_keys",
                                             "n_level1", "n_segments", "n_fallback", "n_fill",
                                             "n_launches", "sample_size")}}
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
