"""Seeded synthetic inputs for the learned-sort tests and benchmarks.

Holds none of the sorting method's arithmetic; only draws keys.  The C++
drawing code lives in ``gen.cpp`` and is compiled on first use (or by
``build()``) into ``_lsgen.so`` next to this file.

Workloads (synthetic stand-ins with the shapes of the paper's data sets and
of the benchmark configurations):

* ``normal_f64``            N(0,1) doubles (the paper's Standard Normal set, Sec. 6.1)
* ``zipf_lognormal_f64``    k distinct lognormal values chosen by Zipf rank
* ``uniform_u64``           uniform on [0, 2^64)
* ``gauss_mix_f64``         equal mixture of 5 Gaussians (Mix_Gauss, Sec. 6.1)
* ``timestamp_u32``         sorted runs with exact repeats and local swaps
* ``exponential_f32``       Exponential(1) rounded to float
* ``rootdups_f64`` / ``twodups_f64``  the RootDups/TwoDups sets of Sec. 6.1
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_lsgen.so")
_SRC = os.path.join(_HERE, "gen.cpp")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile gen.cpp into _lsgen.so (host C++ only)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            sig = {
                "lsg_normal_f64": [u64, u64, dbl, dbl, vp],
                "lsg_uniform_f64": [u64, u64, dbl, dbl, vp],
                "lsg_uniform_u64": [u64, u64, vp],
                "lsg_uniform_u32": [u64, u64, i32, vp],
                "lsg_zipf_lognormal_f64": [u64, u64, u64, dbl, dbl, dbl, vp],
                "lsg_zipf_rank_f64": [u64, u64, u64, dbl, vp],
                "lsg_gauss_mix_f64": [u64, u64, vp, i32, dbl, vp],
                "lsg_exponential_f32": [u64, u64, dbl, vp],
                "lsg_timestamp_u32": [u64, u64, u64, dbl, dbl, dbl, u64, vp],
                "lsg_rootdups_f64": [u64, vp],
                "lsg_twodups_f64": [u64, vp],
                "lsg_batch_sizes": [u64, u64, dbl, dbl, u64, u64, i32, vp, vp],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def normal_f64(n: int, seed: int = 0, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().lsg_normal_f64(seed, n, mu, sigma, _ptr(out))
    return out


def uniform_f64(n: int, seed: int = 0, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().lsg_uniform_f64(seed, n, lo, hi, _ptr(out))
    return out


def uniform_u64(n: int, seed: int = 2) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _L().lsg_uniform_u64(seed, n, _ptr(out))
    return out


def uniform_u32(n: int, seed: int = 0, bits: int = 32) -> np.ndarray:
    out = np.empty(n, np.uint32)
    _L().lsg_uniform_u32(seed, n, bits, _ptr(out))
    return out


def zipf_lognormal_f64(n: int, seed: int = 1, k: int = 100_000, s: float = 1.1,
                       mu: float = 0.0, sigma: float = 2.0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().lsg_zipf_lognormal_f64(seed, n, k, s, mu, sigma, _ptr(out))
    return out


def zipf_rank_f64(n: int, seed: int = 0, k: int = 1_000_000, s: float = 0.9) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().lsg_zipf_rank_f64(seed, n, k, s, _ptr(out))
    return out


def gauss_mix_f64(n: int, seed: int = 3, means=(-4.0, -2.0, 0.0, 2.0, 4.0),
                  sd: float = 0.5) -> np.ndarray:
    m = np.ascontiguousarray(means, np.float64)
    out = np.empty(n, np.float64)
    _L().lsg_gauss_mix_f64(seed, n, _ptr(m), len(m), sd, _ptr(out))
    return out


def exponential_f32(n: int, seed: int = 5, lam: float = 1.0) -> np.ndarray:
    out = np.empty(n, np.float32)
    _L().lsg_exponential_f32(seed, n, lam, _ptr(out))
    return out


def timestamp_u32(n: int, seed: int = 4, run_len: int = 1000, p_repeat: float = 0.5,
                  gap_mean: float = 4.0, p_swap: float = 0.05, radius: int = 50) -> np.ndarray:
    if n % run_len:
        raise ValueError("n must be a multiple of run_len")
    out = np.empty(n, np.uint32)
    _L().lsg_timestamp_u32(seed, n, run_len, p_repeat, gap_mean, p_swap, radius, _ptr(out))
    return out


def rootdups_f64(n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().lsg_rootdups_f64(n, _ptr(out))
    return out


def twodups_f64(n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().lsg_twodups_f64(n, _ptr(out))
    return out


def batch_sizes(count: int = 4096, seed: int = 6, median: float = 65536.0, sigma: float = 1.1,
                lo: int = 1024, hi: int = 4_194_304, ndist: int = 3):
    sizes = np.empty(count, np.uint64)
    dist = np.empty(count, np.int32)
    _L().lsg_batch_sizes(seed, count, median, sigma, lo, hi, ndist, _ptr(sizes), _ptr(dist))
    return sizes, dist


def batch_arrays(count: int = 4096, seed: int = 6, scale: float = 1.0, **kw):
    """The batched workload: `count` float64 arrays of lognormal sizes, each drawn
    from one of {N(0,1), U[0,1), Zipf(1.1) over 10^4 lognormal(0,2) values}.
    `scale` shrinks every size (for tests).  Returns a list of arrays."""
    sizes, dist = batch_sizes(count, seed, **kw)
    out = []
    for i in range(count):
        n = max(1, int(int(sizes[i]) * scale))
        s = seed * 1_000_003 + i + 1
        d = int(dist[i])
        if d == 0:
            out.append(normal_f64(n, s))
        elif d == 1:
            out.append(uniform_f64(n, s))
        else:
            out.append(zipf_lognormal_f64(n, s, k=10_000, s=1.1))
    return out


# The named workloads used by the benchmark and the full-size tests.
WORKLOADS = {
    "normal_1m_f64": ("f64", 1_000_000, lambda n: normal_f64(n, 0)),
    "zipf_lognormal_200m_f64": ("f64", 200_000_000, lambda n: zipf_lognormal_f64(n, 1)),
    "uniform_200m_u64": ("u64", 200_000_000, lambda n: uniform_u64(n, 2)),
    "gauss_mix_200m_f64": ("f64", 200_000_000, lambda n: gauss_mix_f64(n, 3)),
    "timestamp_200m_u32": ("u32", 200_000_000, lambda n: timestamp_u32(n - n % 1000, 4)),
    "exponential_200m_f32": ("f32", 200_000_000, lambda n: exponential_f32(n, 5)),
}

# The paper's synthetic suite (Sec. 6.1 data sets, Sec. 6.2 Zipf skew sweep,
# Sec. 6.4 scalability), as further named workloads.  The Zipfian sets draw
# ranks 1..10^6 by Zipf(s) weights (the paper does not state the support).
SUITE = {}
for _s in (0.50, 0.60, 0.70, 0.80, 0.90, 0.99):
    SUITE[f"zipf_s{int(round(_s * 100)):03d}_200m_f64"] = (
        "f64", 200_000_000, (lambda s: lambda n: zipf_rank_f64(n, 8, k=1_000_000, s=s))(_s))
SUITE["rootdups_200m_f64"] = ("f64", 200_000_000, lambda n: rootdups_f64(n))
SUITE["twodups_200m_f64"] = ("f64", 200_000_000, lambda n: twodups_f64(n))
for _tag, _n in (("1m", 1_000_000), ("10m", 10_000_000), ("100m", 100_000_000),
                 ("1b", 1_000_000_000)):
    SUITE[f"normal_{_tag}_f64"] = ("f64", _n, lambda n: normal_f64(n, 0))
    SUITE[f"twodups_{_tag}_f64"] = ("f64", _n, lambda n: twodups_f64(n))
WORKLOADS.update({k: v for k, v in SUITE.items() if k not in WORKLOADS})


def serving_pool(count: int = 64, seed: int = 7, lo: float = 1e4, hi: float = 6.4e7,
                 heavy_share: float = 0.3):
    """Request inputs of the serving workload: sizes log-uniform on [lo, hi],
    key type uniform over {float64, uint64, float32}; a `heavy_share` of them
    Zipf(1.3) over 1,000 lognormal values, the others drawn like the
    200M-key sweep (uniform / Gaussian mixture / exponential).  Returns a list
    of arrays."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        kind = int(rng.integers(0, 3))
        s = seed * 1_000_003 + i + 1
        if rng.uniform() < heavy_share:
            a = zipf_lognormal_f64(n, s, k=1000, s=1.3)
            a = a.astype(np.float32) if kind == 2 else a
            if kind == 1:
                a = (a * 1e6).astype(np.uint64)
        elif kind == 0:
            a = gauss_mix_f64(n, s)
        elif kind == 1:
            a = uniform_u64(n, s)
        else:
            a = exponential_f32(n, s)
        out.append(a)
    return out


def workload(name: str, n: int | None = None) -> np.ndarray:
    dt, n0, fn = WORKLOADS[name]
    return fn(n0 if n is None else n)
