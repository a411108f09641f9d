"""CPU oracle for the learned-sort hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it shares
no code, header, table or helper with the CUDA library.

``lso.cpp`` is a plain, slow C++ LearnedSort 2.0 written from Alg. 1
(Partition) and Alg. 2 (LearnedSort) of Kristo, Vaidya, Kraska (arXiv
2107.03290), in FP64, plus the plain definition of the result
(``reference_sort``: std::sort by IEEE total order) and spec functions that
restate the GPU kernels' documented per-key arithmetic.

Parity pins (tests/test_oracle.py): the output equals std::sort on every input
and on every permutation of small multisets; the sample formula, the fit and
the partition invariants are checked against closed forms.  The FP32 spec
functions are pinned by monotonicity and by agreement with the FP64 model
within FP32 rounding; their exact bit patterns are "parity unpinned" (they
restate a design of this project, not a formula printed in the paper).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lso.cpp")
_HDR = os.path.join(_HERE, "lso.h")
_SO = os.path.join(_HERE, "_lso.so")
_lib = None
_lock = threading.Lock()

DTYPES = {"f64": 0, "u64": 1, "f32": 2, "u32": 3}
NP_DTYPES = {"f64": np.float64, "u64": np.uint64, "f32": np.float32, "u32": np.uint32}


def dtype_name(a: np.ndarray) -> str:
    for k, v in NP_DTYPES.items():
        if a.dtype == np.dtype(v):
            return k
    raise TypeError(f"unsupported dtype {a.dtype}")


def build(force: bool = False) -> str:
    """Compile lso.cpp into _lso.so (plain g++, FP contraction off)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared",
                               "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("fanout", ctypes.c_uint32), ("leaves", ctypes.c_uint32),
                ("sample_div", ctypes.c_uint32), ("frag_cap", ctypes.c_uint32),
                ("sample_max", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("n_small", ctypes.c_uint64)]


class Trace(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "sample_size", "sample_finite", "l0_fragments", "l0_full_fragments", "homogeneous",
        "l1_partitions", "counting_sorts", "insertion_moves", "max_bucket")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Model(ctypes.Structure):
    _fields_ = [("leaves", ctypes.c_uint32), ("s", ctypes.c_uint64), ("s_fin", ctypes.c_uint64),
                ("root", ctypes.c_double * 3), ("leaf", ctypes.POINTER(ctypes.c_double))]


class Eval(ctypes.Structure):
    _fields_ = [("model", ctypes.POINTER(Model)), ("f0", ctypes.c_uint32)]


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, u64, i32, u32, i64 = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_uint32, ctypes.c_int64)
            P = ctypes.POINTER
            lib.lso_default_params.argtypes = [P(Params)]
            lib.lso_sort.argtypes = [vp, u64, i32, P(Params), P(Trace)]
            lib.lso_sort.restype = i32
            lib.lso_sort_stages.argtypes = [vp, u64, i32, P(Params), P(Model), i32, P(Trace)]
            lib.lso_sort_stages.restype = i32
            lib.lso_reference_argsort.argtypes = [vp, u64, i32, vp]
            lib.lso_reference_argsort.restype = i32
            lib.lso_reference_sort.argtypes = [vp, u64, i32]
            lib.lso_reference_sort.restype = i32
            lib.lso_total_order_key.argtypes = [vp, u64, i32]
            lib.lso_total_order_key.restype = u64
            lib.lso_sample_size.argtypes = [u64, P(Params)]
            lib.lso_sample_size.restype = u64
            lib.lso_sample_indices.argtypes = [u64, u64, u64, vp]
            lib.lso_train.argtypes = [vp, u64, i32, P(Params), P(Model)]
            lib.lso_train.restype = i32
            lib.lso_fit_sorted.argtypes = [vp, vp, u64, u32, P(Model)]
            lib.lso_predict.argtypes = [P(Model), ctypes.c_double, i32, i32]
            lib.lso_predict.restype = ctypes.c_double
            lib.lso_partition_f64.argtypes = [vp, u64, P(Model), i32, u32, u32, u64, vp, vp, vp,
                                              u64]
            lib.lso_partition_f64.restype = u64
            lib.lso_defragment_f64.argtypes = [vp, u64, u32, vp, vp, vp, u64]
            lib.lso_spec_thresholds.argtypes = [P(Eval), i32, vp, vp]
            lib.lso_spec_bucket.argtypes = [P(Eval), vp, u64, i32]
            lib.lso_spec_bucket.restype = u32
            lib.lso_spec_heavy.argtypes = [vp, vp, u64, i32, u64, u32, P(Eval), vp, u64]
            lib.lso_spec_heavy.restype = u64
            lib.lso_spec_ext_histogram.argtypes = [P(Eval), vp, u64, i32, vp, u64, vp, u64]
            lib.lso_spec_ext_histogram.restype = u64
            _lib = lib
    return _lib


def params(**kw) -> Params:
    p = Params()
    _L().lso_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def learned_sort(keys: np.ndarray, p: Params | None = None, trace: bool = False):
    """LearnedSort 2.0 (Alg. 2) on a copy of `keys`; returns the sorted copy
    (and the trace dict if `trace`)."""
    a = np.ascontiguousarray(keys).copy()
    tr = Trace()
    rc = _L().lso_sort(_ptr(a), a.size, DTYPES[dtype_name(a)], ctypes.byref(p or params()),
                       ctypes.byref(tr))
    if rc != 0:
        raise RuntimeError("lso_sort failed")
    return (a, tr.as_dict()) if trace else a


def sort_stages(keys: np.ndarray, p: Params | None = None, model: "FittedModel | None" = None,
                touch_up: bool = True):
    """Alg. 2 on a copy of `keys` with an optional given model and, with
    touch_up=False, without the closing insertion sort.  Returns (array, trace)."""
    a = np.ascontiguousarray(keys).copy()
    tr = Trace()
    rc = _L().lso_sort_stages(_ptr(a), a.size, DTYPES[dtype_name(a)], ctypes.byref(p or params()),
                              ctypes.byref(model.m) if model is not None else None,
                              int(touch_up), ctypes.byref(tr))
    if rc != 0:
        raise RuntimeError("lso_sort_stages failed")
    return a, tr.as_dict()


def reference_sort(keys: np.ndarray) -> np.ndarray:
    """The plain definition: keys in ascending total order (std::sort)."""
    a = np.ascontiguousarray(keys).copy()
    _L().lso_reference_sort(_ptr(a), a.size, DTYPES[dtype_name(a)])
    return a


def reference_argsort(keys: np.ndarray) -> np.ndarray:
    """The plain definition of the stable argsort (std::stable_sort of the
    positions by total order); uint32 positions."""
    a = np.ascontiguousarray(keys)
    perm = np.empty(a.size, np.uint32)
    _L().lso_reference_argsort(_ptr(a), a.size, DTYPES[dtype_name(a)], _ptr(perm))
    return perm


def total_order_keys(keys: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(keys)
    d = DTYPES[dtype_name(a)]
    f = _L().lso_total_order_key
    return np.array([f(_ptr(a), i, d) for i in range(a.size)], dtype=np.uint64)


def sample_size(n: int, p: Params | None = None) -> int:
    return int(_L().lso_sample_size(n, ctypes.byref(p or params())))


def sample_indices(n: int, s: int, seed: int = 0) -> np.ndarray:
    out = np.empty(s, np.uint64)
    _L().lso_sample_indices(n, s, seed, _ptr(out))
    return out


class FittedModel:
    """An FP64 RMI: root (a, c, b) and L leaves (a, c, b, lo, hi)."""

    def __init__(self, leaves: int):
        self.buf = np.zeros(5 * leaves, np.float64)
        self.m = Model()
        self.m.leaves = leaves
        self.m.leaf = self.buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    @property
    def root(self):
        return np.array(list(self.m.root))

    @property
    def leaf(self):
        return self.buf.reshape(-1, 5)

    def predict(self, x: float) -> float:
        import math
        nan = math.isnan(x)
        return _L().lso_predict(ctypes.byref(self.m), x, int(nan),
                                int(nan and math.copysign(1.0, x) < 0))


def train(keys: np.ndarray, p: Params | None = None) -> FittedModel:
    p = p or params()
    a = np.ascontiguousarray(keys)
    fm = FittedModel(p.leaves)
    _L().lso_train(_ptr(a), a.size, DTYPES[dtype_name(a)], ctypes.byref(p), ctypes.byref(fm.m))
    return fm


def fit_sorted(xs: np.ndarray, leaves: int) -> FittedModel:
    """Fit on finite doubles sorted ascending (total order of the values)."""
    xs = np.ascontiguousarray(xs, np.float64)
    tk = total_order_keys(xs)
    fm = FittedModel(leaves)
    _L().lso_fit_sorted(_ptr(xs), _ptr(tk), xs.size, leaves, ctypes.byref(fm.m))
    return fm


def partition(a: np.ndarray, model: FittedModel, level: int, f: int, c: int, parent: int = 0):
    """Alg. 1 on a float64 copy; returns (array after Partition, S_B, owners, sizes)."""
    a = np.ascontiguousarray(a, np.float64).copy()
    sizes = np.zeros(f, np.uint64)
    mx = a.size + f + 1
    own = np.zeros(mx, np.uint64)
    sz = np.zeros(mx, np.uint64)
    nf = _L().lso_partition_f64(_ptr(a), a.size, ctypes.byref(model.m), level, f, c, parent,
                                _ptr(sizes), _ptr(own), _ptr(sz), mx)
    return a, sizes, own[:nf], sz[:nf]


def defragment(a: np.ndarray, f: int, sizes, owners, fsizes) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float64).copy()
    sizes = np.ascontiguousarray(sizes, np.uint64)
    owners = np.ascontiguousarray(owners, np.uint64)
    fsizes = np.ascontiguousarray(fsizes, np.uint64)
    _L().lso_defragment_f64(_ptr(a), a.size, f, _ptr(sizes), _ptr(owners), _ptr(fsizes),
                            owners.size)
    return a


class EvalParams:
    """The level-0 map's parameters: the FP64 model and the fan-out f0."""

    def __init__(self, model: "FittedModel", f0: int):
        self.model = model
        self.L = model.m.leaves
        self.f0 = f0

    def struct(self) -> Eval:
        e = Eval()
        e.model = ctypes.pointer(self.model.m)
        e.f0 = self.f0
        self._keep = e
        return e

    @classmethod
    def from_export(cls, m: dict, leaves: int, f0: int) -> "EvalParams":
        """From the GPU's exported FP64 model."""
        fm = FittedModel(leaves)
        fm.m.root[0], fm.m.root[1], fm.m.root[2] = [float(v) for v in m["root"]]
        fm.leaf[:] = m["leaf"][:leaves]
        return cls(fm, f0)


def spec_thresholds(ev: EvalParams, dtype: str):
    """Level-0 thresholds (f0 entries) and the bucket of the largest key."""
    thr = np.zeros(ev.f0, np.uint64)
    pm = np.zeros(1, np.uint32)
    _L().lso_spec_thresholds(ctypes.byref(ev.struct()), DTYPES[dtype], _ptr(thr), _ptr(pm))
    return thr, int(pm[0])


def spec_buckets(ev: EvalParams, keys: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(keys)
    d = DTYPES[dtype_name(a)]
    s = ev.struct()
    f = _L().lso_spec_bucket
    return np.array([f(ctypes.byref(s), _ptr(a), i, d) for i in range(a.size)], np.uint32)


def spec_heavy(sorted_keys: np.ndarray, tau: int, per_bucket: int, ev: EvalParams):
    a = np.ascontiguousarray(sorted_keys)
    tk = total_order_keys(a)
    out = np.zeros(max(1, a.size), np.uint64)
    s = ev.struct()
    nh = _L().lso_spec_heavy(_ptr(tk), _ptr(a), a.size, DTYPES[dtype_name(a)], tau, per_bucket,
                             ctypes.byref(s), _ptr(out), out.size)
    return out[:nh]


def spec_ext_histogram(ev: EvalParams, keys: np.ndarray, heavy_tk: np.ndarray):
    a = np.ascontiguousarray(keys)
    h = np.ascontiguousarray(heavy_tk, np.uint64)
    mx = ev.f0 + 2 * h.size + 1
    hist = np.zeros(mx, np.uint64)
    s = ev.struct()
    ne = _L().lso_spec_ext_histogram(ctypes.byref(s), _ptr(a), a.size, DTYPES[dtype_name(a)],
                                     _ptr(h), h.size, _ptr(hist), mx)
    return hist[:ne]
