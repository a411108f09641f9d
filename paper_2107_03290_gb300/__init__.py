"""GB300 learned sort: the LearnedSort 2.0 hot path (arXiv 2107.03290) in CUDA.

Thin ctypes binding over the C ABI of ``include/ls.h`` (``libls.so``, built
in-tree by ``build()``).  Every step of the sort runs in the library's CUDA
kernels; this module only marshals arguments.  PyTorch supplies device memory
and streams.  There is no CPU fallback: if the library is missing or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INC = os.path.join(os.path.dirname(_HERE), "include")
_SO = os.path.join(_HERE, "libls.so")
_BUILD = os.path.join(_HERE, "_build")
SOURCES = ["ls_train.cu", "ls_partition.cu", "ls_bucket.cu", "ls_api.cu", "ls_server.cpp",
           "ls_noalloc.cu", "ls_pairs.cu", "ls_inplace.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

DTYPE_CODES = {"f64": 0, "u64": 1, "f32": 2, "u32": 3}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
          4: "device wait timed out", 5: "busy", 6: "cancelled"}


class LsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA/C++ source for sm_103a and link ``libls.so`` in-tree."""
    os.makedirs(_BUILD, exist_ok=True)
    hdrs = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(_INC, "ls.h"))
    newest_hdr = max(os.path.getmtime(h) for h in hdrs)
    objs, jobs = [], []
    for src in SOURCES:
        sp = os.path.join(_CSRC, src)
        obj = os.path.join(_BUILD, src + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(
                os.path.getmtime(sp), newest_hdr):
            cmd = [_nvcc(), ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                   "-I", _INC, "-c", sp, "-o", obj]
            if src.endswith(".cpp"):
                cmd[1:1] = ["-x", "cu"]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)

    if jobs:
        with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            list(ex.map(run, jobs))
    if jobs or force or not os.path.exists(_SO):
        tmp = _SO + f".tmp{os.getpid()}"
        run([_nvcc(), ARCH, "-shared", "-o", tmp] + objs + ["-lcuda"])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("fanout", ctypes.c_uint32), ("leaves", ctypes.c_uint32),
                ("sample_div", ctypes.c_uint32), ("heavy_per_bucket", ctypes.c_uint32),
                ("sample_max", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("heavy_min_count", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 7)]


FLAG_NO_HEAVY = 1
FLAG_IN_PLACE = 2


class Stats(ctypes.Structure):
    _fields_ = ([(k, ctypes.c_double) for k in (
        "ms_total", "ms_train", "ms_hist", "ms_scan", "ms_scatter", "ms_classify", "ms_level1",
        "ms_fill", "ms_sort_small", "ms_sort_large", "ms_fallback")]
                + [("sample_size", ctypes.c_uint64), ("sample_finite", ctypes.c_uint64),
                   ("fanout", ctypes.c_uint32), ("leaves", ctypes.c_uint32)]
                + [(k, ctypes.c_uint64) for k in ("n_heavy", "n_ext", "max_bucket", "n_eq_keys",
                                                  "n_level1", "n_segments", "n_fallback",
                                                  "n_fill", "n_launches")]
                + [(k, ctypes.c_uint64) for k in ("n_fallback_keys", "max_fallback", "n_large_keys",
                                                  "n_range", "workspace_bytes")])

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ModelExport(ctypes.Structure):
    _fields_ = [("leaves", ctypes.c_uint32), ("max_heavy", ctypes.c_uint32),
                ("sample_size", ctypes.c_uint64), ("sample_finite", ctypes.c_uint64),
                ("root", ctypes.c_double * 3), ("leaf", ctypes.c_void_p),
                ("fanout", ctypes.c_uint32), ("pos_max", ctypes.c_uint32), ("thr", ctypes.c_void_p),
                ("sorted_sample_tk", ctypes.c_void_p), ("heavy_tk", ctypes.c_void_p),
                ("n_heavy", ctypes.c_uint64), ("tau", ctypes.c_uint64)]


class BatchParams(ctypes.Structure):
    _fields_ = [("split_target", ctypes.c_uint32 * 3), ("reserved", ctypes.c_uint32 * 5)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_queue", ctypes.c_uint32), ("streams", ctypes.c_uint32),
                ("debug_stall", ctypes.c_uint32), ("debug_spin_limit", ctypes.c_uint32),
                ("in_place", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 2)]


class RequestStats(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("status", ctypes.c_int)]


EXPORTED = ["ls_default_params", "ls_status_string", "ls_sort", "ls_sort_ex", "ls_sort_host",
            "ls_sort_batch", "ls_sort_batch_ex", "ls_argsort", "ls_sort_pairs", "ls_stream_status",
            "ls_debug_set_wait", "ls_train",
            "ls_level0_histogram",
            "ls_radix_sort_u64", "ls_radix_sort_u64_noalloc", "ls_sample_sort_u64",
            "ls_kernel_launches",
            "ls_server_create", "ls_server_submit", "ls_server_submit_from", "ls_server_wait",
            "ls_server_destroy", "ls_workspace_bytes"]

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _SO


def load(path: str | None = None):
    """Load libls.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _SO
        if not os.path.exists(p):
            raise RuntimeError(f"{p} not built: run paper_2107_03290_gb300.build()")
        lib = ctypes.CDLL(p)
        vp, sz, i32, u32, u64 = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32,
                                 ctypes.c_uint64)
        P = ctypes.POINTER
        lib.ls_default_params.argtypes = [P(Params)]
        lib.ls_status_string.argtypes = [i32]
        lib.ls_status_string.restype = ctypes.c_char_p
        lib.ls_kernel_launches.argtypes = []
        lib.ls_kernel_launches.restype = u64
        lib.ls_workspace_bytes.argtypes = [sz, i32, P(Params)]
        lib.ls_workspace_bytes.restype = sz
        for f, a in {
            "ls_sort": [vp, sz, i32, vp],
            "ls_sort_ex": [vp, sz, i32, vp, P(Params), P(Stats)],
            "ls_sort_host": [vp, sz, i32, vp, P(Params)],
            "ls_sort_batch": [vp, vp, sz, i32, vp],
            "ls_sort_batch_ex": [vp, vp, sz, i32, vp, P(BatchParams)],
            "ls_argsort": [vp, vp, sz, i32, vp],
            "ls_sort_pairs": [vp, vp, sz, i32, u32, vp],
            "ls_stream_status": [vp],
            "ls_debug_set_wait": [vp, u32, u64],
            "ls_train": [vp, sz, i32, vp, P(Params), P(ModelExport)],
            "ls_level0_histogram": [vp, sz, i32, vp, P(Params), vp, sz, P(ctypes.c_size_t)],
            "ls_radix_sort_u64": [vp, sz, vp],
            "ls_radix_sort_u64_noalloc": [vp, sz, vp],
            "ls_sample_sort_u64": [vp, sz, vp],
            "ls_server_create": [P(ServerConfig), P(vp)],
            "ls_server_submit": [vp, vp, sz, i32, P(u64)],
            "ls_server_submit_from": [vp, vp, vp, sz, i32, P(u64)],
            "ls_server_wait": [vp, u64, u32, P(RequestStats)],
            "ls_server_destroy": [vp],
        }.items():
            fn = getattr(lib, f)
            fn.argtypes = a
            fn.restype = i32
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise LsError(rc, what)


def default_params(**kw) -> Params:
    p = Params()
    load().ls_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    m = {torch.float64: 0, torch.uint64: 1, torch.float32: 2, torch.uint32: 3}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _stream(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _device_tensor(t):
    if not t.is_cuda:
        raise ValueError("keys must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("keys must be contiguous")
    return t


def sort_(t, params: Params | None = None, stats: bool = False, stream=None):
    """Sort a CUDA tensor in place (ls_sort_ex).  Returns stats dict if asked."""
    t = _device_tensor(t)
    st = Stats() if stats else None
    rc = load().ls_sort_ex(t.data_ptr(), t.numel(), dtype_code(t), _stream(stream),
                           ctypes.byref(params) if params is not None else None,
                           ctypes.byref(st) if st is not None else None)
    _check(rc, "ls_sort_ex")
    return st.as_dict() if st is not None else None


def workspace_bytes(n: int, code: int, params: Params | None = None) -> int:
    """Device workspace ls_sort_ex would allocate for n keys of dtype `code`."""
    return int(load().ls_workspace_bytes(n, code,
                                         ctypes.byref(params) if params is not None else None))


def sort(t, params: Params | None = None, stream=None):
    """Return a sorted copy of a CUDA tensor."""
    out = t.clone()
    sort_(out, params, stream=stream)
    return out


def sort_host(a: np.ndarray, params: Params | None = None, stream=None) -> np.ndarray:
    """End-to-end sort of a host array (copy in, sort, copy out); in place."""
    codes = {np.dtype(np.float64): 0, np.dtype(np.uint64): 1, np.dtype(np.float32): 2,
             np.dtype(np.uint32): 3}
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be contiguous")
    rc = load().ls_sort_host(a.ctypes.data, a.size, codes[a.dtype], _stream(stream),
                             ctypes.byref(params) if params is not None else None)
    _check(rc, "ls_sort_host")
    return a


def sort_host_ptr(ptr: int, n: int, code: int, params: Params | None = None, stream=None):
    rc = load().ls_sort_host(ptr, n, code, _stream(stream),
                             ctypes.byref(params) if params is not None else None)
    _check(rc, "ls_sort_host")


def sort_batch_(tensors, stream=None, split_target=None):
    """Sort many CUDA tensors of one dtype in place (ls_sort_batch; with
    split_target, a 3-tuple per array-size class, ls_sort_batch_ex)."""
    if not tensors:
        return
    code = dtype_code(tensors[0])
    ptrs = (ctypes.c_void_p * len(tensors))(*[_device_tensor(t).data_ptr() for t in tensors])
    ns = (ctypes.c_size_t * len(tensors))(*[t.numel() for t in tensors])
    if split_target is None:
        rc = load().ls_sort_batch(ptrs, ns, len(tensors), code, _stream(stream))
    else:
        bp = BatchParams()
        for i, v in enumerate(split_target):
            bp.split_target[i] = int(v)
        rc = load().ls_sort_batch_ex(ptrs, ns, len(tensors), code, _stream(stream), ctypes.byref(bp))
    _check(rc, "ls_sort_batch")


def argsort(t, stream=None):
    """Stable argsort of a CUDA tensor (ls_argsort): an int32 tensor whose
    entry r is the position of the key of rank r (as unsigned 32-bit)."""
    torch = _torch()
    t = _device_tensor(t)
    perm = torch.empty(t.numel(), dtype=torch.int32, device=t.device)
    _check(load().ls_argsort(t.data_ptr(), perm.data_ptr(), t.numel(), dtype_code(t),
                             _stream(stream)), "ls_argsort")
    return perm


def sort_pairs_(keys, values, stream=None):
    """Sort CUDA tensor `keys` in place and permute `values` (4- or 8-byte
    elements, same length) alongside, stably (ls_sort_pairs)."""
    keys = _device_tensor(keys)
    values = _device_tensor(values)
    if values.numel() != keys.numel():
        raise ValueError("values must have as many elements as keys")
    _check(load().ls_sort_pairs(keys.data_ptr(), values.data_ptr(), keys.numel(),
                                dtype_code(keys), values.element_size(), _stream(stream)),
           "ls_sort_pairs")


def kernel_launches() -> int:
    return load().ls_kernel_launches()


def stream_status(stream=None) -> int:
    """Status of the calls on `stream` since the last check (0: ok); clears it."""
    return load().ls_stream_status(_stream(stream))


def debug_set_wait(stall: int = 0, spin_limit: int = 0, stream=None):
    """Test hook (ls_debug_set_wait): bounded waits of later calls on `stream`
    give up after `spin_limit` polls; stall=1 makes the level-0 scan's waits
    run out.  (0, 0) restores normal calls."""
    _check(load().ls_debug_set_wait(_stream(stream), stall, spin_limit), "ls_debug_set_wait")


def radix_sort_u64_(t, stream=None):
    torch = _torch()
    if t.dtype != torch.uint64:
        raise TypeError("uint64 tensor expected")
    _check(load().ls_radix_sort_u64(_device_tensor(t).data_ptr(), t.numel(), _stream(stream)),
           "ls_radix_sort_u64")


def sample_sort_u64_(t, stream=None):
    """Sort a uint64 CUDA tensor in place with the training sample's sample sort
    (ls_sample_sort_u64)."""
    torch = _torch()
    if t.dtype != torch.uint64:
        raise TypeError("uint64 tensor expected")
    _check(load().ls_sample_sort_u64(_device_tensor(t).data_ptr(), t.numel(), _stream(stream)),
           "ls_sample_sort_u64")


NOALLOC_RADIX_MAX = 1 << 20
MAX_FANOUT = 4096


def radix_sort_u64_noalloc_(t, stream=None):
    """ls_radix_sort_u64 without any allocation (static device scratch, at most
    NOALLOC_RADIX_MAX keys); for callers that cannot allocate when they sort."""
    torch = _torch()
    if t.dtype != torch.uint64:
        raise TypeError("uint64 tensor expected")
    _check(load().ls_radix_sort_u64_noalloc(_device_tensor(t).data_ptr(), t.numel(),
                                            _stream(stream)), "ls_radix_sort_u64_noalloc")


def train(t, params: Params | None = None, stream=None, with_sample: bool = False) -> dict:
    """Run the training step only; returns the model as numpy arrays."""
    t = _device_tensor(t)
    p = params or default_params()
    L = p.leaves or 1000
    out = ModelExport()
    out.leaves = L
    out.fanout = MAX_FANOUT
    arr = {"leaf": np.zeros((L, 5), np.float64), "thr": np.zeros(MAX_FANOUT, np.uint64)}
    heavy = np.zeros(16 * MAX_FANOUT, np.uint64)
    out.max_heavy = heavy.size
    for k, v in arr.items():
        setattr(out, k, v.ctypes.data)
    out.heavy_tk = heavy.ctypes.data
    smp = None
    if with_sample:
        n = t.numel()
        smp = np.zeros(max(1, n), np.uint64)
        out.sorted_sample_tk = smp.ctypes.data
    rc = load().ls_train(t.data_ptr(), t.numel(), dtype_code(t), _stream(stream), ctypes.byref(p),
                         ctypes.byref(out))
    _check(rc, "ls_train")
    res = dict(arr)
    res["thr"] = arr["thr"][:out.fanout].copy()
    res.update(fanout=out.fanout, sample_size=out.sample_size, sample_finite=out.sample_finite,
               root=np.array(list(out.root)),
               heavy_tk=heavy[:out.n_heavy].copy(), tau=out.tau, pos_max=out.pos_max)
    if smp is not None:
        res["sorted_sample_tk"] = smp[:out.sample_size].copy()
    return res


def level0_histogram(t, params: Params | None = None, stream=None) -> np.ndarray:
    t = _device_tensor(t)
    p = params or default_params()
    mx = 65536
    h = np.zeros(mx, np.uint64)
    n_ext = ctypes.c_size_t(0)
    rc = load().ls_level0_histogram(t.data_ptr(), t.numel(), dtype_code(t), _stream(stream),
                                    ctypes.byref(p), h.ctypes.data, mx, ctypes.byref(n_ext))
    _check(rc, "ls_level0_histogram")
    return h[:n_ext.value].copy()


class Server:
    """Continuous-batching sort server (ls_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 120 << 30, max_inflight: int = 64,
                 max_queue: int = 4096, streams: int = 8, debug_stall: int = 0,
                 debug_spin_limit: int = 0, in_place: bool = False):
        cfg = ServerConfig(hbm_budget_bytes, max_inflight, max_queue, streams, debug_stall,
                           debug_spin_limit, 1 if in_place else 0)
        self._h = ctypes.c_void_p()
        _check(load().ls_server_create(ctypes.byref(cfg), ctypes.byref(self._h)),
               "ls_server_create")

    def submit(self, t, src=None) -> int:
        """Queue an in-place sort of CUDA tensor `t`; with `src` (a CUDA tensor of
        the same dtype and size) the server first copies `src` into `t`."""
        t = _device_tensor(t)
        tk = ctypes.c_uint64(0)
        if src is None:
            _check(load().ls_server_submit(self._h, t.data_ptr(), t.numel(), dtype_code(t),
                                           ctypes.byref(tk)), "ls_server_submit")
        else:
            src = _device_tensor(src)
            if src.numel() != t.numel() or src.dtype != t.dtype:
                raise ValueError("src must match t in dtype and size")
            _check(load().ls_server_submit_from(self._h, src.data_ptr(), t.data_ptr(), t.numel(),
                                                dtype_code(t), ctypes.byref(tk)),
                   "ls_server_submit_from")
        return tk.value

    def wait(self, ticket: int, timeout_ms: int = 0xFFFFFFFF, check: bool = True) -> dict:
        """Wait for a request; raises LsError on a failed request unless
        check=False (then the dict's "status" holds the code)."""
        st = RequestStats()
        rc = load().ls_server_wait(self._h, ticket, timeout_ms, ctypes.byref(st))
        if check:
            _check(rc, "ls_server_wait")
        return {"queue_ms": st.queue_ms, "device_ms": st.device_ms, "total_ms": st.total_ms,
                "status": rc}

    def close(self):
        if self._h:
            load().ls_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
