"""GB300 (sm_103a) NN-Descent K-nearest-neighbour graphs for the squared l2
metric -- Python binding over the C ABI in include/knng.h.

Every step of the method runs in the CUDA kernels of libknng_gb300.so; this
module only marshals arguments (pointers, sizes, the CUDA stream) and
allocates result buffers with torch (device) or numpy (host).  The library
is loaded on first use, and any call fails loudly (ImportError) if it has not
been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "KnngError", "Stats", "Context", "knng_build", "knng_build_batched", "knng_build_batched_ex", "knng_bruteforce",
    "lib_path", "Desc", "DescEx",
    "bruteforce_last_fallbacks", "bruteforce_last_prefilter_ms", "measure_l2_read",
    "FLAG_REORDER", "FLAG_REORDER_B", "FLAG_TIMING", "FLAG_GRAPH", "FLAG_BF16", "FLAG_AUTOTUNE", "FLAG_HEAP_SAMPLING", "FLAG_REORDER_PARALLEL", "FLAG_FP8", "version", "strerror", "load",
]

FLAG_REORDER = 0x1
FLAG_REORDER_B = 0x2
FLAG_TIMING = 0x4
FLAG_GRAPH = 0x8
FLAG_BF16 = 0x10
FLAG_AUTOTUNE = 0x20
FLAG_HEAP_SAMPLING = 0x40
FLAG_REORDER_PARALLEL = 0x80
FLAG_FP8 = 0x100

OK = 0
WARN_OVERFLOW = 1


class KnngError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("K", ctypes.c_int32), ("s", ctypes.c_int32),
        ("iterations", ctypes.c_int32), ("dist_evals", ctypes.c_int64), ("last_changes", ctypes.c_int64),
        ("inserts", ctypes.c_int64), ("merges", ctypes.c_int64), ("gathered_rows", ctypes.c_int64),
        ("rev_overflow", ctypes.c_int64), ("set_overflow", ctypes.c_int64),
        ("lock_timeouts", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
        ("cand_ids", ctypes.c_int64), ("proposals", ctypes.c_int64), ("bucket_overflow", ctypes.c_int64), ("reordered", ctypes.c_int32),
        ("join_launches", ctypes.c_int32), ("join_ms", ctypes.c_double), ("join_ran", ctypes.c_int32),
        ("join_path", ctypes.c_int32), ("join_ms_ran", ctypes.c_double), ("merge_ms_ran", ctypes.c_double),
        ("sample_ms_ran", ctypes.c_double), ("reorder_ms", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Desc(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("ids", ctypes.c_void_p), ("dists", ctypes.c_void_p)]


class DescEx(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("K", ctypes.c_int32),
                ("rho", ctypes.c_float), ("delta", ctypes.c_float), ("max_iters", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("ids", ctypes.c_void_p), ("dists", ctypes.c_void_p)]


def lib_path() -> str:
    return _build.LIB


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -m paper_2112_06630_gb300.build)")
    lib = ctypes.CDLL(path)
    P, i64, i32, u32, u64, f32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_float)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "knng_build": (i32, [P, i64, i32, i32, f32, f32, i32, u64, P, P]),
        "knng_build_ex": (i32, [P, i64, i32, i32, f32, f32, i32, u64, u32, P, P, P, P]),
        "knng_init": (i32, [PP, P, i64, i32, i32, f32, f32, u64, u32, P]),
        "knng_init_from_graph": (i32, [PP, P, i64, i32, i32, f32, f32, u64, u32, P, P, P, i32]),
        "knng_iterate": (i32, [P, P]),
        "knng_run": (i32, [P, i32]),
        "knng_reorder": (i32, [P]),
        "knng_get": (i32, [P, P, P]),
        "knng_get_state": (i32, [P, P, P, P]),
        "knng_get_samples": (i32, [P, i32, P, P, P, P]),
        "knng_get_permutation": (i32, [P, P]),
        "knng_get_stats": (i32, [P, P]),
        "knng_destroy": (i32, [P]),
        "knng_bruteforce": (i32, [P, i64, i32, i32, P, i64, P, P, P]),
        "knng_bruteforce_last_fallbacks": (i32, []),
        "knng_bruteforce_last_prefilter_ms": (f32, []),
        "knng_measure_l2_read": (i32, [i64, i32, P, ctypes.POINTER(ctypes.c_double)]),
        "knng_build_batched": (i32, [P, i32, i32, f32, f32, i32, u64, u32, P, P]),
        "knng_build_batched_ex": (i32, [P, i32, u32, P, P]),
        "knng_strerror": (ctypes.c_char_p, [i32]),
        "knng_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class _LazyLib:
    """Loads the shared library on first use; raises ImportError if it is
    missing (there is no fallback path)."""

    def __init__(self):
        self._lib = None

    def __getattr__(self, name):
        if self._lib is None:
            self._lib = _load()
        return getattr(self._lib, name)


_lib = _LazyLib()


def load():
    """Load (and return) the shared library now."""
    _lib.knng_version
    return _lib._lib


def strerror(code: int) -> str:
    return _lib.knng_strerror(int(code)).decode()


def version() -> str:
    return _lib.knng_version().decode()


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise KnngError(rc, where)
    return rc


# ------------------------------------------------------------ marshalling ----

def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _as_input(data):
    """(pointer, keepalive, n, d, on_device) for a float32 row-major matrix."""
    if _is_torch(data):
        import torch
        t = data
        if t.dtype != torch.float32 or t.dim() != 2:
            raise ValueError("data must be a 2-D float32 tensor")
        t = t.contiguous()
        return t.data_ptr(), t, t.shape[0], t.shape[1], t.is_cuda
    a = np.ascontiguousarray(data, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("data must be 2-D")
    return a.ctypes.data, a, a.shape[0], a.shape[1], False


def _stream_ptr(stream, on_device):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if on_device:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return 0


def _outputs(n, K, on_device, like=None):
    if on_device:
        import torch
        dev = like.device if like is not None else "cuda"
        ids = torch.empty((n, K), dtype=torch.int32, device=dev)
        dists = torch.empty((n, K), dtype=torch.float32, device=dev)
        return ids, dists, ids.data_ptr(), dists.data_ptr()
    ids = np.empty((n, K), np.int32)
    dists = np.empty((n, K), np.float32)
    return ids, dists, ids.ctypes.data, dists.ctypes.data


def knng_build(data, K: int, rho: float = 1.0, delta: float = 0.001, max_iters: int = 10,
               seed: int = 0, flags: int = 0, stream=None, out=None):
    """K-NNG by NN-Descent.  `data` (n, d) float32: a CUDA tensor gives CUDA
    outputs on the caller's stream; a host array gives host outputs.  Returns
    (ids, dists, stats_dict)."""
    ptr, keep, n, d, dev = _as_input(data)
    if out is not None:
        ids, dists = out
        ip = ids.data_ptr() if _is_torch(ids) else ids.ctypes.data
        dp = dists.data_ptr() if _is_torch(dists) else dists.ctypes.data
    else:
        ids, dists, ip, dp = _outputs(n, K, dev, keep if dev else None)
    st = Stats()
    rc = _lib.knng_build_ex(ptr, n, d, K, rho, delta, max_iters, seed, flags, _stream_ptr(stream, dev),
                            ip, dp, ctypes.byref(st))
    _check(rc, "knng_build_ex")
    info = st.as_dict()
    info["overflow_warning"] = rc == WARN_OVERFLOW
    return ids, dists, info


def knng_build_batched(datasets, K: int, rho: float = 1.0, delta: float = 0.001, max_iters: int = 10,
                       seed: int = 0, flags: int = 0, stream=None):
    """K-NNGs of many independent data sets in one run (one launch per step
    for all of them).  `datasets`: sequence of (n_b, d_b) float32 arrays or
    CUDA tensors.  Returns ([(ids, dists) per data set], stats_dict)."""
    keep, outs = [], []
    descs = (Desc * len(datasets))()
    dev_any = False
    for b, data in enumerate(datasets):
        ptr, k, n, d, dev = _as_input(data)
        dev_any = dev_any or dev
        ids, dists, ip, dp = _outputs(n, K, dev, k if dev else None)
        keep.append(k)
        outs.append((ids, dists))
        descs[b] = Desc(ptr, n, d, ip, dp)
    st = Stats()
    rc = _lib.knng_build_batched(ctypes.addressof(descs), len(datasets), K, rho, delta, max_iters, seed, flags,
                                 _stream_ptr(stream, dev_any), ctypes.byref(st))
    _check(rc, "knng_build_batched")
    info = st.as_dict()
    info["overflow_warning"] = rc == WARN_OVERFLOW
    return outs, info


def knng_build_batched_ex(items, flags: int = 0, stream=None):
    """knng_build_batched with parameters per data set.  `items`: sequence of
    dicts with keys data (an (n_b, d_b) float32 array or CUDA tensor), K, rho,
    delta, max_iters and seed.  Returns ([(ids, dists) per data set],
    stats_dict)."""
    keep, outs = [], []
    descs = (DescEx * len(items))()
    dev_any = False
    for b, it in enumerate(items):
        ptr, k, n, d, dev = _as_input(it["data"])
        dev_any = dev_any or dev
        K = int(it["K"])
        ids, dists, ip, dp = _outputs(n, K, dev, k if dev else None)
        keep.append(k)
        outs.append((ids, dists))
        descs[b] = DescEx(ptr, n, d, K, float(it["rho"]), float(it["delta"]), int(it["max_iters"]),
                          int(it["seed"]), ip, dp)
    st = Stats()
    rc = _lib.knng_build_batched_ex(ctypes.addressof(descs), len(items), flags, _stream_ptr(stream, dev_any),
                                    ctypes.byref(st))
    _check(rc, "knng_build_batched_ex")
    info = st.as_dict()
    info["overflow_warning"] = rc == WARN_OVERFLOW
    return outs, info


def knng_bruteforce(data, K: int, rows=None, stream=None):
    """Exact K-NNG rows (all rows, or the given query ids)."""
    ptr, keep, n, d, dev = _as_input(data)
    rp, rkeep, nq = 0, None, n
    if rows is not None:
        if _is_torch(rows):
            rkeep = rows.to(dtype=__import__("torch").int64).contiguous()
            rp = rkeep.data_ptr()
        else:
            rkeep = np.ascontiguousarray(rows, dtype=np.int64)
            rp = rkeep.ctypes.data
        nq = int(rkeep.shape[0])
    ids, dists, ip, dp = _outputs(nq, K, dev, keep if dev else None)
    _check(_lib.knng_bruteforce(ptr, n, d, K, rp, nq, ip, dp, _stream_ptr(stream, dev)), "knng_bruteforce")
    return ids, dists


def bruteforce_last_fallbacks() -> int:
    """Queries of this thread's last knng_bruteforce that the tensor-core
    prefilter could not certify (recomputed exactly); -1 if it did not run."""
    return int(_lib.knng_bruteforce_last_fallbacks())


def bruteforce_last_prefilter_ms() -> float:
    """CUDA-event time of this thread's last tensor-core prefilter kernel in
    milliseconds; -1 if the last knng_bruteforce did not take that path."""
    return float(_lib.knng_bruteforce_last_prefilter_ms())


def measure_l2_read(nbytes: int = 32 << 20, passes: int = 200, stream=None) -> float:
    """GB/s at which the GPU reads an L2-resident buffer (one launch, 16-byte
    loads cached in L2 only)."""
    out = ctypes.c_double(0.0)
    _check(_lib.knng_measure_l2_read(nbytes, passes, _stream_ptr(stream, True), ctypes.byref(out)),
           "knng_measure_l2_read")
    return float(out.value)


class Context:
    """Step-by-step NN-Descent (knng_init / knng_iterate / knng_get ...)."""

    def __init__(self, data, K: int, rho: float = 1.0, delta: float = 0.001, seed: int = 0,
                 flags: int = 0, stream=None, graph=None, iter: int = 0):
        ptr, self._keep, self.n, self.d, self._dev = _as_input(data)
        self.K = K
        self._stream = _stream_ptr(stream, self._dev)
        h = ctypes.c_void_p()
        if graph is None:
            rc = _lib.knng_init(ctypes.byref(h), ptr, self.n, self.d, K, rho, delta, seed, flags, self._stream)
        else:
            gids = np.ascontiguousarray(graph[0], dtype=np.int32)
            gnew = np.ascontiguousarray(graph[1], dtype=np.uint8)
            rc = _lib.knng_init_from_graph(ctypes.byref(h), ptr, self.n, self.d, K, rho, delta, seed, flags,
                                           self._stream, gids.ctypes.data, gnew.ctypes.data, iter)
        _check(rc, "knng_init")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.knng_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def iterate(self):
        """One iteration; returns (converged, changes)."""
        ch = ctypes.c_int64()
        rc = _check(_lib.knng_iterate(self._h, ctypes.byref(ch)), "knng_iterate")
        return rc == 1, ch.value

    def run(self, max_iters: int):
        _check(_lib.knng_run(self._h, max_iters), "knng_run")

    def reorder(self):
        _check(_lib.knng_reorder(self._h), "knng_reorder")

    def get(self, device: bool | None = None):
        dev = self._dev if device is None else device
        ids, dists, ip, dp = _outputs(self.n, self.K, dev, self._keep if (dev and self._dev) else None)
        _check(_lib.knng_get(self._h, ip, dp), "knng_get")
        return ids, dists

    def state(self):
        ids = np.empty((self.n, self.K), np.int32)
        dists = np.empty((self.n, self.K), np.float32)
        flags = np.empty((self.n, self.K), np.uint8)
        _check(_lib.knng_get_state(self._h, ids.ctypes.data, dists.ctypes.data, flags.ctypes.data),
               "knng_get_state")
        return ids, dists, flags

    def samples(self, cap: int = 256):
        """Raw sampled candidates of the last iteration: (new, old) lists of
        arrays, forward part first, repeats not removed."""
        n = self.n
        ni = np.empty((n, cap), np.int32); nc = np.empty(n, np.int32)
        oi = np.empty((n, cap), np.int32); oc = np.empty(n, np.int32)
        _check(_lib.knng_get_samples(self._h, cap, ni.ctypes.data, nc.ctypes.data, oi.ctypes.data,
                                     oc.ctypes.data), "knng_get_samples")
        return [ni[u, :nc[u]].copy() for u in range(n)], [oi[u, :oc[u]].copy() for u in range(n)]

    def permutation(self):
        sg = np.empty(self.n, np.int32)
        _check(_lib.knng_get_permutation(self._h, sg.ctypes.data), "knng_get_permutation")
        return sg

    def stats(self) -> dict:
        st = Stats()
        _check(_lib.knng_get_stats(self._h, ctypes.byref(st)), "knng_get_stats")
        return st.as_dict()
