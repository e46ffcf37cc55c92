"""CPU oracle for NN-Descent K-NNG construction (squared l2).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may use this package; the library under test never does.
It is a ctypes wrapper over `knng_oracle.c` (plain C, double-precision
accumulation, float32 decisions) plus numpy evaluation helpers in `metrics`.
It shares no code with the CUDA implementation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knng_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_knng.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add, so x86 and Arm hosts give the same
# double-precision sums.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle library in place (gcc); returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm", "-lpthread"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


P_ = ctypes.c_void_p
_i64, _i32, _u64, _f32t = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_float
# name -> (result type, argument types) of every exported oracle function
_SIGS = {
    "orc_hash": (_u64, [_u64, ctypes.c_uint32, ctypes.c_uint32, _u64, _u64]),
    "orc_dist64": (ctypes.c_double, [P_, P_, _i32]),
    "orc_bruteforce": (_i32, [P_, _i64, _i32, _i32, P_, P_]),
    "orc_bruteforce_rows": (_i32, [P_, _i64, _i32, _i32, P_, _i64, P_, P_]),
    "orc_create": (P_, [P_, _i64, _i32, _i32, _f32t, _u64]),
    "orc_init_random": (_i32, [P_]),
    "orc_init_graph": (_i32, [P_, P_, P_, _i32]),
    "orc_sample": (_i32, [P_, _i32, P_]),
    "orc_sample_heap": (_i32, [P_, _i32, P_]),
    "orc_set_sampler": (_i32, [P_, _i32]),
    "orc_join": (_i32, [P_, P_]),
    "orc_join_range": (_i32, [P_, _i64, _i64, P_]),
    "orc_iterate": (_i32, [P_, P_]),
    "orc_reorder": (_i32, [P_, _i32]),
    "orc_get_samples": (_i32, [P_, _i32, P_, P_, P_, P_]),
    "orc_set_samples": (_i32, [P_, _i32, P_, P_, P_, P_]),
    "orc_get_state": (_i32, [P_, P_, P_, P_]),
    "orc_get_graph": (_i32, [P_, P_, P_]),
    "orc_get_sigma": (_i32, [P_, P_]),
    "orc_free": (None, [P_]),
    "orc_greedy_reorder": (_i32, [P_, _i64, _i32, _i32, P_, P_]),
    "orc_parallel_relabel": (_i32, [P_, _i64, _i32, _i32, P_, _i32, P_, P_, P_, P_]),
    "orc_build": (_i32, [P_, _i64, _i32, _i32, _f32t, _f32t, _i32, _u64, _i32, _i32, _i32, P_, P_, P_]),
    "orc_build_mt": (_i32, [P_, _i64, _i32, _i32, _f32t, _f32t, _i32, _u64, _i32, P_, P_, P_]),
    "orc_default_threads": (_i32, []),
    "orc_set_mt_block_pairs": (_i32, [_i64]),
}


def _bind(lib):
    """Set the result and argument types of every oracle function on a loaded
    library (the built oracle, or a deliberately mutated copy in a test)."""
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(data) -> np.ndarray:
    return np.ascontiguousarray(data, dtype=np.float32)


STREAM_INIT, STREAM_FWD, STREAM_REV, STREAM_HEAP = 1, 2, 3, 4
SAMPLERS = {"turbo": 0, "heap": 1}


def hash64(seed: int, stream: int, it: int, u: int, j: int) -> int:
    return int(_load().orc_hash(seed, stream, it, u, j))


def dist64(x, y) -> float:
    x, y = _f32(x), _f32(y)
    return float(_load().orc_dist64(_p(x), _p(y), x.shape[-1]))


def sample_size(rho: float, K: int) -> int:
    """s = ceil(rho * K), clamped to [1, K] (same rule as the C code: rho as
    float32, with a tolerance that absorbs its rounding)."""
    import math
    return max(1, min(K, int(math.ceil(float(np.float32(rho)) * K - 1e-5))))


def bruteforce(data, K: int, rows=None):
    """Exact K-NNG (Section 2): ids (nq, K) int32, dists (nq, K) float32."""
    data = _f32(data)
    n, d = data.shape
    lib = _load()
    if rows is None:
        ids = np.empty((n, K), np.int32)
        dists = np.empty((n, K), np.float32)
        rc = lib.orc_bruteforce(_p(data), n, d, K, _p(ids), _p(dists))
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        ids = np.empty((len(rows), K), np.int32)
        dists = np.empty((len(rows), K), np.float32)
        rc = lib.orc_bruteforce_rows(_p(data), n, d, K, _p(rows), len(rows), _p(ids), _p(dists))
    if rc:
        raise ValueError(f"orc_bruteforce failed ({rc})")
    return ids, dists


def greedy_reorder(lists, reading_b: bool = False):
    """Algorithm 1 on sorted id lists (n, K): returns (sigma, sigma_inv)."""
    lists = np.ascontiguousarray(lists, dtype=np.int32)
    n, K = lists.shape
    sg = np.empty(n, np.int32)
    si = np.empty(n, np.int32)
    _load().orc_greedy_reorder(_p(lists), n, K, int(reading_b), _p(sg), _p(si))
    return sg, si


def parallel_relabel(data, lists, rmax: int = 64):
    """Parallel relabelling variant (single-linkage Boruvka rounds on the list
    graph).  Returns (levels (R, n) int32: each round's component
    representatives, msf_weight, sigma (n,) int32 with every component of
    every round contiguous)."""
    data = _f32(data)
    lists = np.ascontiguousarray(lists, dtype=np.int32)
    n, K = lists.shape
    levels = np.empty((rmax, n), np.int32)
    rounds = ctypes.c_int(0)
    w = ctypes.c_double(0.0)
    sg = np.empty(n, np.int32)
    rc = _load().orc_parallel_relabel(_p(data), n, data.shape[1], K, _p(lists), rmax, _p(levels),
                                      ctypes.byref(rounds), ctypes.byref(w), _p(sg))
    if rc:
        raise MemoryError("orc_parallel_relabel")
    return levels[:rounds.value].copy(), float(w.value), sg


def build_knng(data, K: int, rho: float, delta: float, max_iters: int, seed: int = 0,
               count_mode: str = "batched", reorder: int = 0, sampler: str = "turbo"):
    """Whole NN-Descent.  sampler: "turbo" (Section 3.1's one-pass
    probability sampling) or "heap" (priority heaps).  Returns (ids, dists,
    stats dict)."""
    data = _f32(data)
    n, d = data.shape
    ids = np.empty((n, K), np.int32)
    dists = np.empty((n, K), np.float32)
    st = np.zeros(4, np.int64)
    rc = _load().orc_build(_p(data), n, d, K, rho, delta, max_iters, seed,
                           1 if count_mode == "inplace" else 0, int(reorder), SAMPLERS[sampler],
                           _p(ids), _p(dists), _p(st))
    if rc:
        raise ValueError(f"orc_build failed ({rc})")
    return ids, dists, dict(iters=int(st[0]), evals=int(st[1]), last_changes=int(st[2]),
                            reordered=bool(st[3]))


def build_knng_mt(data, K: int, rho: float, delta: float, max_iters: int, seed: int = 0, threads: int = 0):
    """Whole NN-Descent in batched mode on `threads` host threads (0: every
    online core); the same lists as build_knng(count_mode="batched").
    Returns (ids, dists, stats dict with the threads used)."""
    data = _f32(data)
    n, d = data.shape
    ids = np.empty((n, K), np.int32)
    dists = np.empty((n, K), np.float32)
    st = np.zeros(5, np.int64)
    rc = _load().orc_build_mt(_p(data), n, d, K, rho, delta, max_iters, seed, int(threads), _p(ids), _p(dists),
                              _p(st))
    if rc:
        raise ValueError(f"orc_build_mt failed ({rc})")
    return ids, dists, dict(iters=int(st[0]), evals=int(st[1]), last_changes=int(st[2]), threads=int(st[4]))


def default_threads() -> int:
    """Host threads build_knng_mt uses by default (the online cores)."""
    return int(_load().orc_default_threads())


class State:
    """Step-by-step NN-Descent state (for step-level parity tests)."""

    def __init__(self, data, K: int, rho: float, seed: int = 0, sampler: str = "turbo"):
        self._data = _f32(data)
        self.n, self.d = self._data.shape
        self.K = K
        self.s = sample_size(rho, K)
        self.sampler = sampler
        self._lib = _load()
        self._h = self._lib.orc_create(_p(self._data), self.n, self.d, K, rho, seed)
        if not self._h:
            raise ValueError("orc_create: invalid arguments")
        self._lib.orc_set_sampler(self._h, SAMPLERS[sampler])

    def close(self):
        if self._h:
            self._lib.orc_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init_random(self):
        self._lib.orc_init_random(self._h)

    def init_graph(self, ids, is_new, it: int = 0):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        is_new = np.ascontiguousarray(is_new, dtype=np.uint8)
        if self._lib.orc_init_graph(self._h, _p(ids), _p(is_new), it):
            raise ValueError("orc_init_graph: invalid graph")

    def sample(self, it: int):
        st = np.zeros(3, np.int64)
        fn = self._lib.orc_sample_heap if self.sampler == "heap" else self._lib.orc_sample
        if fn(self._h, it, _p(st)):
            raise MemoryError
        return dict(max_rev_new=int(st[0]), max_rev_old=int(st[1]), max_cands=int(st[2]))

    def join(self):
        out = np.zeros(3, np.int64)
        self._lib.orc_join(self._h, _p(out))
        return dict(evals=int(out[0]), inserts=int(out[1]), changes=int(out[2]))

    def join_range(self, u0: int, u1: int):
        """Calculation step of nodes u0 <= u < u1 only (for timing a bounded
        share of an iteration): distance evaluations and insertions."""
        out = np.zeros(2, np.int64)
        self._lib.orc_join_range(self._h, int(u0), int(u1), _p(out))
        return dict(evals=int(out[0]), inserts=int(out[1]))

    def iterate(self):
        out = np.zeros(6, np.int64)
        if self._lib.orc_iterate(self._h, _p(out)):
            raise MemoryError
        return dict(evals=int(out[0]), inserts=int(out[1]), changes=int(out[2]),
                    max_rev_new=int(out[3]), max_rev_old=int(out[4]), max_cands=int(out[5]))

    def reorder(self, reading_b: bool = False):
        if self._lib.orc_reorder(self._h, int(reading_b)):
            raise MemoryError

    def samples(self, cap: int = 256):
        n = self.n
        ni = np.empty((n, cap), np.int32); nc = np.empty(n, np.int32)
        oi = np.empty((n, cap), np.int32); oc = np.empty(n, np.int32)
        self._lib.orc_get_samples(self._h, cap, _p(ni), _p(nc), _p(oi), _p(oc))
        return ([ni[u, :nc[u]].copy() for u in range(n)], [oi[u, :oc[u]].copy() for u in range(n)])

    def set_samples(self, new_sets, old_sets):
        n = self.n
        cap = max(1, max((len(x) for x in list(new_sets) + list(old_sets)), default=1))
        ni = np.full((n, cap), -1, np.int32); nc = np.zeros(n, np.int32)
        oi = np.full((n, cap), -1, np.int32); oc = np.zeros(n, np.int32)
        for u in range(n):
            nc[u] = len(new_sets[u]); ni[u, :nc[u]] = new_sets[u]
            oc[u] = len(old_sets[u]); oi[u, :oc[u]] = old_sets[u]
        self._lib.orc_set_samples(self._h, cap, _p(ni), _p(nc), _p(oi), _p(oc))

    def state(self):
        n, K = self.n, self.K
        ids = np.empty((n, K), np.int32); dists = np.empty((n, K), np.float32)
        flags = np.empty((n, K), np.uint8)
        self._lib.orc_get_state(self._h, _p(ids), _p(dists), _p(flags))
        return ids, dists, flags

    def graph(self):
        n, K = self.n, self.K
        ids = np.empty((n, K), np.int32); dists = np.empty((n, K), np.float32)
        self._lib.orc_get_graph(self._h, _p(ids), _p(dists))
        return ids, dists

    def sigma(self):
        sg = np.empty(self.n, np.int32)
        self._lib.orc_get_sigma(self._h, _p(sg))
        return sg
