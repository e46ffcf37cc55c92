"""Write tests/golden/oracle_recall.json: the oracle's NN-Descent recall@K on
the full-size workloads, for the parity tests that compare the GPU build's
recall against it (the two must be within 0.005 at the same rho, delta,
iteration cap and seed).

Calls only `oracle` (the batched build on every host core, the exact
brute-force rows, the tie-aware recall) and `workloads` (the seeded inputs);
nothing here touches the CUDA library.  The oracle's arithmetic is plain
IEEE double in a fixed order (no fused multiply-add), so the numbers are the
same on any host; each record carries a checksum of its input and of the
oracle sources it came from, which the tests compare before using it.

    python tests/golden/make_oracle_recall.py [name ...]

Recall rows: RECALL_ROWS rows drawn with numpy's PCG64 seeded ROWS_SEED
(`recall_rows` in the tests).  Several hours of CPU time in total on eight
cores; each case is written as soon as it is done.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

OUT = os.path.join(HERE, "oracle_recall.json")
RECALL_ROWS = 2000
ROWS_SEED = 7

# name: (workload, rho, delta, max_iters) -- the stated parameters of each
# workload, and the 1M x 128 mixture's recall-0.99 operating point
CASES = {
    "mixture_n1m_d128": ("mixture_n1m_d128", 0.3, 0.001, 12),
    "mixture_n1m_d128_rho0.7_delta0.001_iters12": ("mixture_n1m_d128", 0.7, 0.001, 12),
    "mnist_like_n70k_d784": ("mnist_like_n70k_d784", 0.5, 0.001, 15),
    "audio_like_n54k_d192": ("audio_like_n54k_d192", 0.5, 0.001, 15),
    "clustered_n100k_d16": ("clustered_n100k_d16", 0.5, 0.001, 15),
    "clustered_n100k_d16_rho0.55_delta0.001_iters15": ("clustered_n100k_d16", 0.55, 0.001, 15),
}


def recall_rows(n: int) -> np.ndarray:
    return np.sort(np.random.Generator(np.random.PCG64(ROWS_SEED)).choice(n, RECALL_ROWS, replace=False))


def data_checksum(x: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(x, dtype=np.float32).tobytes()).hexdigest()[:16]


def oracle_sources_sha() -> str:
    h = hashlib.sha256()
    for f in ("knng_oracle.c", "metrics.py"):
        h.update(open(os.path.join(ROOT, "oracle", f), "rb").read())
    return h.hexdigest()[:16]


def _exact_rows(args):
    name, rows = args
    import oracle
    import workloads
    x = workloads.WORKLOADS[name].data()
    return oracle.bruteforce(x, workloads.WORKLOADS[name].K, rows=rows)[0]


def exact_ids(wname: str, rows: np.ndarray, procs: int) -> np.ndarray:
    parts = np.array_split(rows, procs)
    with mp.get_context("spawn").Pool(procs) as pool:
        out = pool.map(_exact_rows, [(wname, p) for p in parts])
    return np.concatenate(out, axis=0)


def main(names):
    import oracle
    import workloads
    from oracle import metrics

    db = json.load(open(OUT)) if os.path.exists(OUT) else {}
    procs = min(8, os.cpu_count() or 1)
    exact_cache = {}
    for name in names:
        wname, rho, delta, iters = CASES[name]
        w = workloads.WORKLOADS[wname]
        x = w.data()
        rows = recall_rows(w.n)
        if wname not in exact_cache:
            t0 = time.time()
            exact_cache[wname] = exact_ids(wname, rows, procs)
            print(f"{wname}: exact rows in {time.time() - t0:.0f} s", flush=True)
        t0 = time.time()
        ids, _, st = oracle.build_knng_mt(x, w.K, rho, delta, iters, seed=0)
        secs = time.time() - t0
        rec = metrics.recall(x, ids, exact_cache[wname], rows)
        db[name] = {
            "workload": wname, "n": w.n, "d": w.d, "K": w.K, "rho": rho, "delta": delta, "max_iters": iters,
            "seed": 0, "recall_at_k": rec, "recall_rows": RECALL_ROWS, "rows_seed": ROWS_SEED,
            "iterations": st["iters"], "dist_evals": st["evals"], "last_changes": st["last_changes"],
            "data_sha256_16": data_checksum(x), "oracle_sha256_16": oracle_sources_sha(),
            "oracle_seconds": round(secs, 1), "oracle_threads": st["threads"],
        }
        print(name, json.dumps(db[name]), flush=True)
        json.dump(db, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
