"""Evaluation helpers on the CPU (numpy, float64): recall, graph invariants,
window purity.  Test and benchmark infrastructure, not part of the library.

Recall (Section 2: how close the approximate K-NNG is to the exact one) is
taken tie-aware: an approximate neighbour of u counts as a hit when its exact
squared distance is at most the exact K-th smallest squared distance of u
(relative slack 1e-6), so that equally distant points are interchangeable.
"""
from __future__ import annotations

import numpy as np


def _chunks(n: int, step: int):
    for a in range(0, n, step):
        yield a, min(n, a + step)


def sqdist64(data: np.ndarray, rows: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """float64 squared l2 between data[rows[i]] and data[ids[i, k]]."""
    x = np.asarray(data, dtype=np.float64)
    out = np.empty(ids.shape, dtype=np.float64)
    step = max(1, (1 << 24) // max(1, ids.shape[1] * x.shape[1]))
    for a, b in _chunks(len(rows), step):
        diff = x[ids[a:b]] - x[rows[a:b]][:, None, :]
        out[a:b] = np.einsum("ikd,ikd->ik", diff, diff)
    return out


def recall(data, approx_ids, exact_ids, rows=None, rtol: float = 1e-6) -> float:
    """Tie-aware recall@K of approx_ids[rows] against exact_ids (one row per
    entry of `rows`; rows=None means all rows in order)."""
    approx_ids = np.asarray(approx_ids)
    exact_ids = np.asarray(exact_ids)
    if rows is None:
        rows = np.arange(exact_ids.shape[0])
    rows = np.asarray(rows, dtype=np.int64)
    K = exact_ids.shape[1]
    a = approx_ids[rows]
    dk = sqdist64(data, rows, exact_ids).max(axis=1)
    da = sqdist64(data, rows, a)
    hits = (da <= dk[:, None] * (1.0 + rtol) + 1e-30)
    # recall is a set measure: a repeated id is one neighbour, so every copy of
    # an id after its first is dropped, whether that id is a hit or a miss
    order = np.argsort(a, axis=1, kind="stable")
    srt = np.take_along_axis(a, order, axis=1)
    dup_sorted = np.zeros(a.shape, dtype=bool)
    dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
    dup = np.empty_like(dup_sorted)
    np.put_along_axis(dup, order, dup_sorted, axis=1)
    return float((hits & ~dup).sum()) / float(len(rows) * K)


def check_graph(data, ids, dists, rtol: float = 1e-4, atol: float = 1e-6, rows=None):
    """Invariants of a returned K-NNG: no self-loop, no repeated id, rows sorted
    ascending by (dist, id), every dist within rtol of its float64 recomputation
    (atol where that value is 0).  Returns a list of problems (empty if none)."""
    ids = np.asarray(ids)
    dists = np.asarray(dists)
    n = ids.shape[0]
    if rows is None:
        rows = np.arange(n)
    rows = np.asarray(rows)
    I, D = ids[rows], dists[rows]
    probs = []
    if (I == rows[:, None]).any():
        probs.append("self-loop")
    if (I < 0).any() or (I >= np.asarray(data).shape[0]).any():
        probs.append("id out of range")
        return probs
    srt = np.sort(I, axis=1)
    if (srt[:, 1:] == srt[:, :-1]).any():
        probs.append("repeated id")
    d0, d1 = D[:, :-1], D[:, 1:]
    i0, i1 = I[:, :-1], I[:, 1:]
    if ((d1 < d0) | ((d1 == d0) & (i1 < i0))).any():
        probs.append("not sorted by (dist, id)")
    ref = sqdist64(data, rows, I)
    err = np.abs(D.astype(np.float64) - ref)
    bad = np.where(ref > 0, err > rtol * ref, err > atol)
    if bad.any():
        probs.append(f"distance off: max rel err {float((err / np.maximum(ref, 1e-300)).max()):.3g}")
    return probs


def window_purity(labels_in_order: np.ndarray, window: int, clusters: int):
    """Fraction of the most frequent cluster in each window of `window`
    consecutive spots (the measure plotted for the greedy heuristic in
    Section 4, 'Greedy Clustering Heuristic Evaluation')."""
    lab = np.asarray(labels_in_order)
    out = []
    for a in range(0, len(lab) - window + 1, window):
        cnt = np.bincount(lab[a:a + window], minlength=clusters)
        out.append(cnt.max() / window)
    return np.array(out)
