"""Pins for the evaluation helpers (oracle/metrics.py: recall, graph
invariants, window purity) and for the old-kind acceptance counts of the
oracle's selection step (Section 3.1).  Every case is built by hand with a
known answer, and each is chosen so that a plausible mistake fails it: a
recall that over-counts repeats or ignores ties, a graph check that reports
nothing, acceptance counts taken from the wrong counter.  The last tests plant
those counter mistakes in copies of the oracle compiled here, on the CPU, and
check that the pins catch them.  CPU only."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads
from oracle import metrics

ORACLE_SRC = os.path.join(os.path.dirname(oracle.__file__), "knng_oracle.c")


# -------------------------------------------------------------- recall ----

def _far_ids(x, u, exclude, count):
    """`count` ids farthest from u (float64), none of them in `exclude`."""
    d = ((x.astype(np.float64) - x[u].astype(np.float64)) ** 2).sum(1)
    order = np.argsort(-d, kind="stable")
    return [int(v) for v in order if v != u and v not in exclude][:count]


def test_recall_half_replaced_is_exactly_half():
    """Replacing the last half of every exact list by far points gives 0.5."""
    x = workloads.uniform(300, 5, seed=11)
    K = 8
    ei, _ = oracle.bruteforce(x, K)
    approx = ei.copy()
    for u in range(len(x)):
        approx[u, K // 2:] = _far_ids(x, u, set(ei[u].tolist()), K - K // 2)
    assert metrics.recall(x, ei, ei) == 1.0
    assert metrics.recall(x, approx, ei) == 0.5


def test_recall_counts_equal_distance_swaps():
    """Points on a line at 0, 1, 2, ...: for an interior node the K = 3 exact
    list (ties by id) is u-1, u+1, u-2; u+2 is as far as u-2, so a list with
    u+2 in its place is exact (recall 1), while u+3 is a miss (2/3)."""
    n, K = 40, 3
    x = np.arange(n, dtype=np.float32)[:, None]
    rows = np.arange(3, n - 3)
    ei, _ = oracle.bruteforce(x, K)
    assert (ei[rows, 2] == rows - 2).all()
    tie = ei.copy()
    tie[rows, 2] = rows + 2
    miss = ei.copy()
    miss[rows, 2] = rows + 3
    assert metrics.recall(x, tie, ei[rows], rows) == 1.0
    assert metrics.recall(x, miss, ei[rows], rows) == pytest.approx(2.0 / 3.0, abs=1e-12)


def test_recall_repeated_id_counts_once():
    """A list holding one id twice holds one neighbour: a repeated hit counts
    once, and a repeated miss takes nothing away from the other hits."""
    x = workloads.uniform(200, 4, seed=12)
    K = 4
    ei, _ = oracle.bruteforce(x, K)
    rep_hit = ei.copy()
    rep_hit[:, 1] = rep_hit[:, 0]                      # hit, hit again, hit, hit
    assert metrics.recall(x, rep_hit, ei) == 0.75
    rep_miss = ei.copy()
    for u in range(len(x)):
        f = _far_ids(x, u, set(ei[u].tolist()), 1)[0]
        rep_miss[u, 2] = f
        rep_miss[u, 3] = f                             # hit, hit, miss, miss again
    assert metrics.recall(x, rep_miss, ei) == 0.5


# --------------------------------------------------------- check_graph ----

def _clean_graph():
    x = workloads.uniform(120, 4, seed=13)
    ids, dists = oracle.bruteforce(x, 6)
    return x, ids, dists


def test_check_graph_clean_graph_has_no_problem():
    x, ids, dists = _clean_graph()
    assert metrics.check_graph(x, ids, dists) == []
    # 5e-5 relative is inside the 1e-4 tolerance of the returned distances
    d2 = dists.copy()
    d2[:, -1] *= np.float32(1.0 + 5e-5)
    assert metrics.check_graph(x, ids, d2) == []


@pytest.mark.parametrize("fault,expect", [
    ("self", "self-loop"),
    ("repeat", "repeated id"),
    ("order", "not sorted by (dist, id)"),
    ("dist", "distance off"),
])
def test_check_graph_reports_each_fault(fault, expect):
    """One planted fault per case, and the check names it (and nothing the
    fault does not cause)."""
    x, ids, dists = _clean_graph()
    ids, dists = ids.copy(), dists.copy()
    u = 7
    if fault == "self":
        ids[u, 2] = u
    elif fault == "repeat":
        ids[u, 3] = ids[u, 4]
        dists[u, 3] = dists[u, 4]
    elif fault == "order":
        ids[u, [1, 2]] = ids[u, [2, 1]]
        dists[u, [1, 2]] = dists[u, [2, 1]]
    elif fault == "dist":
        dists[u, -1] *= np.float32(1.0 + 2e-4)
    probs = metrics.check_graph(x, ids, dists)
    assert any(p.startswith(expect) for p in probs), probs
    if fault in ("order", "dist"):
        assert len(probs) == 1, probs


# -------------------------------------------------------- window purity ----

def test_window_purity_hand_cases():
    """Fraction of the most frequent cluster in each full window (Section 4,
    greedy heuristic evaluation); a trailing partial window is not counted."""
    lab = np.array([0, 0, 1, 1, 1, 2, 2, 2, 2, 0])
    np.testing.assert_allclose(metrics.window_purity(lab, 3, 3), [2 / 3, 2 / 3, 1.0])
    np.testing.assert_allclose(metrics.window_purity(lab, 5, 3), [3 / 5, 4 / 5])
    lab2 = np.array([0, 1, 2, 3] * 4)
    np.testing.assert_allclose(metrics.window_purity(lab2, 4, 4), [0.25] * 4)
    np.testing.assert_allclose(metrics.window_purity(np.sort(lab2), 4, 4), [1.0] * 4)


# --------------------------------- selection step: old-kind acceptance ----

def _three_groups(na, nb, nc, K, seed, a_new_p):
    """A -> B edges (new with probability a_new_p, else old), B -> C new edges,
    C -> C new edges.  Nothing points at A, and only A points at B."""
    g = np.random.default_rng(seed)
    n = na + nb + nc
    ids = np.empty((n, K), np.int32)
    is_new = np.zeros((n, K), np.uint8)
    for u in range(na):
        ids[u] = na + g.choice(nb, K, replace=False)
        is_new[u] = g.random(K) < a_new_p
    for b in range(na, na + nb):
        ids[b] = na + nb + g.choice(nc, K, replace=False)
        is_new[b] = 1
    for c in range(na + nb, n):
        others = np.array([v for v in range(na + nb, n) if v != c])
        ids[c] = g.choice(others, K, replace=False)
        is_new[c] = 1
    return ids, is_new


def check_forward_old_mean():
    """Node a of A is pointed at by nobody, so old[a] is exactly a's accepted
    forward-old entries (its forward-new ones go to new[a]).  Each old entry is
    accepted with probability min(1, s / (K - fwd_new(a))) (Section 3.1 with
    |N(u)| counted per kind), so |old[a]| averages min(s, K - fwd_new(a))."""
    na, nb, nc, K, rho = 2000, 300, 40, 20, 0.25
    s = oracle.sample_size(rho, K)
    ids, is_new = _three_groups(na, nb, nc, K, seed=21, a_new_p=0.1)
    n = na + nb + nc
    st = oracle.State(workloads.uniform(n, 2, 4), K, rho, seed=5)
    st.init_graph(ids, is_new)
    st.sample(1)
    new, old = st.samples()
    cnt = (K - is_new[:na].sum(1)).astype(np.float64)
    got = np.array([len(old[a]) for a in range(na)], np.float64)
    for a in range(na):
        assert set(old[a].tolist()) <= set(ids[a][is_new[a] == 0].tolist())
    p = np.minimum(1.0, s / cnt)
    var = (cnt * p * (1 - p)).sum()
    assert abs(got.sum() - np.minimum(s, cnt).sum()) < 5 * np.sqrt(var) + 1


def check_reverse_old_mean():
    """Sinks B receive only A's edges, all old, and their own edges are new
    (into C): old[b] is exactly b's accepted reverse-old set, each source kept
    with probability min(1, s / in-degree(b)), so |old[b]| averages
    min(s, in-degree(b))."""
    na, nb, nc, K, rho = 2000, 200, 40, 10, 0.5
    s = oracle.sample_size(rho, K)
    ids, is_new = _three_groups(na, nb, nc, K, seed=22, a_new_p=0.0)
    n = na + nb + nc
    st = oracle.State(workloads.uniform(n, 2, 5), K, rho, seed=6)
    st.init_graph(ids, is_new)
    st.sample(1)
    new, old = st.samples()
    indeg = np.bincount(ids[:na].ravel(), minlength=n)[na:na + nb].astype(np.float64)
    got = np.array([len(old[b]) for b in range(na, na + nb)], np.float64)
    for b in range(na, na + nb):
        assert set(old[b].tolist()) <= set(np.nonzero((ids[:na] == b).any(1))[0].tolist())
    p = np.minimum(1.0, s / indeg)
    var = (indeg * p * (1 - p)).sum()
    assert abs(got.sum() - np.minimum(s, indeg).sum()) < 5 * np.sqrt(var) + 1


def test_sampling_forward_old_mean_is_min_s_old_count():
    check_forward_old_mean()


def test_sampling_reverse_old_mean_is_min_s_old_indegree():
    check_reverse_old_mean()


# Mistakes planted in copies of the oracle: each swaps the counter that an
# old-kind acceptance divides by.
MUTANTS = {
    "forward_old_uses_new_count": ("(uint64_t)(K - fwd_new[u])", "(uint64_t)fwd_new[u]"),
    "forward_old_uses_all_K": ("(uint64_t)(K - fwd_new[u])", "(uint64_t)K"),
    "reverse_old_uses_new_count": ("(uint64_t)rev_old[v]", "(uint64_t)rev_new[v]"),
}


def _mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"knng_oracle_{name}.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / f"liboracle_{name}.so"
    subprocess.run(["gcc", *oracle.CFLAGS, str(path), "-o", str(lib), "-lm", "-lpthread"], check=True)
    return oracle._bind(ctypes.CDLL(str(lib)))


@pytest.mark.parametrize("name,check", [
    ("forward_old_uses_new_count", check_forward_old_mean),
    ("forward_old_uses_all_K", check_forward_old_mean),
    ("reverse_old_uses_new_count", check_reverse_old_mean),
])
def test_old_kind_pins_catch_planted_count_mistakes(tmp_path, monkeypatch, name, check):
    oracle._load()
    monkeypatch.setattr(oracle, "_lib", _mutant(tmp_path, name))
    with pytest.raises(AssertionError):
        check()
