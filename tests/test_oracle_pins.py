"""Pins for the CPU oracle: checks against facts fixed outside the oracle itself
(published generator outputs, hand traces of Algorithm 1, library special
cases, brute force on tiny inputs, closed forms and invariants).  CPU only."""
import ctypes
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from oracle import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _exact_topk(data64, K, cand_sets=None):
    """Exact K smallest (dist, id) per row by numpy float64 and lexsort."""
    n = data64.shape[0]
    diff = data64[:, None, :] - data64[None, :, :]
    D = np.einsum("ijd,ijd->ij", diff, diff)
    np.fill_diagonal(D, np.inf)
    if cand_sets is not None:
        mask = np.ones_like(D, dtype=bool)
        for p in range(n):
            mask[p, list(cand_sets[p])] = False
        D = np.where(mask, np.inf, D)
    ids = np.broadcast_to(np.arange(n), D.shape)
    order = np.lexsort((ids, D), axis=1)[:, :K]
    return order.astype(np.int32), np.take_along_axis(D, order, axis=1)


# ----------------------------------------------------------- generator ----

def test_splitmix64_published_vector():
    lib = oracle._load()
    lib.orc_splitmix64.restype = ctypes.c_uint64
    lib.orc_splitmix64.argtypes = [ctypes.c_uint64]
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    got = [lib.orc_splitmix64((k * gamma) % (1 << 64)) for k in range(len(want))]
    assert got == want


def test_hash_streams_independent():
    # different counters give different words (no accidental aliasing of fields)
    hs = {oracle.hash64(7, s, it, u, j) for s in (1, 2, 3) for it in range(3)
          for u in range(5) for j in range(5)}
    assert len(hs) == 3 * 3 * 5 * 5


# --------------------------------------------------------- brute force ----

@pytest.mark.parametrize("n,d,K,seed", [(40, 3, 5, 0), (64, 8, 10, 1), (17, 1, 16, 2), (50, 33, 7, 3)])
def test_bruteforce_matches_cdist_lexsort(n, d, K, seed):
    """Section 2 brute force against scipy cdist + full lexsort (library special case)."""
    from scipy.spatial.distance import cdist
    x = workloads.uniform(n, d, seed)
    ids, dists = oracle.bruteforce(x, K)
    D = cdist(x.astype(np.float64), x.astype(np.float64), "sqeuclidean")
    np.fill_diagonal(D, np.inf)
    order = np.lexsort((np.broadcast_to(np.arange(n), D.shape), D), axis=1)[:, :K]
    # equal ids wherever the float64 distances are not tied to within rounding
    kth = np.take_along_axis(D, order, axis=1)
    mism = ids != order
    assert not mism.any() or np.allclose(kth[mism], np.take_along_axis(D, ids.astype(np.int64), 1)[mism], rtol=1e-12)
    np.testing.assert_allclose(dists, kth.astype(np.float32), rtol=1e-6)


def test_bruteforce_integer_data_exact_with_ties():
    """Integer-valued data: distances are exact integers, so ids (with the
    (dist, id) tie order) and dists must match an integer computation exactly."""
    g = np.random.default_rng(5)
    xi = g.integers(0, 4, size=(60, 3))
    x = xi.astype(np.float32)
    K = 12
    ids, dists = oracle.bruteforce(x, K)
    Di = ((xi[:, None, :] - xi[None, :, :]) ** 2).sum(-1)
    n = len(xi)
    Di[np.arange(n), np.arange(n)] = 1 << 40
    order = np.lexsort((np.broadcast_to(np.arange(n), Di.shape), Di), axis=1)[:, :K]
    assert (ids == order).all()
    assert (dists == np.take_along_axis(Di, order, 1).astype(np.float32)).all()


def test_bruteforce_rows_subset():
    x = workloads.uniform(300, 5, 9)
    ids, dists = oracle.bruteforce(x, 6)
    rows = np.array([0, 17, 299, 150])
    i2, d2 = oracle.bruteforce(x, 6, rows)
    assert (i2 == ids[rows]).all() and (d2 == dists[rows]).all()


# ---------------------------------------------------------------- init ----

def test_init_lists_valid():
    x = workloads.uniform(500, 6, 1)
    st = oracle.State(x, 10, 0.5, seed=3)
    st.init_random()
    ids, dists, flags = st.state()
    assert metrics.check_graph(x, ids, dists, rtol=1e-6) == []
    assert (flags == 1).all()


def test_init_uniform_chi_square():
    """Section 2: initial neighbours uniform over V \\ {u}; each id is expected
    K times over all lists."""
    from scipy.stats import chi2
    n, K = 400, 20
    st = oracle.State(workloads.uniform(n, 2, 0), K, 1.0, seed=11)
    st.init_random()
    ids, _, _ = st.state()
    cnt = np.bincount(ids.ravel(), minlength=n)
    stat = ((cnt - K) ** 2 / K).sum()
    assert stat < chi2.ppf(0.9999, n - 1)
    assert stat > chi2.ppf(0.0001, n - 1)


@pytest.mark.parametrize("n", [30, 65])
def test_init_complete_graph_is_exact(n):
    """K = n-1: the random initialisation already lists every other node
    (also at K = 64, the widest list the GPU builds)."""
    x = workloads.uniform(n, 4, 2)
    st = oracle.State(x, n - 1, 1.0, seed=0)
    st.init_random()
    ids, dists, _ = st.state()
    ei, ed = oracle.bruteforce(x, n - 1)
    assert (ids == ei).all() and (dists == ed).all()


def test_cluster_miss_bound():
    """Section 3.2: with c equal clusters, Pr[no initial neighbour in own
    cluster] <= ((c-1)/c)^K; sampling without replacement sits just below it."""
    c, K, n = 8, 5, 4000
    x, lab = workloads.gaussian_mixture(n, 4, c, seed=2, return_labels=True)
    st = oracle.State(x, K, 1.0, seed=4)
    st.init_random()
    ids, _, _ = st.state()
    miss = (lab[ids] != lab[:, None]).all(axis=1).mean()
    bound = ((c - 1) / c) ** K
    sd = math.sqrt(bound * (1 - bound) / n)
    assert miss <= bound + 4 * sd
    assert miss >= bound - 0.05


# ------------------------------------------------------------ sampling ----

def test_sampling_takes_everything_when_counts_small():
    """Section 3.1 probability rho*K/|N(u)| >= 1 when |N(u)| <= rho*K: with
    rho = 1 every forward entry is accepted and every new entry loses its flag."""
    n, K = 200, 8
    x = workloads.uniform(n, 3, 3)
    ids, is_new = workloads.random_graph(n, K, seed=5, p_new=0.5)
    st = oracle.State(x, K, 1.0, seed=1)
    st.init_graph(ids, is_new)
    st.sample(1)
    new, old = st.samples()
    sid, _, sflags = st.state()
    assert (sflags == 0).all()
    for u in range(n):
        fwd_new = set(ids[u][is_new[u] == 1].tolist())
        fwd_old = set(ids[u][is_new[u] == 0].tolist())
        assert fwd_new <= set(new[u].tolist())
        assert fwd_old - fwd_new <= set(old[u].tolist()) | set(new[u].tolist())
        assert len(set(new[u].tolist())) == len(new[u])
        assert not (set(new[u].tolist()) & set(old[u].tolist()))
        assert u not in set(new[u].tolist()) | set(old[u].tolist())


def test_sampling_forward_mean_is_min_s_cnt():
    """Accepted forward-new entries (= cleared flags) average min(s, cnt)."""
    n, K, rho = 3000, 20, 0.25
    s = oracle.sample_size(rho, K)
    ids, is_new = workloads.random_graph(n, K, seed=8, p_new=0.7)
    st = oracle.State(workloads.uniform(n, 2, 0), K, rho, seed=2)
    st.init_graph(ids, is_new)
    st.sample(1)
    _, _, flags = st.state()
    cnt = is_new.sum(1).astype(np.float64)
    cleared = cnt - flags.sum(1)
    expect = np.minimum(s, cnt).sum()
    # Binomial(cnt, s/cnt) variance per node
    var = np.where(cnt > s, cnt * (s / np.maximum(cnt, 1)) * (1 - s / np.maximum(cnt, 1)), 0).sum()
    assert abs(cleared.sum() - expect) < 5 * math.sqrt(var) + 1


def test_sampling_reverse_mean_is_min_s_indegree():
    """Reverse half: sources A point only at sinks B with new edges, sinks point
    only at A with old edges, so new[b] is exactly b's accepted reverse-new
    set; its mean size is min(s, indegree)."""
    g = np.random.default_rng(3)
    na, nb, K, rho = 2000, 200, 10, 0.5
    s = oracle.sample_size(rho, K)
    n = na + nb
    ids = np.empty((n, K), np.int32)
    is_new = np.zeros((n, K), np.uint8)
    for u in range(na):
        ids[u] = na + g.choice(nb, K, replace=False)
        is_new[u] = 1
    for b in range(na, n):
        ids[b] = g.choice(na, K, replace=False)
    st = oracle.State(workloads.uniform(n, 2, 1), K, rho, seed=9)
    st.init_graph(ids, is_new)
    st.sample(1)
    new, old = st.samples()
    indeg = np.bincount(ids[:na].ravel(), minlength=n)[na:]
    got = np.array([len(new[b]) for b in range(na, n)], np.float64)
    for b in range(na, n):
        assert set(new[b].tolist()) <= set(np.nonzero((ids[:na] == b).any(1))[0].tolist())
    p = np.minimum(1.0, s / indeg)
    var = (indeg * p * (1 - p)).sum()
    assert abs(got.sum() - np.minimum(s, indeg).sum()) < 5 * math.sqrt(var) + 1


# ------------------------------------------------- priority-heap sampling ----

def _bipartite(na, nb, K, seed):
    """Sources 0..na-1 point at K sinks each with new edges; sinks point at K
    sources each with old edges."""
    g = np.random.default_rng(seed)
    n = na + nb
    ids = np.empty((n, K), np.int32)
    is_new = np.zeros((n, K), np.uint8)
    for u in range(na):
        ids[u] = na + g.choice(nb, K, replace=False)
        is_new[u] = 1
    for b in range(na, n):
        ids[b] = g.choice(na, K, replace=False)
    return ids, is_new


def test_heap_sampling_sizes_are_exact():
    """The heap keeps the s smallest-priority distinct offers: a sink's new
    candidates are exactly min(s, in-degree) of its in-neighbours, and a
    source keeps exactly s of its K new forward entries (and clears exactly
    those flags) -- where turbosampling only matches these in expectation."""
    na, nb, K, rho = 1500, 150, 10, 0.5
    s = oracle.sample_size(rho, K)
    ids, is_new = _bipartite(na, nb, K, seed=4)
    n = na + nb
    st = oracle.State(workloads.uniform(n, 2, 1), K, rho, seed=7, sampler="heap")
    st.init_graph(ids, is_new)
    st.sample(1)
    new, old = st.samples()
    sid, _, flags = st.state()  # lists in their (dist, id) order
    indeg = np.bincount(ids[:na].ravel(), minlength=n)
    for b in range(na, n):
        src = set(np.nonzero((ids[:na] == b).any(1))[0].tolist())
        assert len(new[b]) == min(s, indeg[b]) and set(new[b].tolist()) <= src
        assert len(set(new[b].tolist())) == len(new[b])
    for a in range(na):
        assert len(new[a]) == s and set(new[a].tolist()) <= set(ids[a].tolist())
        cleared = set(sid[a][flags[a] == 0].tolist())
        assert cleared == set(new[a].tolist())
        assert len(old[a]) <= s
    assert (flags[na:] == 0).all()  # sinks' entries were old already


def test_heap_sampling_is_uniform_without_replacement():
    """Each of a sink's m in-neighbours is kept with probability s / m over
    fresh iterations (priorities redrawn per iteration): a chi-square test
    over every (sink, in-neighbour) pair."""
    na, nb, K, rho, T = 600, 60, 10, 0.3, 400
    s = oracle.sample_size(rho, K)
    ids, is_new = _bipartite(na, nb, K, seed=6)
    n = na + nb
    st = oracle.State(workloads.uniform(n, 2, 2), K, rho, seed=3, sampler="heap")
    hits = np.zeros((n, n), np.int64)
    for it in range(1, T + 1):
        st.init_graph(ids, is_new, 0)
        st.sample(it)
        new, _ = st.samples()
        for b in range(na, n):
            hits[b, new[b]] += 1
    chi, dof = 0.0, 0
    for b in range(na, n):
        src = np.nonzero((ids[:na] == b).any(1))[0]
        m = len(src)
        p = min(1.0, s / m)
        if p >= 1.0:
            assert (hits[b, src] == T).all()
            continue
        e = T * p
        chi += (((hits[b, src] - e) ** 2) / (e * (1 - p))).sum()
        dof += m
    # chi-square with dof degrees of freedom: mean dof, sd sqrt(2 dof)
    assert abs(chi - dof) < 5 * math.sqrt(2 * dof)


def test_heap_sampling_one_offer_per_id():
    """A symmetric ring (u lists its K nearest ring neighbours, all new) offers
    every neighbour twice, forward and reverse: the kept sets hold distinct
    ids, exactly s of them, each neighbour with frequency s / K."""
    n, K, rho, T = 400, 8, 0.5, 300
    s = oracle.sample_size(rho, K)
    off = np.array([o for o in range(1, K // 2 + 1)] + [-o for o in range(1, K // 2 + 1)])
    ids = ((np.arange(n)[:, None] + off[None, :]) % n).astype(np.int32)
    is_new = np.ones((n, K), np.uint8)
    st = oracle.State(workloads.uniform(n, 2, 3), K, rho, seed=5, sampler="heap")
    freq = np.zeros((n, K), np.int64)
    for it in range(1, T + 1):
        st.init_graph(ids, is_new, 0)
        st.sample(it)
        new, old = st.samples()
        for u in range(n):
            assert len(new[u]) == s and len(set(new[u].tolist())) == s
            assert set(new[u].tolist()) <= set(ids[u].tolist()) and len(old[u]) == 0
            freq[u] += np.isin(ids[u], new[u])
    p = s / K
    mean = freq.mean() / T
    assert abs(mean - p) < 5 * math.sqrt(p * (1 - p) / (T * n * K))


def test_heap_sampling_takes_everything_at_rho_one():
    """rho = 1 on the ring: s = K >= the K distinct offers, so every list
    entry is kept as a new candidate and every flag is cleared."""
    n, K = 300, 6
    off = np.array([1, 2, 3, -1, -2, -3])
    ids = ((np.arange(n)[:, None] + off[None, :]) % n).astype(np.int32)
    st = oracle.State(workloads.uniform(n, 2, 4), K, 1.0, seed=1, sampler="heap")
    st.init_graph(ids, np.ones((n, K), np.uint8))
    st.sample(1)
    new, old = st.samples()
    _, _, flags = st.state()
    assert (flags == 0).all()
    for u in range(n):
        assert set(new[u].tolist()) == set(ids[u].tolist()) and len(old[u]) == 0


def test_heap_sampling_build_recall():
    """Whole NN-Descent with the heap sampler on 2,000 uniform points in
    [0,1)^8 (K=10, rho=1) reaches recall 0.99 like turbosampling."""
    w, x = workloads.make("uniform_n2k_d8")
    ei, _ = oracle.bruteforce(x, w.K)
    oi, od, st = oracle.build_knng(x, w.K, w.rho, w.delta, w.max_iters, seed=0, sampler="heap")
    assert metrics.check_graph(x, oi, od) == []
    assert metrics.recall(x, oi, ei) >= 0.99


# ---------------------------------------------------------------- join ----

@pytest.mark.parametrize("n,K", [(48, 6), (90, 48)])
def test_join_all_pairs_reduces_to_topk(n, K):
    """Section 2 update rule fed with every pair among nodes 1..n-1 (placed in
    new[0]): each list becomes the K smallest distinct (dist, id) over its start
    entries and all other nodes except 0 -- brute force, integer data."""
    g = np.random.default_rng(1)
    xi = g.integers(0, 5, size=(n, 4))
    x = xi.astype(np.float32)
    ids0, is_new0 = workloads.random_graph(n, K, seed=3)
    st = oracle.State(x, K, 1.0, seed=0)
    st.init_graph(ids0, is_new0)
    others = np.arange(1, n, dtype=np.int32)
    st.set_samples([others] + [np.empty(0, np.int32)] * (n - 1), [np.empty(0, np.int32)] * n)
    out = st.join()
    assert out["evals"] == (n - 1) * (n - 2) // 2
    ids, dists, _ = st.state()
    cand = [set(range(1, n)) - {p} | set(ids0[p].tolist()) for p in range(n)]
    eids, ed = _exact_topk(xi.astype(np.float64), K, cand)
    assert (ids[1:] == eids[1:]).all()
    assert (dists[1:] == ed[1:].astype(np.float32)).all()
    # node 0 is in no candidate set: its list keeps its start entries
    assert set(ids[0].tolist()) == set(ids0[0].tolist())
    assert out["inserts"] >= out["changes"]


@pytest.mark.parametrize("K", [8, 40])
def test_iterations_monotone_and_valid(K):
    x = workloads.uniform(800, 4, 7)
    st = oracle.State(x, K, 0.5, seed=5)
    st.init_random()
    prev = st.state()[1]
    for _ in range(5):
        r = st.iterate()
        ids, dists, _ = st.state()
        assert metrics.check_graph(x, ids, dists, rtol=1e-6) == []
        assert (dists[:, -1] <= prev[:, -1]).all()
        assert dists.sum() <= prev.sum()
        assert r["inserts"] >= r["changes"]
        prev = dists


def test_build_complete_graph_recall_one():
    x = workloads.uniform(40, 3, 1)
    ids, dists, st = oracle.build_knng(x, 39, 1.0, 0.0, 3, seed=2)
    ei, _ = oracle.bruteforce(x, 39)
    assert metrics.recall(x, ids, ei) == 1.0


def test_build_small_reaches_exact():
    x = workloads.uniform(120, 3, 4)
    ids, dists, st = oracle.build_knng(x, 6, 1.0, 0.0, 30, seed=1)
    ei, _ = oracle.bruteforce(x, 6)
    assert metrics.recall(x, ids, ei) == 1.0
    assert metrics.check_graph(x, ids, dists, rtol=1e-6) == []


def test_build_uniform_n2k_recall_over_099():
    """Section 2: recall above 99% (uniform n=2000, d=8, K=10, rho=1)."""
    w, x = workloads.make("uniform_n2k_d8")
    ei, _ = oracle.bruteforce(x, w.K)
    for mode in ("batched", "inplace"):
        ids, dists, st = oracle.build_knng(x, w.K, w.rho, w.delta, w.max_iters, 0, mode)
        assert metrics.recall(x, ids, ei) >= 0.99
        assert metrics.check_graph(x, ids, dists, rtol=1e-6) == []


def test_termination_threshold():
    """Section 2: iterations stop once changes < delta*n*K (count of the last
    iteration run is below the threshold, unless the cap was hit)."""
    x = workloads.uniform(1000, 4, 3)
    K, delta = 8, 0.01
    ids, d, st = oracle.build_knng(x, K, 1.0, delta, 50, seed=0)
    assert st["iters"] < 50
    assert st["last_changes"] < delta * 1000 * K


# ----------------------------------------------------------- Algorithm 1 ----

def test_alg1_hand_trace_both_readings():
    g = json.load(open(os.path.join(GOLDEN, "alg1_line5.json")))
    lists = np.array(g["lists"], np.int32)
    # the fixture lists are the exact lists of the points
    pts = np.array(g["points_1d"], np.float32)[:, None]
    ei, _ = oracle.bruteforce(pts, g["K"])
    assert (ei == lists).all()
    for rd in ("a", "b"):
        sg, si = oracle.greedy_reorder(lists, reading_b=(rd == "b"))
        assert sg.tolist() == g[f"sigma_reading_{rd}"]
        assert si.tolist() == g[f"sigma_inv_reading_{rd}"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_alg1_is_permutation_with_inverse(seed):
    n, K = 500, 7
    x = workloads.uniform(n, 3, seed)
    ei, _ = oracle.bruteforce(x, K)
    for rb in (False, True):
        sg, si = oracle.greedy_reorder(ei, rb)
        assert sorted(sg.tolist()) == list(range(n))
        assert (si[sg] == np.arange(n)).all()


def test_alg1_line_is_identity():
    """Points on a line in id order: every next spot is already held by the
    nearest unplaced neighbour, so sigma stays the identity."""
    n, K = 100, 4
    x = np.arange(n, dtype=np.float32)[:, None]
    ei, _ = oracle.bruteforce(x, K)
    sg, si = oracle.greedy_reorder(ei)
    assert (sg == np.arange(n)).all()


def test_alg1_recovers_clusters_early():
    """Section 4 (clustering quality, Fig. 4): on clusters in random order the
    leading windows after reordering are dominated by single clusters, far
    above the uniform 1/c, while the tail falls back towards 1/c.  The literal
    reading (list of node i) does not cluster, which is why the node on spot i
    is the default reading."""
    c, n, K = 8, 4096, 10
    x, lab = workloads.gaussian_mixture(n, 8, c, seed=3, centre_low=-50, centre_high=50,
                                        return_labels=True)
    ei, _ = oracle.bruteforce(x, K)
    before = metrics.window_purity(lab, 256, c)
    after = metrics.window_purity(lab[oracle.greedy_reorder(ei)[1]], 256, c)
    lit = metrics.window_purity(lab[oracle.greedy_reorder(ei, True)[1]], 256, c)
    half = len(after) // 2
    assert before.max() < 0.4
    assert after[:half].mean() > 4.0 / c
    assert after[:half].mean() > after[-2:].mean()
    assert lit[:half].mean() < after[:half].mean()


# ------------------------------------------- parallel relabelling variant ----

def _contiguous(levels, sigma):
    """Every component of every round occupies one contiguous range of spots."""
    for lv in levels:
        order = np.argsort(lv, kind="stable")
        lab = lv[order]
        pos = sigma[order]
        cut = np.flatnonzero(np.diff(lab)) + 1
        for seg in np.split(pos, cut):
            if seg.max() - seg.min() + 1 != len(seg):
                return False
    return True


@pytest.mark.parametrize("n,K,seed", [(300, 4, 1), (2000, 6, 2), (5000, 3, 3)])
def test_parallel_relabel_is_single_linkage(n, K, seed):
    """The hooked edges form a minimum spanning forest of the list graph
    (single linkage): same total weight and same components as scipy's
    minimum_spanning_tree / connected_components on the symmetrised graph."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    x = workloads.uniform(n, 3, seed)
    ids, _ = workloads.random_graph(n, K, seed=seed + 10, p_new=1.0)
    levels, w, sg = oracle.parallel_relabel(x, ids)
    rows = np.repeat(np.arange(n), K)
    cols = ids.ravel()
    x64 = x.astype(np.float64)
    wt = np.array([np.float32(((x64[a] - x64[b]) ** 2).sum()) for a, b in zip(rows, cols)], np.float64)
    g = sp.coo_matrix((wt, (rows, cols)), shape=(n, n)).tocsr()
    g = g.maximum(g.T)
    mst = csgraph.minimum_spanning_tree(g)
    assert abs(w - mst.sum()) <= 1e-9 * max(1.0, mst.sum())
    ncomp, _ = csgraph.connected_components(g, directed=False)
    assert len(np.unique(levels[-1])) == ncomp
    assert sorted(sg.tolist()) == list(range(n))
    assert _contiguous(levels, sg)


def test_parallel_relabel_recovers_clusters_everywhere():
    """Fig. 4 setting (clustered, n = 16,384, d = 8, 8 clusters; lists after
    one iteration, windows of 2,000): single linkage merges the clusters last,
    so every cluster is one run of spots -- every window holds at most two
    clusters -- where Algorithm 1's tail falls towards 1/c."""
    n, d, c = 16384, 8, 8
    x, lab = workloads.gaussian_mixture(n, d, c, seed=2, return_labels=True)
    st = oracle.State(x, 20, 0.5, seed=1)
    st.init_random()
    st.iterate()
    ids, _, _ = st.state()
    levels, _, sg = oracle.parallel_relabel(x, ids)
    inv = np.empty(n, np.int64)
    inv[sg] = np.arange(n)
    par = metrics.window_purity(lab[inv], 2000, c)
    runs = (np.diff(lab[inv]) != 0).sum() + 1
    assert runs == c
    a1, _ = oracle.greedy_reorder(ids)
    inv1 = np.empty(n, np.int64)
    inv1[a1] = np.arange(n)
    alg1 = metrics.window_purity(lab[inv1], 2000, c)
    assert par.min() >= 0.8 and par.mean() > alg1.mean()
    assert _contiguous(levels, sg)


def test_build_with_reorder_returns_original_labels():
    w, x = workloads.make("uniform_n2k_d8")
    ei, _ = oracle.bruteforce(x, w.K)
    ids, dists, st = oracle.build_knng(x, w.K, w.rho, w.delta, w.max_iters, 0, reorder=1)
    assert st["reordered"]
    assert metrics.check_graph(x, ids, dists, rtol=1e-6) == []
    assert metrics.recall(x, ids, ei) >= 0.99


# ------------------------------------------- batched build on many threads ----

@pytest.mark.parametrize("threads,block_pairs", [(1, 1 << 25), (3, 1 << 25), (8, 5000), (5, 1)])
def test_multithread_build_equals_serial_build(threads, block_pairs):
    """Reading 6 (Section 2 loop, update visibility): with the candidate sets
    fixed for an iteration, the lists end the same whatever order the
    proposals are applied in.  The threaded build (blocks of nodes, proposals
    filtered against the current worst entry, applied per target range) must
    therefore equal the serial build with the batched change count, bit for
    bit and with the same number of iterations, for any thread count and any
    block size (block_pairs 1: one node per block)."""
    lib = oracle._load()
    lib.orc_set_mt_block_pairs(block_pairs)
    try:
        for (n, d, K, rho, delta, it, seed) in [(1500, 8, 10, 1.0, 0.001, 10, 3), (2500, 12, 12, 0.5, 0.0, 6, 4)]:
            x = workloads.gaussian_mixture(n, d, clusters=12, seed=seed)
            a_ids, a_d, a_st = oracle.build_knng(x, K, rho, delta, it, seed=seed, count_mode="batched")
            b_ids, b_d, b_st = oracle.build_knng_mt(x, K, rho, delta, it, seed=seed, threads=threads)
            assert b_st["threads"] == threads
            np.testing.assert_array_equal(a_ids, b_ids)
            np.testing.assert_array_equal(a_d, b_d)
            assert (a_st["iters"], a_st["evals"], a_st["last_changes"]) == \
                (b_st["iters"], b_st["evals"], b_st["last_changes"])
    finally:
        lib.orc_set_mt_block_pairs(1 << 25)


def test_multithread_build_equals_inplace_lists():
    """The in-place build (later joins see earlier updates within an
    iteration, the paper's single-core order) gives the same lists when both
    run the same iterations (delta = 0): reading 6 against the in-place code."""
    x = workloads.uniform(1200, 6, seed=8)
    a_ids, a_d, _ = oracle.build_knng(x, 8, 0.6, 0.0, 7, seed=1, count_mode="inplace")
    b_ids, b_d, b_st = oracle.build_knng_mt(x, 8, 0.6, 0.0, 7, seed=1, threads=4)
    assert b_st["iters"] == 7
    np.testing.assert_array_equal(a_ids, b_ids)
    np.testing.assert_array_equal(a_d, b_d)


def test_join_range_halves_make_the_whole_step():
    """The calculation step of two node ranges in turn is the whole step: the
    same evaluations and (reading 6) the same lists."""
    x = workloads.uniform(1500, 6, seed=2)
    a = oracle.State(x, 8, 0.7, seed=3)
    b = oracle.State(x, 8, 0.7, seed=3)
    for s in (a, b):
        s.init_random()
        s.sample(1)
    whole = a.join()
    h1, h2 = b.join_range(0, 700), b.join_range(700, 1500)
    assert h1["evals"] + h2["evals"] == whole["evals"]
    np.testing.assert_array_equal(a.state()[0], b.state()[0])
    np.testing.assert_array_equal(a.state()[1], b.state()[1])
