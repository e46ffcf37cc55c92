"""GPU parity: every CUDA step against the CPU oracle on the same seeded
inputs, through the C ABI.

Integer-valued inputs make every squared distance an exact float32 integer on
both sides, so there the two implementations must agree bit for bit (ids,
distances, flags, change counts), including ties, which both break by id.
Real-valued inputs are compared with the tolerances of the method: ids equal
up to ties (|d_a - d_b| <= 1e-5 d_b), distances within 1e-5 relative (brute
force), recall within 0.005 of the oracle's, every returned distance within
1e-4 relative of its float64 recomputation.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2112_06630_gb300 as knng  # noqa: E402


def _int_data(n, d, hi, seed, density=1.0):
    g = np.random.default_rng(seed)
    x = g.integers(0, hi, size=(n, d))
    if density < 1.0:
        x = np.where(g.random((n, d)) < density, x, 0)
    return x.astype(np.float32)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def assert_ids_up_to_ties(gi, gd, oi, od, rtol=1e-5):
    gi, gd = np.asarray(gi), np.asarray(gd)
    np.testing.assert_allclose(gd, od, rtol=rtol, atol=1e-7)
    mism = gi != oi
    if mism.any():
        assert np.allclose(gd[mism], od[mism], rtol=rtol, atol=1e-7)


# ------------------------------------------------------------ brute force ----

@pytest.mark.parametrize("n,d,K", [(2000, 8, 10), (1037, 5, 7), (700, 33, 16), (513, 16, 32), (300, 130, 20),
                                   (2, 3, 1), (33, 4, 32), (700, 6, 48), (130, 3, 64), (65, 33, 64)])
def test_bruteforce_matches_oracle(n, d, K):
    x = workloads.uniform(n, d, seed=n + d)
    gi, gd = knng.knng_bruteforce(_cuda(x), K)
    oi, od = oracle.bruteforce(x, K)
    assert_ids_up_to_ties(gi.cpu().numpy(), gd.cpu().numpy(), oi, od)


def test_bruteforce_integer_data_bit_exact_with_ties():
    x = _int_data(1500, 12, 4, seed=1)     # many equal distances
    gi, gd = knng.knng_bruteforce(_cuda(x), 20)
    oi, od = oracle.bruteforce(x, 20)
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


TC_CASES = [
    # n, d, K, rows (None = all), data kind
    (6000, 16, 20, None, "mix"),
    (20000, 128, 32, 700, "mix"),
    (9000, 8, 10, None, "int"),      # many equal distances: ties by id
    (50000, 64, 16, 500, "mix"),
    (8191, 100, 32, 333, "int"),     # ragged last tile and slice, padded rows
]


@pytest.mark.parametrize("n,d,K,nrows,kind", TC_CASES)
def test_tensor_core_bruteforce_equals_exact_kernel(n, d, K, nrows, kind, monkeypatch):
    """The tcgen05 split-bf16 prefilter with exact re-rank (and exact
    recomputation of uncertified queries) returns the same ids and distances,
    bit for bit, as the CUDA-core kernel that evaluates every pair."""
    x = _int_data(n, d, 5, seed=n) if kind == "int" else workloads.gaussian_mixture(n, d, 30, seed=n)
    rows = None if nrows is None else torch.from_numpy(np.random.default_rng(1).choice(n, nrows, replace=False)).cuda()
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "tensor")
    ti, td = knng.knng_bruteforce(_cuda(x), K, rows=rows)
    fallbacks = knng.bruteforce_last_fallbacks()
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "cuda")
    ci, cd = knng.knng_bruteforce(_cuda(x), K, rows=rows)
    assert knng.bruteforce_last_fallbacks() == -1
    assert fallbacks >= 0
    assert torch.equal(ti, ci) and torch.equal(td, cd)
    if kind == "mix":  # real-valued data: the bound certifies nearly every query
        assert fallbacks <= 0.05 * ti.shape[0], fallbacks


def test_tensor_core_bruteforce_offset_data_and_fallbacks(monkeypatch):
    """Data far from the origin (non-negative features plus an offset): the
    prefilter centres the points, so the error bound stays small and almost
    every query is certified.  Integer data with many equal distances sends
    queries to the exact kernel (sliced over the points); both give the exact
    kernel's answer bit for bit."""
    g = np.random.default_rng(7)
    x = (g.random((30000, 64), dtype=np.float32) + 50.0).astype(np.float32)
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "tensor")
    ti, td = knng.knng_bruteforce(_cuda(x), 20)
    fb = knng.bruteforce_last_fallbacks()
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "cuda")
    ci, cd = knng.knng_bruteforce(_cuda(x), 20)
    assert torch.equal(ti, ci) and torch.equal(td, cd)
    assert 0 <= fb <= 0.05 * x.shape[0], fb
    xi = _int_data(40000, 8, 4, seed=3)
    rows = torch.arange(0, 40000, 37, device="cuda")
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "tensor")
    ti, td = knng.knng_bruteforce(_cuda(xi), 16, rows=rows)
    fb = knng.bruteforce_last_fallbacks()
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "cuda")
    ci, cd = knng.knng_bruteforce(_cuda(xi), 16, rows=rows)
    assert fb > 0
    assert torch.equal(ti, ci) and torch.equal(td, cd)


def test_bruteforce_query_rows_and_host_pointers():
    x = workloads.gaussian_mixture(5000, 16, 20, seed=3)
    rows = np.array([0, 4999, 17, 2500, 1234], np.int64)
    gi, gd = knng.knng_bruteforce(x, 20, rows=rows)          # host in, host out
    oi, od = oracle.bruteforce(x, 20, rows)
    assert_ids_up_to_ties(gi, gd, oi, od)


def test_bruteforce_duplicate_points():
    x = np.zeros((300, 8), np.float32)
    x[150:] = 1.0
    gi, gd = knng.knng_bruteforce(_cuda(x), 5)
    oi, od = oracle.bruteforce(x, 5)
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


# ------------------------------------------------------------ random init ----

@pytest.mark.parametrize("n,d,K", [(3001, 8, 10), (500, 3, 20), (33, 5, 32), (2, 1, 1), (3000, 8, 48), (700, 5, 64),
                                   (65, 4, 64), (900, 70, 40)])
def test_init_matches_oracle_exactly(n, d, K):
    x = _int_data(n, d, 16, seed=K)
    with knng.Context(_cuda(x), K, rho=0.5, seed=7) as c:
        gi, gd, gf = c.state()
    st = oracle.State(x, K, 0.5, seed=7)
    st.init_random()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()


# ------------------------------------------------------ sampling + join ----

CASES = [
    # n, d, K, rho, int range  (spans several warps/blocks, ragged tails,
    # each list-size template, padded and unpadded rows, the global-row path)
    (3001, 8, 10, 1.0, 16),
    (2500, 16, 20, 0.5, 8),
    (1800, 3, 16, 0.5, 6),
    (1200, 17, 32, 0.3, 5),
    (900, 40, 8, 0.5, 4),
    (400, 600, 12, 0.5, 3),     # block-per-node tile kernel (rows > 64 floats)
    (700, 65, 32, 0.3, 4),      # tile kernel, ragged last 64-float chunk
    (1500, 100, 20, 0.5, 3),    # tile kernel, two passes of new rows possible
    (2000, 8, 40, 0.25, 16),    # two list keys per lane (K > 32)
    (1500, 12, 64, 0.15, 8),    # K = 64
    (800, 140, 48, 0.2, 3),     # K = 48 through the pipelined kernel
]


@pytest.mark.parametrize("n,d,K,rho,hi", CASES)
def test_one_iteration_matches_oracle_bit_exact(n, d, K, rho, hi):
    x = _int_data(n, d, hi, seed=n)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gnew, gold = c.samples()
        gi, gd, gf = c.state()
        stats = c.stats()
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    assert stats["rev_overflow"] == 0 and stats["set_overflow"] == 0
    onew, oold = st.samples()
    for u in range(n):
        sn = set(gnew[u].tolist())
        assert sn == set(onew[u].tolist())
        assert set(gold[u].tolist()) - sn == set(oold[u].tolist())
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]
    assert stats["dist_evals"] == r["evals"]


PATH_CASES = [
    # n, d, K, rho, int range, bf16 flag
    (4000, 600, 12, 0.5, 3, False),   # ~48 KB ring slots: every block wraps its ring
    (700, 65, 32, 0.3, 4, False),     # 17 float4 per row, K = 32 list snapshots
    (1500, 100, 20, 0.5, 3, False),
    (1200, 64, 16, 0.5, 4, True),     # one 64-bf16 k-block
    (600, 128, 32, 0.3, 4, True),
    (2000, 150, 20, 1.0, 4, True),    # up to 64 candidates: four 16-row tiles
    (2000, 200, 20, 1.0, 3, False),   # two column blocks of the pipelined kernel, up to 64 candidates
    (1500, 33, 16, 0.5, 4, False),    # 9 float4 per row: the narrowest pipelined row
    (3000, 256, 24, 0.5, 3, False),   # the widest pipelined row (64 float4)
    (1200, 100, 48, 0.2, 3, False),   # K = 48: two list keys per lane, 48-entry list snapshots
    (900, 300, 64, 0.15, 3, False),   # K = 64
]
PATH_IDS = {"warp": 0, "tile": 1, "ring": 2, "pipe": 3, "pipe8": 4}


def _pipe_eligible(d, bf16):
    """The pipelined block kernel takes float32 rows of 33 to 256 floats."""
    dp = (d + 3) // 4 * 4
    return not bf16 and 32 < dp <= 256


@pytest.mark.parametrize("path", ["tile", "ring", "pipe"])
@pytest.mark.parametrize("n,d,K,rho,hi,bf16", PATH_CASES)
def test_join_kernels_match_oracle_bit_exact(path, n, d, K, rho, hi, bf16, monkeypatch):
    """The block-per-node tile kernel, the ring kernel and the pipelined
    block kernel, forced on the same inputs: one iteration bit-exact against
    the oracle (integer data: the bf16 expansion is exact too)."""
    if path == "pipe" and not _pipe_eligible(d, bf16):
        pytest.skip("rows outside the pipelined kernel's range")
    monkeypatch.setenv("KNNG_TEST_JOIN_PATH", path)
    x = _int_data(n, d, hi, seed=n + d)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    flags = knng.FLAG_BF16 if bf16 else 0
    with knng.Context(_cuda(x), K, rho=rho, seed=11, graph=(ids0, new0), iter=0, flags=flags) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    assert stats["join_path"] == PATH_IDS[path]
    assert stats["set_overflow"] == 0 and stats["lock_timeouts"] == 0
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]
    assert stats["dist_evals"] == r["evals"]


@pytest.mark.parametrize("path", ["warp", "tile", "ring", "pipe"])
def test_join_kernels_agree_on_real_valued_builds(path, monkeypatch):
    """Whole float32 builds on real-valued clustered data through each join
    kernel: every float32 distance uses the same arithmetic, so the four
    kernels give the same graph bit for bit."""
    monkeypatch.setenv("KNNG_TEST_JOIN_PATH", path)
    x = workloads.gaussian_mixture(6000, 72, 20, seed=4)
    ids, dists, st = knng.knng_build(_cuda(x), 16, 0.5, 0.001, 8, seed=2)
    assert st["join_path"] == PATH_IDS[path]
    monkeypatch.setenv("KNNG_TEST_JOIN_PATH", "warp")
    ids_w, dists_w, _ = knng.knng_build(_cuda(x), 16, 0.5, 0.001, 8, seed=2)
    assert torch.equal(ids, ids_w) and torch.equal(dists, dists_w)


@pytest.mark.parametrize("d", [24, 72])
def test_capped_candidate_sets_are_deterministic(d, monkeypatch):
    """K = 32 at rho 1.0: a node's sampled union (forward up to K, reverse
    new and old up to s each) passes the cap of 64 candidates on many nodes,
    and the cap drops the tail of a canonical order (reverse parts ordered by
    a fixed bijection of the ids, first copy of a repeat kept).  So the graph
    does not depend on the order in which other warps took the reverse slots:
    repeated builds, every join kernel and a batched build (other data sets
    interleaved in the same launches) give the same graph bit for bit."""
    x = workloads.gaussian_mixture(4000, d, 12, seed=d)
    xd = _cuda(x)
    ref_i, ref_d, st = knng.knng_build(xd, 32, 1.0, 0.001, 6, seed=3)
    assert st["set_overflow"] > 0 and st["lock_timeouts"] == 0
    for _ in range(2):
        ids, dists, _ = knng.knng_build(xd, 32, 1.0, 0.001, 6, seed=3)
        assert torch.equal(ids, ref_i) and torch.equal(dists, ref_d)
    for path in ("warp", "tile", "ring", "pipe") if d > 32 else ("warp", "tile", "ring"):
        monkeypatch.setenv("KNNG_TEST_JOIN_PATH", path)
        ids, dists, st_p = knng.knng_build(xd, 32, 1.0, 0.001, 6, seed=3)
        assert st_p["join_path"] == PATH_IDS[path]
        assert torch.equal(ids, ref_i) and torch.equal(dists, ref_d), path
    monkeypatch.delenv("KNNG_TEST_JOIN_PATH")
    others = [workloads.gaussian_mixture(3000 + 500 * b, d, 10, seed=100 + b) for b in range(3)]
    outs, _ = knng.knng_build_batched([_cuda(o) for o in others[:2]] + [xd] + [_cuda(others[2])], 32, 1.0,
                                      0.001, 6, seed=3)
    assert torch.equal(outs[2][0], ref_i) and torch.equal(outs[2][1], ref_d)


@pytest.mark.parametrize("pool", ["1", "40"])
def test_bucket_overflow_paths_match_oracle_bit_exact(pool, monkeypatch):
    """A (test-only) tiny proposal pool forces runs past the first 256 keys of
    a bucket onto poisoned runs and locked list insertions; the lists must
    still equal the oracle's."""
    monkeypatch.setenv("KNNG_TEST_BUCKET_POOL_CHUNKS", pool)
    n, d, K, rho, hi = 1800, 3, 16, 0.5, 6
    x = _int_data(n, d, hi, seed=n)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    assert stats["bucket_overflow"] > 0 and stats["lock_timeouts"] == 0
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]


@pytest.mark.parametrize("path", ["tile", "ring", "pipe"])
def test_bucket_overflow_paths_high_d_kernels(path, monkeypatch):
    """The same tiny-pool overflow drive through the tile, ring and
    pipelined kernels."""
    monkeypatch.setenv("KNNG_TEST_BUCKET_POOL_CHUNKS", "1")
    monkeypatch.setenv("KNNG_TEST_JOIN_PATH", path)
    n, d, K, rho, hi = 1800, 70, 16, 0.5, 3
    x = _int_data(n, d, hi, seed=n)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    assert stats["join_path"] == PATH_IDS[path]
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    assert stats["bucket_overflow"] > 0 and stats["lock_timeouts"] == 0
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]


@pytest.mark.parametrize("n,d,K,rho", [(1200, 64, 16, 0.5), (800, 150, 20, 1.0), (600, 128, 32, 0.3)])
def test_bf16_tensor_core_join_exact_on_small_integers(n, d, K, rho):
    """bf16 tensor-core Gram blocks: with integer data in [0, 3] every product
    and every partial sum is an exact float32 integer, so the expansion
    |x|^2 + |y|^2 - 2 x.y equals the difference form and the iteration must
    match the oracle bit for bit."""
    x = _int_data(n, d, 4, seed=d)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 3, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=5, graph=(ids0, new0), iter=0, flags=knng.FLAG_BF16) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        assert c.stats()["set_overflow"] == 0
    st = oracle.State(x, K, rho, seed=5)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]


def test_bf16_build_recall_and_rerank_on_mnist_shaped_data():
    """bf16 dots with float32 re-rank on MNIST-shaped integer data (0..255,
    mostly zeros): recall within 0.005 of the float32 build, and every
    returned distance the float32 difference form (1e-4 of float64)."""
    x = workloads.mnist_like(6000, 784, seed=1)
    rows = np.random.default_rng(2).choice(len(x), 400, replace=False)
    ei, _ = oracle.bruteforce(x, 20, rows)
    fi, fd, _ = knng.knng_build(_cuda(x), 20, 0.5, 0.001, 15, seed=0)
    bi, bd, st = knng.knng_build(_cuda(x), 20, 0.5, 0.001, 15, seed=0, flags=knng.FLAG_BF16)
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    assert metrics.check_graph(x, bi, bd, rows=rows) == []
    rf, rb = metrics.recall(x, fi.cpu().numpy(), ei, rows), metrics.recall(x, bi, ei, rows)
    assert rb >= rf - 0.005, (rb, rf)


def test_several_iterations_match_oracle_bit_exact():
    n, d, K, rho = 4000, 8, 12, 0.5
    x = _int_data(n, d, 10, seed=5)
    st = oracle.State(x, K, rho, seed=3)
    st.init_random()
    with knng.Context(_cuda(x), K, rho=rho, seed=3) as c:
        for it in range(6):
            conv, ch = c.iterate()
            r = st.iterate()
            gi, gd, gf = c.state()
            oi, od, of = st.state()
            assert (gi == oi).all() and (gd == od).all() and (gf == of).all(), f"iteration {it + 1}"
            assert ch == r["changes"]


# ------------------------------------------------------------ Algorithm 1 ----

def test_alg1_golden_on_gpu():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "alg1_line5.json")))
    x = np.array(g["points_1d"], np.float32)[:, None]
    lists = np.array(g["lists"], np.int32)
    for rd, flag in (("a", knng.FLAG_REORDER), ("b", knng.FLAG_REORDER | knng.FLAG_REORDER_B)):
        with knng.Context(_cuda(x), g["K"], rho=1.0, flags=flag,
                          graph=(lists, np.ones_like(lists, np.uint8))) as c:
            c.reorder()
            assert c.permutation().tolist() == g[f"sigma_reading_{rd}"]


@pytest.mark.parametrize("reading_b,K", [(False, 10), (True, 10), (False, 40), (True, 64)])
def test_alg1_matches_oracle(reading_b, K):
    n = 6000
    x = _int_data(n, 6, 20, seed=9)
    ei, _ = oracle.bruteforce(x, K)
    flags = knng.FLAG_REORDER | (knng.FLAG_REORDER_B if reading_b else 0)
    with knng.Context(_cuda(x), K, rho=1.0, flags=flags, graph=(ei, np.ones_like(ei, np.uint8))) as c:
        c.reorder()
        sg = c.permutation()
        gi, gd, _ = c.state()
    osg, osi = oracle.greedy_reorder(ei, reading_b)
    assert (sg == osg).all()
    # lists were moved to their new spots with renamed ids
    ri = osg[ei]
    for u in range(0, n, 97):
        assert set(gi[osg[u]].tolist()) == set(ri[u].tolist())


def test_build_with_reorder_matches_oracle_bit_exact():
    n, d, K = 3000, 8, 10
    x = _int_data(n, d, 12, seed=21)
    gi, gd, st = knng.knng_build(_cuda(x), K, rho=0.5, delta=0.002, max_iters=8, seed=4, flags=knng.FLAG_REORDER)
    oi, od, ost = oracle.build_knng(x, K, 0.5, 0.002, 8, seed=4, reorder=1)
    assert st["reordered"] == 1 and ost["reordered"]
    assert st["iterations"] == ost["iters"]
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


def test_build_plain_matches_oracle_bit_exact():
    n, d, K = 5000, 6, 16
    x = _int_data(n, d, 9, seed=2)
    gi, gd, st = knng.knng_build(_cuda(x), K, rho=0.5, delta=0.001, max_iters=12, seed=9)
    oi, od, ost = oracle.build_knng(x, K, 0.5, 0.001, 12, seed=9)
    assert st["iterations"] == ost["iters"] and st["dist_evals"] == ost["evals"]
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


@pytest.mark.parametrize("pool", ["1", "40"])
def test_wide_lists_bucket_overflow_and_builds_match_oracle(pool, monkeypatch):
    """K = 64 (two keys per lane): a tiny proposal pool drives proposals
    through poisoned runs and locked insertions into 64-entry lists, one
    iteration bit-exact against the oracle; then a whole K = 48 build and a
    relabelled K = 40 build equal the oracle's."""
    monkeypatch.setenv("KNNG_TEST_BUCKET_POOL_CHUNKS", pool)
    n, d, K, rho, hi = 1500, 3, 64, 0.15, 8
    x = _int_data(n, d, hi, seed=n)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    assert stats["bucket_overflow"] > 0 and stats["lock_timeouts"] == 0 and stats["set_overflow"] == 0
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]
    monkeypatch.delenv("KNNG_TEST_BUCKET_POOL_CHUNKS")
    x = _int_data(3000, 6, 9, seed=3)
    gi, gd, st = knng.knng_build(_cuda(x), 48, rho=0.2, delta=0.001, max_iters=10, seed=9)
    oi, od, ost = oracle.build_knng(x, 48, 0.2, 0.001, 10, seed=9)
    assert st["iterations"] == ost["iters"] and st["set_overflow"] == 0
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()
    x = _int_data(2500, 8, 12, seed=21)
    gi, gd, st = knng.knng_build(_cuda(x), 40, rho=0.25, delta=0.002, max_iters=8, seed=4, flags=knng.FLAG_REORDER)
    oi, od, ost = oracle.build_knng(x, 40, 0.25, 0.002, 8, seed=4, reorder=1)
    assert st["reordered"] == 1 and st["iterations"] == ost["iters"]
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


def test_wide_lists_real_data_recall_batched_and_refusals():
    """K = 64 on real-valued clustered data: list invariants and every
    distance within 1e-4 of its float64 recomputation, recall within 0.005 of
    the oracle's build; a batched K = 48 build equals the single builds; the
    flags that keep one key per lane refuse K > 32."""
    x = workloads.gaussian_mixture(6000, 24, 15, seed=8)
    gi, gd, st = knng.knng_build(_cuda(x), 64, 0.3, 0.001, 10, seed=2)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert metrics.check_graph(x, gi, gd) == []
    rows = np.arange(0, 6000, 7)
    ei, _ = oracle.bruteforce(x, 64, rows)
    oi, _, _ = oracle.build_knng_mt(x, 64, 0.3, 0.001, 10, seed=2)
    assert abs(metrics.recall(x, gi, ei, rows) - metrics.recall(x, oi, ei, rows)) <= 0.005
    sets = [workloads.gaussian_mixture(n, d, 6, seed=n) for n, d in [(2000, 24), (1500, 70), (2500, 24)]]
    outs, _ = knng.knng_build_batched([_cuda(v) for v in sets], 48, 0.25, 0.001, 8, seed=5)
    for v, (bi, bd) in zip(sets, outs):
        si, sd, _ = knng.knng_build(_cuda(v), 48, 0.25, 0.001, 8, seed=5)
        assert torch.equal(bi, si) and torch.equal(bd, sd)
    for flag in (knng.FLAG_BF16, knng.FLAG_FP8, knng.FLAG_HEAP_SAMPLING):
        with pytest.raises(knng.KnngError):
            knng.knng_build(_cuda(sets[1]), 40, 0.5, 0.001, 4, seed=0, flags=flag)


# ------------------------------------------------------- whole builds ----

def test_uniform_n2k_recall_and_invariants():
    """2,000 uniform points in [0,1)^8, K=10, rho=1, delta=0.001, 10 iterations."""
    w, x = workloads.make("uniform_n2k_d8")
    ei, _ = oracle.bruteforce(x, w.K)
    gi, gd, st = knng.knng_build(_cuda(x), w.K, w.rho, w.delta, w.max_iters, seed=0)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert metrics.check_graph(x, gi, gd) == []
    oi, od, ost = oracle.build_knng(x, w.K, w.rho, w.delta, w.max_iters, seed=0, count_mode="inplace")
    rg, ro = metrics.recall(x, gi, ei), metrics.recall(x, oi, ei)
    assert rg >= 0.99
    assert abs(rg - ro) <= 0.005


@pytest.mark.parametrize("flags", [0, knng.FLAG_REORDER, knng.FLAG_BF16])
def test_graph_capture_gives_the_same_graph(flags):
    """The captured-graph loop and one-by-one launches build the same graph,
    also with the relabelling and bf16 staging inside the captured loop."""
    d = 72 if flags == knng.FLAG_BF16 else 16
    x = workloads.gaussian_mixture(4000, d, 12, seed=6)
    a_i, a_d, sa = knng.knng_build(_cuda(x), 12, 0.5, 0.001, 10, seed=1, flags=flags)
    b_i, b_d, sb = knng.knng_build(_cuda(x), 12, 0.5, 0.001, 10, seed=1, flags=flags | knng.FLAG_GRAPH)
    assert (a_i.cpu().numpy() == b_i.cpu().numpy()).all() and (a_d.cpu().numpy() == b_d.cpu().numpy()).all()
    assert sa["iterations"] == sb["iterations"] and sa["dist_evals"] == sb["dist_evals"]


def test_host_and_device_pointers_agree():
    x = workloads.gaussian_mixture(3000, 16, 10, seed=1)
    hi, hd, _ = knng.knng_build(x, 10, 0.5, 0.001, 8, seed=2)             # host in/out
    di, dd, _ = knng.knng_build(_cuda(x), 10, 0.5, 0.001, 8, seed=2)      # device in/out
    assert (hi == di.cpu().numpy()).all() and (hd == dd.cpu().numpy()).all()


def test_complete_graph_k_equals_n_minus_1():
    x = workloads.uniform(33, 4, seed=3)
    gi, gd, st = knng.knng_build(_cuda(x), 32, 1.0, 0.0, 2, seed=0)
    oi, od = oracle.bruteforce(x, 32)
    assert_ids_up_to_ties(gi.cpu().numpy(), gd.cpu().numpy(), oi, od)


@pytest.mark.parametrize("n,K", [(65, 64), (34, 33), (50, 40)])
def test_complete_graph_wide_lists(n, K):
    """K = n - 1 with two keys per lane: the random init already lists
    every other point, so the result is the exact K-NNG."""
    x = workloads.uniform(n, 5, seed=n)
    gi, gd, st = knng.knng_build(_cuda(x), K, 1.0, 0.0, 2, seed=1)
    oi, od = oracle.bruteforce(x, K)
    assert_ids_up_to_ties(gi.cpu().numpy(), gd.cpu().numpy(), oi, od)


def test_wide_lists_k33_iteration_relabels_and_mixed_batch():
    """K = 33 (a single entry in the second half of each lane pair): one
    iteration bit-exact against the oracle; K = 64 lists through the parallel
    relabelling keep a valid graph in the caller's labels; a batched call
    with K = 20 and K = 50 data sets equals their single builds."""
    n, d, K, rho = 1500, 6, 33, 0.3
    x = _int_data(n, d, 8, seed=33)
    ids0, new0 = workloads.random_graph(n, K, seed=34, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=5, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    st = oracle.State(x, K, rho, seed=5)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    assert stats["set_overflow"] == 0
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]
    y = workloads.gaussian_mixture(5000, 12, 10, seed=2)
    flags = knng.FLAG_REORDER | knng.FLAG_REORDER_PARALLEL
    ri, rd, rst = knng.knng_build(_cuda(y), 64, 0.25, 0.001, 8, seed=3, flags=flags)
    assert rst["reordered"] == 1
    assert metrics.check_graph(y, ri.cpu().numpy(), rd.cpu().numpy()) == []
    sets = [workloads.gaussian_mixture(m, 24, 6, seed=m) for m in (1800, 2600)]
    items = [dict(data=_cuda(sets[0]), K=20, rho=0.5, delta=0.001, max_iters=8, seed=1),
             dict(data=_cuda(sets[1]), K=50, rho=0.25, delta=0.001, max_iters=8, seed=1)]
    outs, _ = knng.knng_build_batched_ex(items)
    for it, (bi, bd) in zip(items, outs):
        si, sd, _ = knng.knng_build(it["data"], it["K"], it["rho"], it["delta"], it["max_iters"], seed=it["seed"])
        assert torch.equal(bi, si) and torch.equal(bd, sd)


def test_all_points_equal():
    x = np.ones((500, 8), np.float32)
    gi, gd, st = knng.knng_build(_cuda(x), 10, 0.5, 0.0, 3, seed=0)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert (gd == 0).all()
    assert metrics.check_graph(x, gi, gd) == []


def test_clustered_n100k_full_size_sampled_parity():
    """The benchmark's workload and launch configuration: 100,000 points, 16
    dims, 50 clusters, K=20, rho=0.5, delta=0.001, 15 iterations.  Recall on
    2,000 sampled rows (oracle brute force, one row at a time) must be >= the
    oracle's recall - 0.005; sampled distances within 1e-4 of float64."""
    w, x = workloads.make("clustered_n100k_d16")
    rows = np.random.default_rng(0).choice(w.n, 2000, replace=False)
    ei, _ = oracle.bruteforce(x, w.K, rows)
    gi, gd, st = knng.knng_build(_cuda(x), w.K, w.rho, w.delta, w.max_iters, seed=0)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert metrics.check_graph(x, gi, gd, rows=rows) == []
    oi, od, ost = oracle.build_knng(x, w.K, w.rho, w.delta, w.max_iters, seed=0, count_mode="inplace")
    rg = metrics.recall(x, gi, ei, rows)
    ro = metrics.recall(x, oi, ei, rows)
    assert rg >= ro - 0.005, (rg, ro)
    assert st["lock_timeouts"] == 0


# ---------------------------------------------------------------- batched ----

def test_batched_matches_oracle_per_data_set_bit_exact():
    """Many data sets (different n and d, incl. rows below and above 64
    floats) in one batched build: each result equals the oracle's build of
    that data set alone, bit for bit (integer data)."""
    g = np.random.default_rng(4)
    sets = []
    for b, (n, d) in enumerate([(700, 8), (1500, 3), (400, 96), (2100, 16), (333, 130), (50, 5)]):
        sets.append(_int_data(n, d, 6, seed=100 + b))
    K, rho, delta, iters = 8, 0.5, 0.002, 8
    outs, st = knng.knng_build_batched([_cuda(x) for x in sets], K, rho, delta, iters, seed=3)
    for x, (gi, gd) in zip(sets, outs):
        oi, od, ost = oracle.build_knng(x, K, rho, delta, iters, seed=3)
        assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


def test_batched_equals_single_builds_float_data():
    sets = [workloads.gaussian_mixture(n, d, 7, seed=n) for n, d in [(3000, 32), (1200, 96), (5000, 128), (800, 32)]]
    outs, st = knng.knng_build_batched(sets, 16, 0.5, 0.001, 15, seed=9)     # host in / host out
    for x, (bi, bd) in zip(sets, outs):
        si, sd, _ = knng.knng_build(_cuda(x), 16, 0.5, 0.001, 15, seed=9)
        assert (bi == si.cpu().numpy()).all() and (bd == sd.cpu().numpy()).all()


# -------------------------------------------------------------- autotuner ----

def test_batched_ex_per_data_set_parameters_equal_single_builds():
    """knng_build_batched_ex with K, rho, delta, max_iters and seed per data
    set: data sets that share (width class, K, sample size, max_iters, seed)
    run together with their own delta, the others in runs of their own; every
    result equals that data set's own build bit for bit."""
    params = [(3000, 24, 16, 0.5, 0.001, 8, 1), (2500, 24, 16, 0.5, 0.01, 8, 1), (2000, 24, 16, 0.52, 0.0, 8, 1),
              (1800, 72, 20, 0.6, 0.001, 6, 7), (2200, 72, 12, 1.0, 0.002, 10, 3), (900, 150, 8, 0.3, 0.001, 5, 0),
              (1200, 24, 32, 0.7, 0.001, 8, 1)]
    items, sets = [], []
    for b, (n, d, K, rho, delta, it, seed) in enumerate(params):
        x = _cuda(workloads.gaussian_mixture(n, d, 8, seed=50 + b))
        sets.append(x)
        items.append(dict(data=x, K=K, rho=rho, delta=delta, max_iters=it, seed=seed))
    outs, st = knng.knng_build_batched_ex(items)
    assert st["lock_timeouts"] == 0
    for it, (bi, bd) in zip(items, outs):
        si, sd, _ = knng.knng_build(it["data"], it["K"], it["rho"], it["delta"], it["max_iters"], seed=it["seed"])
        assert torch.equal(bi, si) and torch.equal(bd, sd), (it["K"], it["rho"], it["delta"])


def test_autotuned_builds_equal_default_builds():
    """KNNG_FLAG_AUTOTUNE times every eligible join kernel on the first
    iteration, undoes each trial and keeps the fastest: the graph is the same
    bit for bit (every kernel computes the same pairs and keys), and the
    second build of the geometry reuses the choice."""
    x = workloads.gaussian_mixture(5000, 48, 15, seed=9)
    ref_i, ref_d, _ = knng.knng_build(_cuda(x), 16, 0.5, 0.001, 8, seed=4)
    a_i, a_d, sa = knng.knng_build(_cuda(x), 16, 0.5, 0.001, 8, seed=4, flags=knng.FLAG_AUTOTUNE)
    b_i, b_d, sb = knng.knng_build(_cuda(x), 16, 0.5, 0.001, 8, seed=4, flags=knng.FLAG_AUTOTUNE)
    assert torch.equal(a_i, ref_i) and torch.equal(a_d, ref_d)
    assert torch.equal(b_i, ref_i) and torch.equal(b_d, ref_d)
    assert sa["join_path"] in (0, 1, 2, 3, 4) and sb["join_path"] == sa["join_path"]
    # the tuning build ran three trial joins on top of the real ones
    assert sa["kernel_launches"] > sb["kernel_launches"]


def test_autotuned_bf16_and_batched_match_the_oracle():
    x = _int_data(900, 96, 4, seed=96)
    ids0, new0 = workloads.random_graph(900, 16, seed=97, p_new=0.6)
    with knng.Context(_cuda(x), 16, rho=0.5, seed=5, graph=(ids0, new0), iter=0,
                      flags=knng.FLAG_BF16 | knng.FLAG_AUTOTUNE) as c:
        c.iterate()
        gi, gd, gf = c.state()
    st = oracle.State(x, 16, 0.5, seed=5)
    st.init_graph(ids0, new0, 0)
    st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    sets = [_int_data(n, d, 4, seed=n) for n, d in [(700, 20), (1500, 40), (900, 100)]]
    outs, _ = knng.knng_build_batched([_cuda(s) for s in sets], 10, 0.5, 0.001, 6, seed=2, flags=knng.FLAG_AUTOTUNE)
    for s, (bi, bd) in zip(sets, outs):
        oi, od, _ = oracle.build_knng(s, 10, 0.5, 0.001, 6, seed=2)
        assert (bi.cpu().numpy() == oi).all()


# ------------------------------------------------- priority-heap sampling ----

HEAP_CASES = [
    # n, d, K, rho, int range (ragged warps, s < K and s = K, high reverse degrees)
    (3001, 8, 10, 0.5, 16),
    (2500, 16, 20, 0.3, 8),
    (1200, 17, 32, 1.0, 5),
    (700, 100, 12, 0.5, 3),
]


@pytest.mark.parametrize("n,d,K,rho,hi", HEAP_CASES)
def test_heap_sampling_one_iteration_matches_oracle_bit_exact(n, d, K, rho, hi):
    """KNNG_FLAG_HEAP_SAMPLING from a given graph: the kept candidate sets,
    the lists, the flags and the counters equal the oracle's priority-heap
    iteration exactly."""
    x = _int_data(n, d, hi, seed=n + 7)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 8, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=13, graph=(ids0, new0), iter=0,
                      flags=knng.FLAG_HEAP_SAMPLING) as c:
        conv, ch = c.iterate()
        gnew, gold = c.samples()
        gi, gd, gf = c.state()
        stats = c.stats()
    st = oracle.State(x, K, rho, seed=13, sampler="heap")
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    s = oracle.sample_size(rho, K)
    onew, oold = st.samples()
    assert stats["rev_overflow"] == 0 and stats["set_overflow"] == 0
    for u in range(n):
        assert len(gnew[u]) <= s and len(gold[u]) <= s
        assert set(gnew[u].tolist()) == set(onew[u].tolist())
        assert set(gold[u].tolist()) == set(oold[u].tolist())
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"] and stats["dist_evals"] == r["evals"]


@pytest.mark.parametrize("flags", [0, knng.FLAG_GRAPH])
def test_heap_sampling_build_matches_oracle_bit_exact(flags):
    n, d, K = 4000, 6, 16
    x = _int_data(n, d, 9, seed=31)
    gi, gd, st = knng.knng_build(_cuda(x), K, rho=0.5, delta=0.001, max_iters=12, seed=6,
                                 flags=knng.FLAG_HEAP_SAMPLING | flags)
    oi, od, ost = oracle.build_knng(x, K, 0.5, 0.001, 12, seed=6, sampler="heap")
    assert st["iterations"] == ost["iters"] and st["dist_evals"] == ost["evals"]
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


def test_heap_sampling_batched_matches_oracle_per_data_set():
    sets = [_int_data(n, d, 6, seed=200 + n) for n, d in [(700, 8), (1500, 3), (400, 96), (60, 5)]]
    K, rho, delta, iters = 8, 0.5, 0.002, 8
    outs, _ = knng.knng_build_batched([_cuda(x) for x in sets], K, rho, delta, iters, seed=5,
                                      flags=knng.FLAG_HEAP_SAMPLING)
    for x, (gi, gd) in zip(sets, outs):
        oi, od, _ = oracle.build_knng(x, K, rho, delta, iters, seed=5, sampler="heap")
        assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


# ------------------------------------------- parallel relabelling variant ----

def _contiguous(levels, sigma):
    for lv in levels:
        order = np.argsort(lv, kind="stable")
        pos = sigma[order]
        for seg in np.split(pos, np.flatnonzero(np.diff(lv[order])) + 1):
            if seg.max() - seg.min() + 1 != len(seg):
                return False
    return True


@pytest.mark.parametrize("n,d,K,hi", [(3000, 4, 8, 6), (20000, 8, 16, 5), (777, 17, 5, 3)])
def test_parallel_relabel_matches_oracle_hierarchy(n, d, K, hi):
    """KNNG_FLAG_REORDER_PARALLEL on given lists (integer data, so the float32
    distances and their ties equal the oracle's): sigma is a permutation in
    which every component of every round of the oracle's single-linkage
    hierarchy is contiguous, and the lists moved to their new spots."""
    x = _int_data(n, d, hi, seed=n + 3)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 4, p_new=1.0)
    flags = knng.FLAG_REORDER | knng.FLAG_REORDER_PARALLEL
    with knng.Context(_cuda(x), K, rho=1.0, flags=flags, graph=(ids0, new0)) as c:
        c.reorder()
        sg = c.permutation()
        gi, _, _ = c.state()
    levels, _, _ = oracle.parallel_relabel(x, ids0)
    assert sorted(sg.tolist()) == list(range(n))
    assert _contiguous(levels, sg)
    ri = sg[ids0]
    for u in range(0, n, 37):
        assert set(gi[sg[u]].tolist()) == set(ri[u].tolist())


def test_parallel_relabel_builds_and_periodic_relabels():
    """Whole builds with the parallel variant after iteration 1 reach the
    plain build's recall (within 0.005), and relabelling again every two
    iterations through the step API keeps a valid graph in the caller's
    labels."""
    x, lab = workloads.gaussian_mixture(30000, 16, 20, seed=8, return_labels=True)
    K = 16
    rows = np.random.default_rng(0).choice(len(x), 1500, replace=False)
    ei, _ = knng.knng_bruteforce(_cuda(x), K, rows=torch.from_numpy(rows).cuda())
    ei = ei.cpu().numpy()
    pi, pd, _ = knng.knng_build(_cuda(x), K, 0.5, 0.001, 12, seed=3)
    flags = knng.FLAG_REORDER | knng.FLAG_REORDER_PARALLEL
    ri, rd, st = knng.knng_build(_cuda(x), K, 0.5, 0.001, 12, seed=3, flags=flags)
    assert st["reordered"] == 1
    rp = metrics.recall(x, pi.cpu().numpy(), ei, rows)
    rr = metrics.recall(x, ri.cpu().numpy(), ei, rows)
    assert rr >= rp - 0.005
    assert metrics.check_graph(x, ri.cpu().numpy(), rd.cpu().numpy()) == []
    with knng.Context(_cuda(x), K, rho=0.5, seed=3, flags=flags) as c:
        for it in range(8):
            c.iterate()
            if it % 2 == 1:
                c.reorder()
        gi, gd = c.get(device=False)
        sg = c.permutation()
    assert sorted(sg.tolist()) == list(range(len(x)))
    assert metrics.check_graph(x, gi, gd) == []
    assert metrics.recall(x, gi, ei, rows) >= rp - 0.01


# ------------------------------------------------------------ edge cases ----

@pytest.mark.parametrize("n,d,K,rows", [
    (50, 3, 1, None),          # one query tile, one point tile, K = 1
    (4096, 1, 5, None),        # d = 1 (one 16-wide bf16 k-block, 15 zero columns)
    (5000, 125, 32, [7]),      # a single query row, rows padded to 128 columns
    (6000, 16, 10, [3, 3, 5999, 0, 3]),  # repeated query rows
])
def test_tensor_core_bruteforce_edges(n, d, K, rows, monkeypatch):
    x = workloads.gaussian_mixture(n, d, 7, seed=n + d)
    r = None if rows is None else torch.tensor(rows, dtype=torch.int64, device="cuda")
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "tensor")
    ti, td = knng.knng_bruteforce(_cuda(x), K, rows=r)
    assert knng.bruteforce_last_fallbacks() >= 0
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "cuda")
    ci, cd = knng.knng_bruteforce(_cuda(x), K, rows=r)
    assert torch.equal(ti, ci) and torch.equal(td, cd)


def test_tensor_core_bruteforce_identical_points(monkeypatch):
    """All points equal: every distance is 0, the answer is the K smallest
    ids other than the query, and no bound can separate the candidates (the
    exact kernel redoes what the bound cannot certify)."""
    x = np.ones((5000, 24), np.float32)
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "tensor")
    ti, td = knng.knng_bruteforce(_cuda(x), 8)
    monkeypatch.setenv("KNNG_TEST_BF_PATH", "cuda")
    ci, cd = knng.knng_bruteforce(_cuda(x), 8)
    assert torch.equal(ti, ci) and torch.equal(td, cd) and float(td.abs().max()) == 0.0


@pytest.mark.parametrize("n,K,rho", [(3, 1, 1.0), (200, 1, 0.5), (500, 12, 0.05)])
def test_heap_sampling_small_cases_match_oracle(n, K, rho):
    x = _int_data(n, 3, 7, seed=n)
    gi, gd, st = knng.knng_build(_cuda(x), K, rho=rho, delta=0.0, max_iters=5, seed=2,
                                 flags=knng.FLAG_HEAP_SAMPLING)
    oi, od, ost = oracle.build_knng(x, K, rho, 0.0, 5, seed=2, sampler="heap")
    assert st["iterations"] == ost["iters"]
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()


def test_parallel_relabel_edges():
    """n = 2; two disconnected halves (each list points into its own half);
    all points equal (every distance ties, so ids decide)."""
    flags = knng.FLAG_REORDER | knng.FLAG_REORDER_PARALLEL
    cases = []
    cases.append((np.array([[0.0], [1.0]], np.float32), np.array([[1], [0]], np.int32)))
    n, K = 400, 4
    g = np.random.default_rng(5)
    ids = np.empty((n, K), np.int32)
    for u in range(n):
        lo = 0 if u < n // 2 else n // 2
        ids[u] = lo + g.choice([v for v in range(n // 2) if lo + v != u], K, replace=False)
    cases.append((_int_data(n, 2, 4, seed=1), ids))
    ids2, _ = workloads.random_graph(300, 5, seed=9, p_new=1.0)
    cases.append((np.zeros((300, 4), np.float32), ids2))
    for x, ids in cases:
        n, K = ids.shape
        with knng.Context(_cuda(x), K, rho=1.0, flags=flags, graph=(ids, np.ones_like(ids, np.uint8))) as c:
            c.reorder()
            sg = c.permutation()
        levels, _, _ = oracle.parallel_relabel(x, ids)
        assert sorted(sg.tolist()) == list(range(n))
        assert _contiguous(levels, sg)
        if n == 400:
            assert len(np.unique(levels[-1])) == 2
            assert set(sg[: n // 2].tolist()) in (set(range(n // 2)), set(range(n // 2, n)))


@pytest.mark.parametrize("path", ["warp", "tile", "ring", "pipe"])
@pytest.mark.parametrize("passes,pool", [(3, None), (5, "1")])
def test_join_in_node_range_passes_matches_oracle_bit_exact(path, passes, pool, monkeypatch):
    """An iteration's join split into node-range passes, each followed by a
    list merge (what large sample rates use so that one pass's proposals fit
    the buckets): by reading 6 the lists end the same, and the change count --
    merges and locked insertions each adding the entries they made new --
    equals the oracle's batched count.  With a one-chunk pool the passes also
    run through poisoned runs and locked insertions."""
    monkeypatch.setenv("KNNG_TEST_JOIN_PATH", path)
    monkeypatch.setenv("KNNG_TEST_JOIN_PASSES", str(passes))
    if pool:
        monkeypatch.setenv("KNNG_TEST_BUCKET_POOL_CHUNKS", pool)
    n, d, K, rho, hi = 1800, 8 if path == "warp" else 70, 16, 0.5, 3
    x = _int_data(n, d, hi, seed=n + d)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    assert stats["join_path"] == PATH_IDS[path]
    assert stats["set_overflow"] == 0 and stats["lock_timeouts"] == 0
    if pool:
        assert stats["bucket_overflow"] > 0
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]
    assert stats["dist_evals"] == r["evals"]


@pytest.mark.parametrize("shape", ["pipe", "pipe8"])
@pytest.mark.parametrize("n,d,K,rho", [(2000, 200, 20, 1.0), (1500, 33, 16, 0.5)])
def test_pipelined_join_block_shapes_match_oracle_bit_exact(shape, n, d, K, rho, monkeypatch):
    """The pipelined kernel's two block shapes (four warps with one row slot,
    eight warps with two) give the same iteration, bit for bit against the
    oracle."""
    monkeypatch.setenv("KNNG_TEST_JOIN_PATH", shape)
    x = _int_data(n, d, 3, seed=n + d)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    assert stats["join_path"] == PATH_IDS[shape] and stats["set_overflow"] == 0
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]


@pytest.mark.parametrize("n,d,K,rho,bf16", [(900, 1600, 16, 0.5, False), (900, 2000, 16, 0.5, True),
                                            (700, 3144, 12, 0.5, False)])
def test_wide_rows_match_oracle_bit_exact(n, d, K, rho, bf16):
    """Row widths the dimension sweep times (up to the paper's d = 3144),
    beyond the ring and pipelined kernels: the block-per-node tile kernel in
    float32 and with bf16 tensor-core Gram blocks, one iteration bit-exact
    against the oracle on small integers (every product and partial sum
    exact in float32, so the bf16 expansion equals the difference form)."""
    x = _int_data(n, d, 3, seed=d)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 5, p_new=0.6)
    flags = knng.FLAG_BF16 if bf16 else 0
    with knng.Context(_cuda(x), K, rho=rho, seed=13, graph=(ids0, new0), iter=0, flags=flags) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    assert stats["join_path"] == PATH_IDS["tile"]
    assert stats["set_overflow"] == 0 and stats["lock_timeouts"] == 0
    st = oracle.State(x, K, rho, seed=13)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]


@pytest.mark.parametrize("n,d,K,rho", [(1200, 64, 16, 0.5), (800, 150, 20, 1.0), (600, 128, 32, 0.3),
                                       (900, 784, 20, 0.5)])
def test_fp8_tensor_core_join_exact_on_small_integers(n, d, K, rho):
    """FP8 (e4m3) Gram blocks on the tensor cores: integers up to 15 are exact
    in e4m3 (four significant bits) and every product and partial sum is an
    exact float32 integer, so |x|^2 + |y|^2 - 2 x.y equals the difference form
    and the iteration matches the oracle bit for bit."""
    x = _int_data(n, d, 16, seed=d + 1)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 7, p_new=0.6)
    with knng.Context(_cuda(x), K, rho=rho, seed=5, graph=(ids0, new0), iter=0, flags=knng.FLAG_FP8) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        stats = c.stats()
    assert stats["join_path"] == PATH_IDS["ring"] and stats["set_overflow"] == 0
    st = oracle.State(x, K, rho, seed=5)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]


def test_fp8_build_rounds_large_values_and_stays_valid():
    """Above 16 e4m3 keeps four significant bits (17 rounds to 16, 255 to 256),
    so on 0..255 data the FP8 join ranks pairs by rounded distances: the
    build still returns valid lists whose distances are the float32
    difference form of the original points (the output is re-ranked), and
    its recall is below the float32 build's, by the rounding (measured about
    0.04 on the MNIST-shaped workload)."""
    x = workloads.mnist_like(3000, 784, seed=3)
    xd = _cuda(x)
    oi, _ = oracle.bruteforce(x, 10)
    fi, fd, fst = knng.knng_build(xd, 10, 0.5, 0.001, 10, seed=1, flags=knng.FLAG_FP8)
    gi, gd, _ = knng.knng_build(xd, 10, 0.5, 0.001, 10, seed=1)
    fi, fd, gi = fi.cpu().numpy(), fd.cpu().numpy(), gi.cpu().numpy()
    assert fst["join_path"] == PATH_IDS["ring"]
    assert metrics.check_graph(x, fi, fd) == []
    r8, r32 = metrics.recall(x, fi, oi), metrics.recall(x, gi, oi)
    assert 0.8 <= r8 < r32, (r8, r32)
