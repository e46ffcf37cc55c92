"""The full-size workloads, in the launch configuration bench.py times
(knng_build with each workload's parameters, seed 0), against the oracle.

At full size the checks are:
- the GPU brute force equals the oracle's brute force on sampled rows (ids up
  to ties), so it serves as the ground truth of recall on more rows;
- list invariants and every returned distance within 1e-4 relative of its
  float64 recomputation (the accuracy audit), on the recall rows;
- recall@K within 0.005 of the oracle's NN-Descent at the same rho, delta,
  iteration cap and seed (the tolerance of the method's parity).  The oracle
  runs here, in batched mode on every host core, where that takes seconds;
  for the 1,000,000 x 128 mixture (minutes of host time) its recall comes
  from tests/golden/oracle_recall.json, written by make_oracle_recall.py with
  the oracle alone, after checking that the inputs and the oracle sources are
  the ones it was computed from;
- the bf16 tensor-core form against the float32 path: within 0.005 where its
  rounding is small against the spacing of neighbour distances; on the
  1,000,000 x 128 mixture it is not (the measured gap is asserted as such).
"""
import hashlib
import json
import os

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

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RECALL_ROWS, ROWS_SEED = 2000, 7
PARITY = 0.005


def recall_rows(n):
    return np.sort(np.random.Generator(np.random.PCG64(ROWS_SEED)).choice(n, RECALL_ROWS, replace=False))


def _golden(case, x):
    db = json.load(open(os.path.join(GOLDEN, "oracle_recall.json")))
    rec = db[case]
    assert hashlib.sha256(np.ascontiguousarray(x).tobytes()).hexdigest()[:16] == rec["data_sha256_16"], \
        "inputs differ from the ones the stored oracle recall was computed on"
    h = hashlib.sha256()
    for f in ("knng_oracle.c", "metrics.py"):
        h.update(open(os.path.join(os.path.dirname(oracle.__file__), f), "rb").read())
    assert h.hexdigest()[:16] == rec["oracle_sha256_16"], "the oracle changed since the stored recall was written"
    assert rec["recall_rows"] == RECALL_ROWS and rec["rows_seed"] == ROWS_SEED
    return rec


def _ground_truth(x, xd, K, rows, oracle_rows=12):
    """GPU brute force on the recall rows, checked against the oracle's brute
    force on the first `oracle_rows` of them."""
    bi, bd = knng.knng_bruteforce(xd, K, rows=torch.from_numpy(rows).cuda())
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    oi, od = oracle.bruteforce(x, K, rows[:oracle_rows])
    np.testing.assert_allclose(bd[:oracle_rows], od, rtol=1e-5, atol=1e-7)
    mism = bi[:oracle_rows] != oi
    assert np.allclose(bd[:oracle_rows][mism], od[mism], rtol=1e-5, atol=1e-7)
    return bi


def _gpu_recall(x, xd, w, rho, delta, iters, rows, exact, flags=0):
    gi, gd, st = knng.knng_build(xd, w.K, rho, delta, iters, seed=0, flags=flags)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert metrics.check_graph(x, gi, gd, rows=rows) == []
    assert st["lock_timeouts"] == 0
    return metrics.recall(x, gi, exact, rows), st


def _live_case(name, bf16_tol):
    w, x = workloads.make(name)
    xd = torch.from_numpy(x).cuda()
    rows = recall_rows(w.n)
    exact = _ground_truth(x, xd, w.K, rows)
    oi, _, ost = oracle.build_knng_mt(x, w.K, w.rho, w.delta, w.max_iters, seed=0)
    r_orc = metrics.recall(x, oi, exact, rows)
    r_gpu, st = _gpu_recall(x, xd, w, w.rho, w.delta, w.max_iters, rows, exact)
    assert st["set_overflow"] == 0 and st["rev_overflow"] == 0
    assert abs(r_gpu - r_orc) <= PARITY, (r_gpu, r_orc)
    if bf16_tol is not None:
        r_bf, _ = _gpu_recall(x, xd, w, w.rho, w.delta, w.max_iters, rows, exact, knng.FLAG_BF16)
        assert abs(r_bf - r_gpu) <= bf16_tol, (r_bf, r_gpu)
    return r_gpu, r_orc


def test_mnist_like_n70k_d784_full_size_vs_oracle():
    """70,000 x 784 MNIST-shaped integers, K=20, rho=0.5 (tile kernel in
    float32, ring kernel in bf16; integers up to 255 are exact in bf16)."""
    _live_case("mnist_like_n70k_d784", bf16_tol=PARITY)


def test_audio_like_n54k_d192_full_size_vs_oracle():
    """Audio-shaped 54,387 x 192, K=20, rho=0.5 (pipelined kernel in float32,
    ring kernel in bf16)."""
    _live_case("audio_like_n54k_d192", bf16_tol=PARITY)


def test_clustered_n100k_d16_full_size_vs_oracle():
    """The 100,000 x 16 clustered workload, K=20, rho=0.5 (warp kernel)."""
    _live_case("clustered_n100k_d16", bf16_tol=None)


@pytest.mark.parametrize("case,rho,delta,iters", [
    ("mixture_n1m_d128", 0.3, 0.001, 12),
    ("mixture_n1m_d128_rho0.7_delta0.001_iters12", 0.7, 0.001, 12),
])
def test_mixture_n1m_d128_full_size_vs_stored_oracle(case, rho, delta, iters):
    """1,000,000 x 128, 1,000 clusters, K=32 (pipelined join kernel in
    float32, ring kernel in bf16): at the stated parameters and at the
    recall-0.99 operating point the benchmark times.  The bf16 form is measured beside it: its rounding of the points
    (about 1e-3 of a distance) is as large as the spacing of the 32nd and 33rd
    neighbour distances in this intrinsically 128-dimensional data, so it
    stays below float32 by more than the parity tolerance, and never more
    than 0.015."""
    w, x = workloads.make("mixture_n1m_d128")
    rec = _golden(case, x)
    assert (rec["rho"], rec["delta"], rec["max_iters"]) == (rho, delta, iters)
    xd = torch.from_numpy(x).cuda()
    rows = recall_rows(w.n)
    exact = _ground_truth(x, xd, w.K, rows)
    r_gpu, st = _gpu_recall(x, xd, w, rho, delta, iters, rows, exact)
    assert abs(r_gpu - rec["recall_at_k"]) <= PARITY, (r_gpu, rec["recall_at_k"])
    r_bf, _ = _gpu_recall(x, xd, w, rho, delta, iters, rows, exact, knng.FLAG_BF16)
    assert r_gpu - 0.015 <= r_bf <= r_gpu, (r_bf, r_gpu)


def test_batched_workload_slice_equals_single_builds():
    """32 data sets of the batched workload (every row-width class of it):
    the batched build equals each data set's own build bit for bit, and on
    the largest data set of each width its recall is the oracle's within the
    parity tolerance."""
    specs = workloads.batched_specs(256, 0)[:32]
    sets = [workloads.gaussian_mixture(s["n"], s["d"], s["clusters"], seed=s["seed"]) for s in specs]
    xs = [torch.from_numpy(x).cuda() for x in sets]
    cfg = workloads.BATCHED
    outs, st = knng.knng_build_batched(xs, cfg["K"], cfg["rho"], cfg["delta"], cfg["max_iters"], seed=0)
    assert st["lock_timeouts"] == 0
    for x, (bi, bd) in zip(xs, outs):
        si, sd, _ = knng.knng_build(x, cfg["K"], cfg["rho"], cfg["delta"], cfg["max_iters"], seed=0)
        assert torch.equal(bi, si) and torch.equal(bd, sd)
    # and against the oracle: the largest data set of each row width, recall
    # within the parity tolerance of the oracle's build at the same parameters
    for d in sorted({s["d"] for s in specs}):
        b = max((i for i, s in enumerate(specs) if s["d"] == d), key=lambda i: specs[i]["n"])
        x = sets[b]
        rows = np.random.default_rng(b).choice(len(x), min(1000, len(x)), replace=False)
        exact = _ground_truth(x, xs[b], cfg["K"], rows)
        oi, _, _ = oracle.build_knng_mt(x, cfg["K"], cfg["rho"], cfg["delta"], cfg["max_iters"], seed=0)
        r_gpu = metrics.recall(x, outs[b][0].cpu().numpy(), exact, rows)
        r_orc = metrics.recall(x, oi, exact, rows)
        assert abs(r_gpu - r_orc) <= PARITY, (d, r_gpu, r_orc)


@pytest.mark.parametrize("name,rho", [("mnist_like_n70k_d784", 0.6), ("audio_like_n54k_d192", 0.7)])
def test_recall_099_points_vs_oracle(name, rho):
    """The recall-0.99 operating points bench.py times for the MNIST- and
    audio-shaped workloads: the GPU reaches 0.99 and is within the parity
    tolerance of the oracle's build at the same parameters."""
    w, x = workloads.make(name)
    xd = torch.from_numpy(x).cuda()
    rows = recall_rows(w.n)
    exact = _ground_truth(x, xd, w.K, rows)
    oi, _, _ = oracle.build_knng_mt(x, w.K, rho, w.delta, w.max_iters, seed=0)
    r_orc = metrics.recall(x, oi, exact, rows)
    r_gpu, st = _gpu_recall(x, xd, w, rho, w.delta, w.max_iters, rows, exact)
    assert r_gpu >= 0.99 and abs(r_gpu - r_orc) <= PARITY, (r_gpu, r_orc)


def test_batched_recall_ceiling_is_the_methods():
    """The batched workload stays below recall 0.99 at every sample rate: on
    its hardest data set (47,530 x 128, 11 isotropic Gaussian clusters,
    K = 16) NN-Descent converges near 0.7 even at rho 1.0 with 30 iterations
    and no stopping threshold.  The oracle's build stops at the same recall,
    so the ceiling is the method's, not the kernels'."""
    specs = workloads.batched_specs(256, 0)
    s = next(v for v in specs if v["seed"] == 1058)
    x = workloads.gaussian_mixture(s["n"], s["d"], s["clusters"], seed=s["seed"])
    xd = torch.from_numpy(x).cuda()
    rows = np.sort(np.random.default_rng(3).choice(len(x), 1000, replace=False))
    exact = _ground_truth(x, xd, 16, rows)
    gi, _, _ = knng.knng_build(xd, 16, 1.0, 0.0, 30, seed=0)
    oi, _, _ = oracle.build_knng_mt(x, 16, 1.0, 0.0, 30, seed=0)
    r_gpu = metrics.recall(x, gi.cpu().numpy(), exact, rows)
    r_orc = metrics.recall(x, oi, exact, rows)
    assert r_gpu < 0.8 and r_orc < 0.8 and abs(r_gpu - r_orc) <= PARITY, (r_gpu, r_orc)


def test_audio_like_relabelled_build_keeps_recall():
    """Audio-shaped 54,387 x 192 with Algorithm 1 relabelling after iteration 1:
    the relabelling changes where rows live, not the method's graph quality,
    so recall stays within the parity tolerance of the oracle's plain build."""
    w, x = workloads.make("audio_like_n54k_d192")
    xd = torch.from_numpy(x).cuda()
    rows = recall_rows(w.n)
    exact = _ground_truth(x, xd, w.K, rows)
    oi, _, _ = oracle.build_knng_mt(x, w.K, w.rho, w.delta, w.max_iters, seed=0)
    r_orc = metrics.recall(x, oi, exact, rows)
    r_rel, st = _gpu_recall(x, xd, w, w.rho, w.delta, w.max_iters, rows, exact, knng.FLAG_REORDER)
    assert st["reordered"] == 1
    assert abs(r_rel - r_orc) <= PARITY, (r_rel, r_orc)
