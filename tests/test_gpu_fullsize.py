"""The high-dimensional workloads at full size, in the launch configuration
bench.py times (knng_build with each workload's parameters, seed 0).

The oracle's NN-Descent cannot run at these sizes in a test, so the checks
are the properties that hold at any size, on sampled rows:
- list invariants and every returned distance within 1e-4 of its float64
  recomputation (the accuracy audit);
- the GPU brute force equals the oracle's brute force on sampled rows (ids up
  to ties), so it can serve as ground truth for recall on more rows;
- recall at the level measured for the workload, and bf16 within 0.01 of
  float32.
The float32 builds are bit-exact against the oracle at smaller sizes through
the same kernels (test_gpu_parity: every join kernel forced on the same
inputs).
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


def _check_workload(name, min_recall, oracle_rows=12, recall_rows=2000):
    w, x = workloads.make(name)
    xd = torch.from_numpy(x).cuda()
    g = np.random.default_rng(7)
    rows = g.choice(w.n, recall_rows, replace=False)
    # ground truth: GPU brute force, itself checked against the oracle
    bi, bd = knng.knng_bruteforce(xd, w.K, rows=torch.from_numpy(rows).cuda())
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    sub = rows[:oracle_rows]
    oi, od = oracle.bruteforce(x, w.K, sub)
    np.testing.assert_allclose(bd[:oracle_rows], od, rtol=1e-5, atol=1e-7)
    mism = bi[:oracle_rows] != oi
    assert np.allclose(bd[:oracle_rows][mism], od[mism], rtol=1e-5, atol=1e-7)
    out = {}
    for flags in (0, knng.FLAG_BF16):
        gi, gd, st = knng.knng_build(xd, w.K, w.rho, w.delta, w.max_iters, seed=0, flags=flags)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        assert metrics.check_graph(x, gi, gd, rows=rows) == []
        assert st["lock_timeouts"] == 0 and st["set_overflow"] == 0
        out[flags] = metrics.recall(x, gi, bi, rows)
    assert out[0] >= min_recall, out
    assert out[knng.FLAG_BF16] >= out[0] - 0.01, out
    return out


def test_mixture_n1m_d128_full_size():
    """1,000,000 x 128, 1,000 clusters, K=32, rho=0.3, 12 iterations (ring
    join kernel, float32 and bf16)."""
    _check_workload("mixture_n1m_d128", min_recall=0.955)


def test_mnist_like_n70k_d784_full_size():
    """70,000 x 784 MNIST-shaped integers, K=20, rho=0.5 (tile kernel in
    float32, ring kernel in bf16)."""
    _check_workload("mnist_like_n70k_d784", min_recall=0.98)


def test_batched_workload_slice_equals_single_builds():
    """32 data sets of the batched workload (every row-width class of it):
    the batched build equals each data set's own build bit for bit."""
    specs = workloads.batched_specs(256, 0)[:32]
    sets = [workloads.gaussian_mixture(s["n"], s["d"], s["clusters"], seed=s["seed"]) for s in specs]
    xs = [torch.from_numpy(x).cuda() for x in sets]
    cfg = workloads.BATCHED
    outs, st = knng.knng_build_batched(xs, cfg["K"], cfg["rho"], cfg["delta"], cfg["max_iters"], seed=0)
    assert st["lock_timeouts"] == 0
    for x, (bi, bd) in zip(xs, outs):
        si, sd, _ = knng.knng_build(x, cfg["K"], cfg["rho"], cfg["delta"], cfg["max_iters"], seed=0)
        assert torch.equal(bi, si) and torch.equal(bd, sd)


def test_audio_like_n54k_d192_full_size_plain_and_relabelled():
    """Audio-shaped 54,387 x 192 (K=20, rho=0.5): plain and Algorithm-1
    relabelled builds both meet the invariants and the same recall level
    (the relabelling changes the visiting order of the nodes, not the
    method's graph quality)."""
    w, x = workloads.make("audio_like_n54k_d192")
    xd = torch.from_numpy(x).cuda()
    rows = np.random.default_rng(3).choice(w.n, 1000, replace=False)
    bi, _ = knng.knng_bruteforce(xd, w.K, rows=torch.from_numpy(rows).cuda())
    bi = bi.cpu().numpy()
    rec = {}
    for flags in (0, knng.FLAG_REORDER):
        gi, gd, st = knng.knng_build(xd, w.K, w.rho, w.delta, w.max_iters, seed=0, flags=flags)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        assert metrics.check_graph(x, gi, gd, rows=rows) == []
        rec[flags] = metrics.recall(x, gi, bi, rows)
    assert rec[0] >= 0.97 and abs(rec[0] - rec[knng.FLAG_REORDER]) <= 0.01, rec
