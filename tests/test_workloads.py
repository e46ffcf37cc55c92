"""The seeded synthetic inputs match their stated recipes (CPU only): shapes,
float32, determinism per seed, and the distribution facts the workloads are
chosen for."""
import numpy as np
import pytest

import workloads


def test_every_named_workload_has_its_stated_shape():
    small = {"uniform_n2k_d8", "gaussian_n16k_d8"}
    for name, w in workloads.WORKLOADS.items():
        if name not in small:
            continue
        x = w.data()
        assert x.shape == (w.n, w.d) and x.dtype == np.float32
        assert np.isfinite(x).all()
        assert 1 <= w.K <= w.n - 1 and 0 < w.rho <= 1


def test_generators_are_deterministic_per_seed():
    a = workloads.gaussian_mixture(3000, 16, 7, seed=5)
    b = workloads.gaussian_mixture(3000, 16, 7, seed=5)
    c = workloads.gaussian_mixture(3000, 16, 7, seed=6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(workloads.uniform(500, 3, 1), workloads.uniform(500, 3, 1))


def test_mixture_clusters_are_equal_and_centred_as_stated():
    x, lab = workloads.gaussian_mixture(10_000, 16, 50, seed=0, return_labels=True)
    counts = np.bincount(lab, minlength=50)
    assert counts.min() == counts.max() == 200
    # each point is its centre plus N(0, I): per-cluster spread ~1, centres in [-10, 10]
    for c in range(0, 50, 7):
        pts = x[lab == c]
        assert abs(pts.std(axis=0).mean() - 1.0) < 0.15
        assert np.all(np.abs(pts.mean(axis=0)) < 10.5)


def test_single_gaussian_covariance_is_2i():
    x = workloads.single_gaussian(20_000, 8, seed=3, var=2.0)
    cov = np.cov(x.astype(np.float64), rowvar=False)
    assert np.allclose(np.diag(cov), 2.0, atol=0.1)
    assert np.abs(cov - np.diag(np.diag(cov))).max() < 0.1


def test_mnist_like_values_and_sparsity():
    x = workloads.mnist_like(3000, 784, seed=0)
    assert x.shape == (3000, 784) and x.dtype == np.float32
    assert np.array_equal(x, np.round(x)) and x.min() >= 0 and x.max() <= 255
    zeros = (x == 0).mean()
    assert 0.72 <= zeros <= 0.88, zeros


def test_audio_like_shape():
    x = workloads.audio_like(5000, 192, seed=0)
    assert x.shape == (5000, 192) and x.dtype == np.float32 and np.isfinite(x).all()


def test_batched_specs_follow_the_recipe():
    specs = workloads.batched_specs(256, 0)
    assert len(specs) == 256
    assert all(500 <= s["n"] <= 50_000 for s in specs)
    assert {s["d"] for s in specs} <= {32, 96, 128}
    assert all(5 <= s["clusters"] <= 50 for s in specs)
    assert [s["seed"] for s in specs] == [1000 + i for i in range(256)]


def test_random_graph_is_a_valid_list_graph():
    ids, is_new = workloads.random_graph(500, 12, seed=4, p_new=0.3)
    assert ids.shape == (500, 12) and is_new.shape == (500, 12)
    for u in range(500):
        assert u not in ids[u] and len(set(ids[u].tolist())) == 12
    assert 0.2 < is_new.mean() < 0.4
