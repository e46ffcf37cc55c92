"""Seeded synthetic inputs for K-NNG construction.

This module is the one piece of code that both the CUDA path (tests, bench)
and the CPU oracle may use.  It draws input point sets and random graphs and
holds none of the method's arithmetic: no distances, no sampling decisions,
no neighbour selection.  All generators use numpy's PCG64 with an explicit
seed, so the same call gives the same array on every machine running the same
numpy.

The workloads mirror the paper's data sets (Section 4, "Experimental setup"):
the Synthetic Gaussian and Synthetic Clustered sets are drawn as described
there; MNIST (70,000 x 784 integer pixel intensities) is not available, so an
MNIST-shaped stand-in of the same size, value range and sparsity is drawn
instead (no MNIST record is reproduced).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "uniform", "gaussian_mixture", "single_gaussian",
    "mnist_like", "audio_like", "batched_specs", "random_graph", "make",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(n: int, d: int, seed: int = 0) -> np.ndarray:
    """n points uniform in [0, 1)^d, float32, row-major (n, d)."""
    return _rng(seed).random((n, d), dtype=np.float32)


def single_gaussian(n: int, d: int, seed: int = 0, var: float = 2.0) -> np.ndarray:
    """Section 4 'Single Gaussian' set: all points from N(0, var * I_d)."""
    x = _rng(seed).standard_normal((n, d), dtype=np.float32)
    return (x * np.float32(math.sqrt(var))).astype(np.float32)


def gaussian_mixture(n: int, d: int, clusters: int, seed: int = 0,
                     centre_low: float | None = -10.0, centre_high: float | None = 10.0,
                     centre_std: float | None = None, sigma: float = 1.0,
                     return_labels: bool = False):
    """Equal-weight isotropic Gaussian mixture ('Synthetic Clustered', Section 4).

    Centres are uniform in [centre_low, centre_high]^d, or N(0, centre_std^2 I)
    when centre_std is given.  Each cluster gets n // clusters points (the first
    n % clusters clusters one more), assigned in a random order, and every point
    is its centre plus N(0, sigma^2 I).
    """
    g = _rng(seed)
    if centre_std is not None:
        centres = g.standard_normal((clusters, d)) * centre_std
    else:
        centres = g.uniform(centre_low, centre_high, size=(clusters, d))
    labels = g.permutation(np.arange(n) % clusters)
    noise = g.standard_normal((n, d)) * sigma
    x = (centres[labels] + noise).astype(np.float32)
    if return_labels:
        return x, labels.astype(np.int32)
    return x


def mnist_like(n: int = 70_000, d: int = 784, seed: int = 0, prototypes: int = 10, latent: int = 6,
               proto_on: float = 0.20, flip: float = 0.01, return_labels: bool = False):
    """MNIST-shaped stand-in: integer intensities 0..255 stored as float32,
    about 80% zeros, points on low-dimensional manifolds around prototypes.

    Recipe: `prototypes` random binary masks (each pixel on with probability
    `proto_on`) with base intensities uniform in {100..200} and a
    `latent`-dimensional deformation basis with N(0, 25^2) entries.  A point
    takes a random prototype, a latent vector z ~ N(0, I), and sets every on
    pixel to base + basis . z + a uniform integer in [-3, 3], rounded and
    clamped to [1, 255]; then every pixel is flipped on/off independently with
    probability `flip` (switched-on pixels get a uniform intensity in
    {64..255}).  Handwritten digits vary along a few smooth directions around
    a class shape; so do these points, which keeps nearest neighbours
    meaningful (pure per-pixel noise would make all same-class points about
    equally far apart).
    """
    g = _rng(seed)
    masks = g.random((prototypes, d)) < proto_on
    base = g.integers(100, 201, size=(prototypes, d)).astype(np.float64)
    basis = g.standard_normal((prototypes, d, latent)) * 25.0
    labels = g.integers(0, prototypes, size=n)
    z = g.standard_normal((n, latent))
    jitter = g.integers(-3, 4, size=(n, d))
    x = np.empty((n, d), dtype=np.float64)
    for c in range(prototypes):
        idx = np.nonzero(labels == c)[0]
        x[idx] = base[c] + z[idx] @ basis[c].T
    x = np.clip(np.rint(x + jitter), 1, 255)
    on = masks[labels]
    x = np.where(on, x, 0.0)
    flips = g.random((n, d)) < flip
    fresh = g.integers(64, 256, size=(n, d))
    x = np.where(flips & on, 0.0, x)
    x = np.where(flips & ~on, fresh, x)
    x = x.astype(np.float32)
    if return_labels:
        return x, labels.astype(np.int32)
    return x


def audio_like(n: int = 54_387, d: int = 192, seed: int = 0, sentences: int = 500, latent: int = 12,
               corr: float = 0.9, noise: float = 0.1, return_labels: bool = False):
    """Audio-shaped stand-in (the Audio set: 54,387 frames of 192 features
    from spoken English sentences; not available): frames of `sentences`
    utterances of random lengths, each utterance a smooth trajectory in a
    `latent`-dimensional space (AR(1) with coefficient `corr`, unit
    stationary variance) mapped to d features by one fixed random linear map
    (N(0, 1/latent) entries), plus a per-utterance offset (N(0, 0.5^2)) and
    per-feature noise N(0, noise^2).  Consecutive frames are close, as
    spectral frames of speech are; float32."""
    g = _rng(seed)
    A = g.standard_normal((d, latent)) / math.sqrt(latent)
    cuts = np.sort(g.choice(np.arange(1, n), sentences - 1, replace=False))
    lengths = np.diff(np.concatenate([[0], cuts, [n]]))
    x = np.empty((n, d), dtype=np.float64)
    labels = np.empty(n, dtype=np.int32)
    pos = 0
    innov = math.sqrt(1.0 - corr * corr)
    for s_, L in enumerate(lengths):
        z = np.empty((L, latent))
        z[0] = g.standard_normal(latent)
        eps = g.standard_normal((L, latent)) * innov
        for t in range(1, L):
            z[t] = corr * z[t - 1] + eps[t]
        off = g.standard_normal(d) * 0.5
        x[pos:pos + L] = z @ A.T + off
        labels[pos:pos + L] = s_
        pos += L
    x += g.standard_normal((n, d)) * noise
    x = x.astype(np.float32)
    if return_labels:
        return x, labels
    return x


def batched_specs(count: int = 256, seed: int = 0):
    """Sizes for the batched workload: n ~ U{500..50000}, d ~ {32, 96, 128},
    clusters ~ U{5..50}; dataset i is drawn with generator seed 1000 + i."""
    g = _rng(seed)
    ns = g.integers(500, 50_001, size=count)
    ds = g.choice(np.array([32, 96, 128]), size=count)
    cs = g.integers(5, 51, size=count)
    return [dict(n=int(ns[i]), d=int(ds[i]), clusters=int(cs[i]), seed=1000 + i)
            for i in range(count)]


def random_graph(n: int, K: int, seed: int = 0, p_new: float = 0.5):
    """A random directed K-regular graph state for step-level parity tests.

    Returns ids (n, K) int32 with K distinct ids != u per row (uniform), and
    is_new (n, K) uint8 with each entry 1 with probability p_new.  Only random
    ids are drawn here; any distance, ordering or selection is left to the
    code under test.
    """
    if not (1 <= K <= n - 1):
        raise ValueError("need 1 <= K <= n-1")
    g = _rng(seed)
    ids = np.empty((n, K), dtype=np.int32)
    for u in range(n):
        # K distinct values from [0, n-1) shifted past u
        c = g.choice(n - 1, size=K, replace=False)
        c = c + (c >= u)
        ids[u] = c
    is_new = (g.random((n, K)) < p_new).astype(np.uint8)
    return ids, is_new


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named workload: data recipe plus NN-Descent parameters."""
    name: str
    n: int
    d: int
    K: int
    rho: float
    delta: float
    max_iters: int
    kind: str
    params: tuple = ()
    seed: int = 0

    def data(self) -> np.ndarray:
        p = dict(self.params)
        if self.kind == "uniform":
            return uniform(self.n, self.d, self.seed)
        if self.kind == "mixture":
            return gaussian_mixture(self.n, self.d, seed=self.seed, **p)
        if self.kind == "mnist_like":
            return mnist_like(self.n, self.d, seed=self.seed, **p)
        if self.kind == "single_gaussian":
            return single_gaussian(self.n, self.d, seed=self.seed, **p)
        if self.kind == "audio_like":
            return audio_like(self.n, self.d, seed=self.seed, **p)
        raise ValueError(self.kind)


WORKLOADS = {
    # plain FP32, small: the oracle finishes it in seconds
    "uniform_n2k_d8": Workload("uniform_n2k_d8", 2_000, 8, 10, 1.0, 0.001, 10, "uniform"),
    # low-dim clustered, 50 clusters, centres U[-10,10]^16, sigma 1
    "clustered_n100k_d16": Workload("clustered_n100k_d16", 100_000, 16, 20, 0.5, 0.001, 15,
                                    "mixture", (("clusters", 50),)),
    # MNIST-shaped integer data
    "mnist_like_n70k_d784": Workload("mnist_like_n70k_d784", 70_000, 784, 20, 0.5, 0.001, 15,
                                     "mnist_like"),
    # the selection-step comparison setting: Single Gaussian, covariance 2 I
    "gaussian_n16k_d8": Workload("gaussian_n16k_d8", 16_384, 8, 20, 0.5, 0.001, 15, "single_gaussian",
                                 (("var", 2.0),)),
    # Audio-shaped: 54,387 x 192 frames of 500 smooth utterances
    "audio_like_n54k_d192": Workload("audio_like_n54k_d192", 54_387, 192, 20, 0.5, 0.001, 15, "audio_like"),
    # large dense, 1000 clusters, centres N(0, 4I), sigma 0.5
    "mixture_n1m_d128": Workload("mixture_n1m_d128", 1_000_000, 128, 32, 0.3, 0.001, 12,
                                 "mixture", (("clusters", 1000), ("centre_std", 2.0),
                                             ("sigma", 0.5))),
}


BATCHED = dict(name="batched_256", count=256, K=16, rho=0.5, delta=0.001, max_iters=15, seed=0)


def batched_data(count: int = 256, seed: int = 0):
    """Data sets of the batched workload: equal-weight Gaussian mixtures with
    the sizes of batched_specs (centres U[-10, 10]^d, sigma 1)."""
    return [gaussian_mixture(s["n"], s["d"], s["clusters"], seed=s["seed"]) for s in batched_specs(count, seed)]


def make(name: str) -> tuple[Workload, np.ndarray]:
    w = WORKLOADS[name]
    return w, w.data()
