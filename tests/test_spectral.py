"""The downstream consumer (spectral clustering of the graph, Rand index;
Sec. 5) on the oracle's graphs, no GPU: the Rand index against a direct
count over pairs, the normalised adjacency against its dense formula, and
cluster recovery on two moons and a segmentation image, where the sampled
graph must cluster about as well as the complete kernel graph (Thm. 2's
cluster preservation, qualitatively)."""
import itertools

import numpy as np
import pytest

import oracle as ora
from paper_2310_13870_gb300 import inputs, spectral

pytest.importorskip("scipy")


def test_rand_index_by_pairs():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.integers(0, 4, 30)
        b = rng.integers(0, 3, 30)
        agree = sum((a[i] == a[j]) == (b[i] == b[j]) for i, j in itertools.combinations(range(30), 2))
        assert spectral.rand_index(a, b) == pytest.approx(agree / (30 * 29 / 2), abs=1e-15)
    a = rng.integers(0, 5, 100)
    assert spectral.rand_index(a, a) == 1.0
    assert spectral.rand_index(a, (a + 3) % 5) == 1.0  # renamed clusters


def test_normalised_adjacency_dense_formula():
    rng = np.random.default_rng(1)
    n = 12
    src = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 0, 0])
    dst = np.array([1, 2, 3, 4, 5, 6, 7, 8, 9, 0, 5, 5])  # a repeated pair adds up; 10 and 11 isolated
    w = rng.uniform(0.5, 2.0, src.size)
    W = np.zeros((n, n))
    for s, t, x in zip(src, dst, w):
        W[s, t] += x
        W[t, s] += x
    deg = W.sum(1)
    inv = np.where(deg > 0, 1.0 / np.sqrt(np.where(deg > 0, deg, 1.0)), 0.0)
    np.testing.assert_allclose(spectral.normalised_adjacency(n, src, dst, w).toarray(), inv[:, None] * W * inv[None, :],
                               rtol=1e-13, atol=0)


def _dense_labels(X, gam, k):
    K = np.exp(-gam * ((X[:, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(K, 0.0)
    i, j = np.nonzero(np.triu(K, 1))
    return spectral.spectral_clustering(len(X), i, j, K[i, j], k)


def test_two_moons_recovered():
    n = 400
    X = inputs.two_moons(n=n, seed=1)
    o = ora.build_graph(X, ora.gamma(0.1), 16, 3)
    lab = spectral.spectral_clustering(n, o["src"], o["dst"], o["w"], 2)
    assert spectral.rand_index(lab, inputs.two_moons_labels(n)) >= 0.99


def test_segmentation_graph_clusters_like_the_complete_graph():
    X, reg = inputs.segmentation_image(24, 36, seed=3, return_labels=True)
    k = len(np.unique(reg))
    gam = ora.gamma(0.05)
    o = ora.build_graph(X, gam, 16, 2)
    ri_sparse = spectral.rand_index(spectral.spectral_clustering(len(X), o["src"], o["dst"], o["w"], k), reg)
    ri_dense = spectral.rand_index(_dense_labels(X, gam, k), reg)
    assert ri_sparse >= 0.85 and ri_sparse >= ri_dense - 0.05, (ri_sparse, ri_dense)
