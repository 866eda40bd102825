"""Downstream consumer of the similarity graph: spectral clustering and the
Rand index, as the paper's experiments use the graph (Sec. 5: the clusters of
the graph's normalised Laplacian, scored by the Rand index against the ground
truth).  Host code on the edge list that fsg_build_graph returns (scipy's
sparse eigensolver, a plain k-means); it is not part of the GPU hot path and
runs the same on an edge list from any source.

    labels = spectral_clustering(n, src, dst, w, k)
    rand_index(labels, truth)
"""
from __future__ import annotations

import numpy as np


def normalised_adjacency(n: int, src, dst, w):
    """D^-1/2 W D^-1/2 of the symmetric graph with an edge {src[e], dst[e]} of
    weight w[e] for every e (repeated pairs add up), D the weighted degrees.
    Isolated vertices get a zero row."""
    import scipy.sparse as sp
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    w = np.asarray(w, np.float64)
    W = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([src, dst]), np.concatenate([dst, src]))),
                      shape=(n, n)).tocsr()
    deg = np.asarray(W.sum(axis=1)).ravel()
    inv = np.zeros(n)
    inv[deg > 0] = 1.0 / np.sqrt(deg[deg > 0])
    Dm = sp.diags(inv)
    return Dm @ W @ Dm


def spectral_embedding(n: int, src, dst, w, k: int) -> np.ndarray:
    """The k leading eigenvectors of D^-1/2 W D^-1/2 (those of the k smallest
    eigenvalues of the normalised Laplacian I - D^-1/2 W D^-1/2), rows scaled
    to unit length.  float64 [n][k]."""
    from scipy.sparse.linalg import eigsh
    M = normalised_adjacency(n, src, dst, w)
    # A graph of c components has eigenvalue 1 c times.  Asking for more
    # eigenpairs than needed lets the solver's deflation find repeated ones
    # (asked for exactly k, it can return one copy and miss the other); the
    # seeded random start vector keeps the result deterministic.
    kk = min(n - 1, max(2 * k, k + 4))
    v0 = np.random.Generator(np.random.PCG64(12345)).standard_normal(n)
    vals, vecs = eigsh(M, k=kk, which="LA", v0=v0, tol=1e-10, maxiter=20 * n)
    vecs = vecs[:, np.argsort(vals)[::-1][:k]]
    norms = np.linalg.norm(vecs, axis=1, keepdims=True)
    return vecs / np.where(norms > 0, norms, 1.0)


def kmeans(Y: np.ndarray, k: int, seed: int = 0, iters: int = 200, restarts: int = 8) -> np.ndarray:
    """Lloyd's k-means with k-means++ seeding, the best of `restarts` runs by
    within-cluster sum of squares.  Returns int64 labels [n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = Y.shape[0]
    best, best_cost = None, np.inf
    for _ in range(restarts):
        C = np.empty((k, Y.shape[1]))
        C[0] = Y[rng.integers(n)]
        d2 = ((Y - C[0]) ** 2).sum(1)
        for j in range(1, k):
            p = d2 / d2.sum() if d2.sum() > 0 else np.full(n, 1.0 / n)
            C[j] = Y[rng.choice(n, p=p)]
            d2 = np.minimum(d2, ((Y - C[j]) ** 2).sum(1))
        lab = np.zeros(n, np.int64)
        for it in range(iters):
            D = ((Y[:, None, :] - C[None, :, :]) ** 2).sum(-1)
            new = D.argmin(1)
            if it > 0 and np.array_equal(new, lab):
                break
            lab = new
            for j in range(k):
                if (lab == j).any():
                    C[j] = Y[lab == j].mean(0)
        cost = ((Y - C[lab]) ** 2).sum()
        if cost < best_cost:
            best, best_cost = lab, cost
    return best


def spectral_clustering(n: int, src, dst, w, k: int, seed: int = 0) -> np.ndarray:
    """k clusters of the graph: k-means on the normalised spectral embedding."""
    return kmeans(spectral_embedding(n, src, dst, w, k), k, seed=seed)


def rand_index(a, b) -> float:
    """Fraction of the n(n-1)/2 point pairs on which two labelings agree
    (both together or both apart), from their contingency table."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    n = a.size
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    table = np.zeros((ai.max() + 1, bi.max() + 1), np.int64)
    np.add.at(table, (ai, bi), 1)
    pairs = lambda x: (x * (x - 1) // 2).sum()  # noqa: E731
    same_both = pairs(table)
    same_a = pairs(table.sum(1))
    same_b = pairs(table.sum(0))
    total = n * (n - 1) // 2
    return float((total + 2 * same_both - same_a - same_b) / total)
