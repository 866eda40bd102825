"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws input point sets; it holds none of the method's
arithmetic, and both the CUDA path's tests/bench and the CPU oracle consume
its output.  Every generator is deterministic in its seed (numpy PCG64).

Workloads (sizes as used by the bench and the parity tests):

* ``two_moons``      -- two interleaved half circles in R^2 with Gaussian noise,
                        the shape of the paper's synthetic data (Sec. 5.1);
* ``gaussian_mixture`` -- equal-weight isotropic blobs, the "blobs" shape of
                        Sec. 5.1 scaled up (centres uniform in a box);
* ``digit_like``     -- 784-dim 8-bit images around 10 sparse prototypes, a
                        stand-in for digit-image data (no such dataset ships);
* ``segmentation_image`` -- (r,g,b,x,y) pixel features of a piecewise-constant
                        Voronoi image, a stand-in for the BSDS images of
                        Sec. 5.2 (the dataset is not available here);
* ``serving_requests`` -- a Poisson arrival trace of graph-build requests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def two_moons(n: int = 2000, noise: float = 0.05, seed: int = 0) -> np.ndarray:
    """n points (n//2 per moon), moon A (cos t, sin t), moon B (1-cos t, 0.5-sin t),
    t evenly spaced on [0, pi], plus N(0, noise^2) per coordinate.  float32 [n][2]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    na = n // 2
    nb = n - na
    ta = np.linspace(0.0, math.pi, na)
    tb = np.linspace(0.0, math.pi, nb)
    a = np.stack([np.cos(ta), np.sin(ta)], axis=1)
    b = np.stack([1.0 - np.cos(tb), 0.5 - np.sin(tb)], axis=1)
    X = np.concatenate([a, b], axis=0)
    X = X + rng.normal(0.0, noise, size=X.shape)
    return X.astype(np.float32)


def two_moons_labels(n: int = 2000) -> np.ndarray:
    """The moon of each point of two_moons(n): 0 for the first n//2, else 1."""
    return (np.arange(n) >= n // 2).astype(np.int64)


def gaussian_mixture(n: int = 100_000, d: int = 10, k: int = 10, box: float = 10.0,
                     seed: int = 0, shuffle: bool = True, return_labels: bool = False):
    """k equal-weight N(c, I) blobs with centres uniform in [-box, box]^d.
    Points are shuffled (as generators of blob data usually do), so tree order
    carries no cluster structure.  float32 [n][d]; with return_labels also the
    blob of each point (the same points either way)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(-box, box, size=(k, d))
    counts = np.full(k, n // k)
    counts[: n - counts.sum()] += 1
    labels = np.repeat(np.arange(k), counts)
    X = centres[labels] + rng.normal(0.0, 1.0, size=(n, d))
    if shuffle:
        order = rng.permutation(n)
        X, labels = X[order], labels[order]
    if return_labels:
        return X.astype(np.float32), labels
    return X.astype(np.float32)


def digit_like(n: int = 70_000, d: int = 784, classes: int = 10, zero_frac: float = 0.8,
               noise: float = 0.1, seed: int = 0) -> np.ndarray:
    """classes prototypes with pixels 0 w.p. zero_frac else U{1..255}/255;
    each sample clip(prototype + N(0, noise^2), 0, 1) quantised to k/255.
    Shuffled.  float32 [n][d]; every value is an exact multiple of 1/255."""
    rng = np.random.Generator(np.random.PCG64(seed))
    proto = rng.integers(1, 256, size=(classes, d)).astype(np.float64) / 255.0
    proto[rng.random((classes, d)) < zero_frac] = 0.0
    counts = np.full(classes, n // classes)
    counts[: n - counts.sum()] += 1
    labels = np.repeat(np.arange(classes), counts)
    labels = labels[rng.permutation(n)]
    X = np.empty((n, d), dtype=np.float32)
    chunk = 8192
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        v = proto[labels[s:e]] + rng.normal(0.0, noise, size=(e - s, d))
        v = np.clip(v, 0.0, 1.0)
        X[s:e] = (np.rint(v * 255.0) / 255.0).astype(np.float32)
    return X


def median_pair_distance(X: np.ndarray, m: int = 4096, seed: int = 0) -> float:
    """Lower median of the pairwise Euclidean distances among a fixed seeded
    subset of m points (FP64).  Used to set the digit workload's bandwidth
    (sigma = median / 2); it is a property of the input, not of the method."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = X.shape[0]
    idx = np.sort(rng.choice(n, size=min(m, n), replace=False))
    Y = X[idx].astype(np.float64)
    sq = (Y * Y).sum(1)
    D2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * (Y @ Y.T), 0.0)
    iu = np.triu_indices(Y.shape[0], k=1)
    dist = np.sqrt(D2[iu])
    dist.sort()
    return float(dist[(dist.shape[0] - 1) // 2])


def segmentation_image(h: int, w: int, seed: int = 0, noise: float = 0.03, return_labels: bool = False):
    """(r,g,b,x,y) features of an h x w image made of 6-12 Voronoi regions of
    uniform random colour plus N(0, noise^2) per channel; x, y scaled to
    [0,1].  float32 [h*w][5], row-major pixel order; with return_labels also
    the region of each pixel (the same features either way)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = int(rng.integers(6, 13))
    sites = rng.uniform(0.0, 1.0, size=(k, 2))
    colours = rng.uniform(0.0, 1.0, size=(k, 3))
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    xs = (xx / max(w - 1, 1)).reshape(-1)
    ys = (yy / max(h - 1, 1)).reshape(-1)
    pts = np.stack([xs, ys], axis=1)
    d2 = ((pts[:, None, :] - sites[None, :, :]) ** 2).sum(-1)
    region = d2.argmin(1)
    rgb = colours[region] + rng.normal(0.0, noise, size=(h * w, 3))
    X = np.concatenate([rgb, pts], axis=1).astype(np.float32)
    return (X, region.astype(np.int64)) if return_labels else X


def segmentation_batch(count: int = 64, h_min: int = 160, h_max: int = 321, w_max: int = 481,
                       seed0: int = 0):
    """count images with heights evenly spaced in [h_min, h_max] and
    w = min(w_max, round(1.5 h)); image t uses seed seed0 + t."""
    hs = np.rint(np.linspace(h_min, h_max, count)).astype(int)
    out = []
    for t, h in enumerate(hs):
        w = min(w_max, int(round(1.5 * h)))
        out.append(segmentation_image(int(h), w, seed=seed0 + t))
    return out


@dataclass
class Request:
    arrival_s: float
    n: int
    d: int
    seed: int


def serving_requests(count: int = 10_000, rate_hz: float = 200.0, n_lo: int = 1_000,
                     n_hi: int = 200_000, dims=(2, 10, 64), seed: int = 0):
    """Poisson arrivals (exponential gaps of mean 1/rate), n log-uniform in
    [n_lo, n_hi], d uniform over dims; each request's data is a Gaussian
    mixture drawn with its own seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps)
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(int)
    ds = rng.choice(np.asarray(dims), size=count)
    return [Request(float(t[r]), int(ns[r]), int(ds[r]), int(seed * 1_000_003 + r + 1)) for r in range(count)]
