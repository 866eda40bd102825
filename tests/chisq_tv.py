"""Goodness of fit of sampled frequencies against an exact distribution p when
the sampler is only known to lie within total variation delta of p.

The composite null is "the sampler's distribution q satisfies TV(q, p) <=
delta".  For a fixed q the Pearson statistic X^2(q) of M samples merged into K
categories is asymptotically chi-square with K - 1 degrees of freedom; under
the null, min over the TV ball of X^2(q) is at most X^2(q_true), so rejecting
when that minimum exceeds the chi-square quantile has level <= alpha.

The minimum is bounded from below by Lagrangian duality (the problem is
convex): for multipliers lambda (sum q = 1) and mu >= 0 (sum |q - p| <=
2 delta) the separable inner minimisation has a closed form per category, and
any dual value is a lower bound of the minimum.  Rejecting when a dual value
exceeds the quantile is therefore still a level-alpha test; maximising the
dual over (lambda, mu) makes it as strong as the exact minimum.
"""
from __future__ import annotations

import numpy as np


def merge_categories(counts: np.ndarray, probs: np.ndarray, min_expected: float = 5.0):
    """Merges categories in order of increasing expected count until every
    merged category expects at least min_expected samples.  Returns
    (observed counts, probabilities) of the merged categories."""
    M = counts.sum()
    order = np.argsort(probs * M, kind="stable")
    oc, pc, ao, ap = [], [], 0.0, 0.0
    for t in order:
        ao += counts[t]
        ap += probs[t]
        if ap * M >= min_expected:
            oc.append(ao)
            pc.append(ap)
            ao = ap = 0.0
    if not oc:
        return np.array([ao]), np.array([ap])
    oc[-1] += ao
    pc[-1] += ap
    return np.array(oc, dtype=np.float64), np.array(pc, dtype=np.float64)


def _dual(o: np.ndarray, p: np.ndarray, M: float, delta: float, lam: float, mu: float) -> float:
    """Dual function D(lambda, mu) of  min sum (o - M q)^2 / (M q)
    s.t. sum q = 1, sum |q - p| <= 2 delta, q >= 0."""
    a_plus = M + lam + mu
    if a_plus <= 0.0:
        return -np.inf
    a_minus = M + lam - mu
    q_plus = o / np.sqrt(M * a_plus)
    with np.errstate(divide="ignore", invalid="ignore"):
        q_minus = np.where(a_minus > 0.0, o / np.sqrt(M * max(a_minus, 1e-300)), np.inf)
    q = np.where(q_plus > p, q_plus, np.where(q_minus < p, q_minus, p))
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(q > 0.0, (o - M * q) ** 2 / (M * np.maximum(q, 1e-300)), np.where(o > 0.0, np.inf, 0.0))
    g = f + lam * q + mu * np.abs(q - p)
    return float(g.sum() - lam - 2.0 * delta * mu)


def min_chi_square_lower_bound(o: np.ndarray, p: np.ndarray, delta: float) -> float:
    """A lower bound (the best dual value found) of the smallest Pearson
    statistic over all q with TV(q, p) <= delta."""
    from scipy.optimize import minimize
    M = float(o.sum())
    if delta <= 0.0:
        return float(((o - M * p) ** 2 / (M * p)).sum())

    def neg(z):
        v = _dual(o, p, M, delta, z[0] * M, M * np.exp(z[1]))
        return 1e300 if not np.isfinite(v) else -v

    best = -np.inf
    for z0 in ([0.0, 0.0], [0.0, -3.0], [0.5, 1.0], [-0.5, -1.0]):
        r = minimize(neg, np.array(z0), method="Nelder-Mead",
                     options={"xatol": 1e-10, "fatol": 1e-10, "maxiter": 4000})
        best = max(best, -float(r.fun))
    return best


def tv_chi_square_pvalue(counts: np.ndarray, probs: np.ndarray, delta: float, min_expected: float = 5.0) -> float:
    """p-value bound of the composite test: the chi-square survival function at
    the lower bound of the minimum statistic (a valid, conservative p-value)."""
    from scipy.stats import chi2
    o, pm = merge_categories(np.asarray(counts, np.float64), np.asarray(probs, np.float64), min_expected)
    if o.size < 2:
        return 1.0
    stat = max(0.0, min_chi_square_lower_bound(o, pm, delta))
    return float(chi2.sf(stat, o.size - 1))
