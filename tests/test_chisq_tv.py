"""The composite goodness-of-fit test of tests/chisq_tv.py (used for the
approximate KDE's samples) on multinomial draws with a known sampler: it must
accept a sampler within the stated total variation of p, reject one five times
further away, and agree with the plain chi-square test when delta = 0."""
import numpy as np
from scipy.stats import chi2

from chisq_tv import merge_categories, min_chi_square_lower_bound, tv_chi_square_pvalue


def _shift(p, tv):
    # moves mass tv from the larger half of the categories to the smaller half
    idx = np.argsort(p)
    lo, hi = idx[: p.size // 2], idx[p.size // 2:]
    q = p.copy()
    q[hi] *= 1.0 - tv / p[hi].sum()
    q[lo] *= 1.0 + tv / p[lo].sum()
    return q


def test_accepts_within_and_rejects_beyond_the_ball():
    rng = np.random.Generator(np.random.PCG64(3))
    p = rng.exponential(size=800)
    p /= p.sum()
    delta, M = 0.02, 40_000
    q_in, q_out = _shift(p, delta), _shift(p, 5 * delta)
    assert abs(0.5 * np.abs(q_in - p).sum() - delta) < 1e-12
    for _ in range(5):
        assert tv_chi_square_pvalue(rng.multinomial(M, q_in), p, delta) > 0.01
        assert tv_chi_square_pvalue(rng.multinomial(M, q_out), p, delta) < 1e-6


def test_delta_zero_is_the_pearson_test():
    rng = np.random.Generator(np.random.PCG64(4))
    p = rng.exponential(size=200)
    p /= p.sum()
    c = rng.multinomial(20_000, p)
    o, pm = merge_categories(c.astype(np.float64), p)
    stat = ((o - o.sum() * pm) ** 2 / (o.sum() * pm)).sum()
    assert np.isclose(tv_chi_square_pvalue(c, p, 0.0), chi2.sf(stat, o.size - 1))


def test_dual_bound_below_the_statistic_of_any_point_in_the_ball():
    # weak duality: the bound never exceeds X^2(q) for a q inside the ball
    rng = np.random.Generator(np.random.PCG64(5))
    p = rng.exponential(size=60)
    p /= p.sum()
    delta = 0.05
    c = rng.multinomial(5_000, _shift(p, 0.5 * delta)).astype(np.float64)
    lb = min_chi_square_lower_bound(c, p, delta)
    M = c.sum()
    for t in np.linspace(0.0, 1.0, 11):
        q = (1 - t) * p + t * _shift(p, delta)
        assert lb <= ((c - M * q) ** 2 / (M * q)).sum() + 1e-9
