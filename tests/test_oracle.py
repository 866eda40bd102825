"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
brute force with an independent library routine (scipy's cdist), the
telescoping of the descent's branch probabilities (Lemma 1's proof, App. A),
per-level conservation (Sec. 4.2), and chi-square tests of the sampler's
output frequencies against the exact target distribution k(x_i,x_j)/deg(v_i)
(Sec. 4.1).  A plausible slip in the oracle (dropped self mask, wrong split,
reversed comparison, wrong degree in the weight) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.spatial.distance import cdist
from scipy.stats import chi2

import oracle as ora
from paper_2310_13870_gb300 import inputs


def _exact_probs(X, gam, i, include_self=False):
    """Target distribution of one sample, from scipy's pairwise distances."""
    X = np.asarray(X, dtype=np.float64)
    k = np.exp(-gam * cdist(X[i:i + 1], X, "sqeuclidean")[0])
    if not include_self:
        k[i] = 0.0
    return k / k.sum()


def _chi2_pvalue(counts, probs, min_expected=5.0):
    """Pearson chi-square with bins of small expectation merged."""
    total = counts.sum()
    exp = probs * total
    order = np.argsort(exp)
    oc, ec = [], []
    acc_o = acc_e = 0.0
    for t in order:
        acc_o += counts[t]
        acc_e += exp[t]
        if acc_e >= min_expected:
            oc.append(acc_o)
            ec.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0 and ec:
        oc[-1] += acc_o
        ec[-1] += acc_e
    oc, ec = np.array(oc), np.array(ec)
    stat = ((oc - ec) ** 2 / ec).sum()
    dof = max(len(ec) - 1, 1)
    return chi2.sf(stat, dof)


def _tree_nodes(n):
    """Node ranges per level of the halving tree: left half = floor(size/2)."""
    levels = [[(0, n)]]
    while any(hi - lo > 1 for lo, hi in levels[-1]):
        nxt = []
        for lo, hi in levels[-1]:
            if hi - lo > 1:
                m = lo + (hi - lo) // 2
                nxt += [(lo, m), (m, hi)]
            else:
                nxt.append((lo, hi))
        levels.append(nxt)
    return levels


def test_split_left_half_is_floor():
    # Sec. 4.1: |X1| = floor(|X|/2), |X2| = ceil(|X|/2).
    for lo in (0, 7, 1000):
        for s in range(2, 41):
            m = ora.split(lo, lo + s)
            assert m - lo == s // 2
            assert lo + s - m == (s + 1) // 2


def test_kernel_bandwidth_conventions():
    # Sec. 2.1 prints exp(-r^2/sigma^2); the default reading is exp(-r^2/(2 sigma^2)).
    sigma = 0.7
    a = np.zeros(3, np.float32)
    b = np.array([sigma, 0.0, 0.0], np.float32)
    b64 = float(np.float32(sigma))
    g2 = ora.gamma(sigma, ora.TWO_SIGMA_SQ)
    g1 = ora.gamma(sigma, ora.SIGMA_SQ)
    assert math.isclose(ora.kernel(a, b, g2), math.exp(-b64 * b64 / (2 * sigma * sigma)), rel_tol=1e-15)
    assert math.isclose(ora.kernel(a, b, g1), math.exp(-b64 * b64 / (sigma * sigma)), rel_tol=1e-15)
    assert ora.kernel(a, a, g2) == 1.0


@pytest.mark.parametrize("self_mode", [ora.SELF_EXCLUDE, ora.SELF_INCLUDE])
def test_kde_and_degrees_match_bruteforce(self_mode):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(57, 3)).astype(np.float32)
    gam = 0.8
    K = np.exp(-gam * cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean"))
    if self_mode == ora.SELF_EXCLUDE:
        np.fill_diagonal(K, 0.0)
    deg = ora.degrees(X, gam, self_mode=self_mode)
    np.testing.assert_allclose(deg, K.sum(1), rtol=1e-13)
    perm = rng.permutation(57)
    for i in (0, 13, 56):
        for lo, hi in ((0, 57), (5, 30), (20, 21), (40, 57)):
            want = K[i, perm[lo:hi]].sum()
            got = ora.kde(X, gam, i, lo, hi, perm=perm, self_mode=self_mode)
            assert math.isclose(got, want, rel_tol=1e-13, abs_tol=1e-300)


def test_level_conservation():
    # Sec. 4.2: the nodes of any level partition the points, so their KDEs sum to the degree.
    X = inputs.two_moons(n=37, seed=5)
    gam = ora.gamma(0.3)
    perm = np.random.default_rng(1).permutation(37)
    deg = ora.degrees(X, gam)
    for i in (0, 18, 36):
        for nodes in _tree_nodes(37):
            tot = sum(ora.kde(X, gam, i, lo, hi, perm=perm) for lo, hi in nodes)
            assert math.isclose(tot, deg[i], rel_tol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13, 16])
@pytest.mark.parametrize("self_mode", [ora.SELF_EXCLUDE, ora.SELF_INCLUDE])
def test_path_probability_telescopes_to_target(n, self_mode):
    # Lemma 1 (App. A) with exact KDE: the product of branch probabilities on the
    # path to j equals k(x_i,x_j)/g_[1,n](x_i); brute force over every (i, j).
    rng = np.random.default_rng(n)
    X = (rng.normal(size=(n, 2)) * 0.6).astype(np.float32)
    gam = 1.3
    perm = rng.permutation(n)
    pos = np.empty(n, dtype=np.int64)
    pos[perm] = np.arange(n)
    for i in range(n):
        want = _exact_probs(X, gam, i, include_self=(self_mode == ora.SELF_INCLUDE))
        got = np.array([ora.path_prob(X, gam, i, pos[j], perm=perm, self_mode=self_mode) for j in range(n)])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)
        assert math.isclose(got.sum(), 1.0, rel_tol=1e-12)


def test_sampler_frequencies_chi_square():
    # Sec. 4.1: a sample of x_i is x_j with probability k(x_i,x_j)/deg(v_i).
    rng = np.random.default_rng(11)
    n = 23
    X = np.concatenate([rng.normal(0, 0.4, size=(15, 2)), rng.normal(2.0, 0.9, size=(8, 2))]).astype(np.float32)
    perm = rng.permutation(n)
    gam = 0.9
    queries = np.array([0, 7, 16, 22])
    L = 64
    counts = np.zeros((len(queries), n))
    for seed in range(500):
        smp, _, _ = ora.sample(X, gam, L, seed, queries=queries, perm=perm)
        for q in range(len(queries)):
            counts[q] += np.bincount(smp[q], minlength=n)
    for q, i in enumerate(queries):
        assert counts[q, i] == 0  # EXCLUDE never returns the query itself
        p = _chi2_pvalue(counts[q], _exact_probs(X, gam, i))
        assert p > 0.01 / len(queries), (i, p)


def test_sampler_include_self_two_points():
    # n = 2 with the self term kept: P(self) = 1 / (1 + exp(-gamma r^2)).
    X = np.array([[0.0, 0.0], [0.5, 0.0]], np.float32)
    gam = 4.0
    k = math.exp(-gam * 0.25)
    hits = trials = 0
    for seed in range(200):
        smp, _, _ = ora.sample(X, gam, 64, seed, self_mode=ora.SELF_INCLUDE)
        hits += int((smp[0] == 0).sum())
        trials += smp.shape[1]
    p_self = 1.0 / (1.0 + k)
    z = (hits - trials * p_self) / math.sqrt(trials * p_self * (1 - p_self))
    assert abs(z) < 4.0


def test_two_point_closed_form():
    # n = 2, EXCLUDE: deg = exp(-gamma r^2), each point samples the other, and
    # p_hat = 1 (L k / deg = L >= 1) so w = k.
    X = np.array([[0.0], [0.8]], np.float32)
    gam = ora.gamma(0.5)
    r2 = float(np.float32(0.8)) ** 2
    k = math.exp(-gam * r2)
    g = ora.build_graph(X, gam, L=4, seed=9)
    np.testing.assert_allclose(g["deg"], [k, k], rtol=1e-15)
    assert (g["samples"][0] == 1).all() and (g["samples"][1] == 0).all()
    assert list(g["src"]) == [0] and list(g["dst"]) == [1]
    assert math.isclose(g["w"][0], k, rel_tol=1e-15)


def test_identical_points_uniform_and_weights():
    # All points equal: k == 1, samples uniform over j != i, and
    # w = 1/p_hat with p_i = p_j = min(L/(n-1), 1).
    n, L = 9, 2
    X = np.ones((n, 3), np.float32)
    counts = np.zeros(n)
    for seed in range(300):
        smp, _, _ = ora.sample(X, 1.0, L, seed, queries=[4])
        counts += np.bincount(smp[0], minlength=n)
    probs = np.full(n, 1.0 / (n - 1))
    probs[4] = 0.0
    assert counts[4] == 0
    assert _chi2_pvalue(counts, probs) > 0.01
    g = ora.build_graph(X, 1.0, L, seed=0)
    p = L / (n - 1)
    np.testing.assert_allclose(g["w"], 1.0 / (2 * p - p * p), rtol=1e-14)


def test_weights_worked_example():
    # Three points on a line at 0, 1, 3 with gamma = 1 (sigma^2 = 1/2) and L = 1.
    # k01 = e^-1, k02 = e^-9, k12 = e^-4; deg0 = e^-1+e^-9, deg1 = e^-1+e^-4,
    # deg2 = e^-9+e^-4.  Edge {0,2}: p_0 = e^-9/deg0 = 1/(1+e^8),
    # p_2 = e^-9/deg2 = 1/(1+e^5), p_hat = p_0 + p_2 - p_0 p_2, w = e^-9/p_hat.
    # Edge {0,1}: p_0 = 1/(1+e^-8), p_1 = 1/(1+e^-3).
    X = np.array([[0.0], [1.0], [3.0]], np.float32)
    gam = ora.gamma(math.sqrt(0.5))
    assert math.isclose(gam, 1.0, rel_tol=1e-15)
    deg = ora.degrees(X, gam)
    k, w = ora.weights(X, gam, 1, deg, [0, 0, 2], [2, 1, 0])
    e = math.exp
    p0, p2 = 1 / (1 + e(8)), 1 / (1 + e(5))
    want02 = e(-9) / (p0 + p2 - p0 * p2)
    q0, q1 = 1 / (1 + e(-8)), 1 / (1 + e(-3))
    want01 = e(-1) / (q0 + q1 - q0 * q1)
    assert math.isclose(k[0], e(-9), rel_tol=1e-14)
    assert math.isclose(w[0], want02, rel_tol=1e-12)
    assert math.isclose(w[1], want01, rel_tol=1e-12)
    assert w[2] == w[0]  # symmetric in (i, j)


def test_weight_properties_random():
    X = inputs.two_moons(n=120, seed=2)
    gam = ora.gamma(0.1)
    L = 8
    g = ora.build_graph(X, gam, L, seed=3)
    k, w = ora.weights(X, gam, L, g["deg"], g["src"], g["dst"])
    np.testing.assert_allclose(w, g["w"], rtol=0, atol=0)
    assert (w >= k * (1 - 1e-15)).all()
    _, wr = ora.weights(X, gam, L, g["deg"], g["dst"], g["src"])
    np.testing.assert_array_equal(wr, w)


def test_build_graph_edge_semantics():
    X = inputs.two_moons(n=80, seed=4)
    gam = ora.gamma(0.1)
    L = 6
    gs = ora.build_graph(X, gam, L, seed=1, edge_mode=ora.EDGES_SET)
    gm = ora.build_graph(X, gam, L, seed=1, edge_mode=ora.EDGES_MULTI)
    smp = gs["samples"]
    pairs = {(min(i, j), max(i, j)) for i in range(80) for j in smp[i] if j >= 0 and j != i}
    got = list(zip(gs["src"].tolist(), gs["dst"].tolist()))
    assert got == sorted(pairs)
    assert len(got) <= 80 * L
    assert (gs["src"] < gs["dst"]).all()
    assert len(gm["src"]) == 80 * L - gm["n_self"]
    assert gm["n_self"] == 0
    gi = ora.build_graph(X, gam, L, seed=1, self_mode=ora.SELF_INCLUDE, edge_mode=ora.EDGES_MULTI)
    assert len(gi["src"]) == 80 * L - gi["n_self"]


def test_descent_depth():
    # The floor split gives leaves at depth floor(log2 n) or ceil(log2 n).
    X = inputs.two_moons(n=300, seed=6)
    smp, mrg, lev = ora.sample(X, ora.gamma(0.1), 16, 2, queries=np.arange(0, 300, 17))
    assert set(np.unique(lev)) <= {8, 9}
    assert (mrg >= 0).all() and (mrg <= 1).all()


def test_zero_degree_has_no_samples():
    X = np.array([[0.0], [1.0e6]], np.float32)
    smp, _, _ = ora.sample(X, 1.0, 4, 0)
    assert (smp == -1).all()
    X1 = np.zeros((1, 2), np.float32)
    smp1, _, _ = ora.sample(X1, 1.0, 3, 0)
    assert (smp1 == -1).all()


def test_philox_uniform_and_bijective():
    # Statistical pins of the generator (the bit-exact pin against an
    # independent implementation, cuRAND, runs on the GPU).
    u = np.array([ora.uniform(7, i, l, lev) for i in range(64) for l in range(16) for lev in range(16)])
    counts = np.histogram(u, bins=64, range=(0, 1))[0]
    assert chi2.sf(((counts - u.size / 64) ** 2 / (u.size / 64)).sum(), 63) > 1e-3
    a = u.reshape(64, 16, 16)
    for ax in range(3):
        x = np.moveaxis(a, ax, -1)
        c = np.corrcoef(x[..., :-1].ravel(), x[..., 1:].ravel())[0, 1]
        assert abs(c) < 0.03
    outs = {tuple(ora.philox4x32_10([c, 0, 0, 0], [1, 2])) for c in range(4096)}
    assert len(outs) == 4096
    # draws for levels 4m..4m+3 are the four words of one block
    blk = ora.philox4x32_10([5, 3, 2, 0], [0xDEADBEEF, 0x1])
    seed = (0x1 << 32) | 0xDEADBEEF
    assert [ora.draw_u32(seed, 5, 3, lev) for lev in range(8, 12)] == list(blk)


def test_golden_two_moons_regression():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "two_moons_64.json")
    with open(path) as f:
        gold = json.load(f)
    X = np.asarray(gold["points"], np.float32)
    np.testing.assert_array_equal(X, inputs.two_moons(n=64, seed=0))
    g = ora.build_graph(X, ora.gamma(0.1), L=8, seed=0)
    np.testing.assert_allclose(g["deg"], gold["deg"], rtol=1e-14)
    np.testing.assert_array_equal(g["samples"], np.asarray(gold["samples"]))
    np.testing.assert_array_equal(g["src"], gold["src"])
    np.testing.assert_array_equal(g["dst"], gold["dst"])
    np.testing.assert_allclose(g["w"], gold["w"], rtol=1e-14)


# ---- the other kernels of Sec. 2.1: Laplacian (l1 norm in the exponent) and
# exponential (l2 norm), k = exp(-c ||x - y||), c = 1/sigma

def _family_matrix(X, c, family):
    X = np.asarray(X, dtype=np.float64)
    metric = {ora.GAUSSIAN: "sqeuclidean", ora.LAPLACIAN: "cityblock", ora.EXPONENTIAL: "euclidean"}[family]
    return np.exp(-c * cdist(X, X, metric))


def test_kernel_families_closed_form():
    # a 3-4-5 triangle: squared l2 25, l1 7, l2 5 give three different values
    a = np.zeros(4, np.float32)
    b = np.array([3.0, 0.0, -4.0, 0.0], np.float32)
    sigma = 2.5
    assert math.isclose(ora.scale(sigma, ora.LAPLACIAN), 0.4, rel_tol=1e-15)
    assert math.isclose(ora.scale(sigma, ora.EXPONENTIAL), 0.4, rel_tol=1e-15)
    assert math.isclose(ora.scale(sigma, ora.GAUSSIAN), 1.0 / (2 * 2.5 * 2.5), rel_tol=1e-15)
    assert math.isclose(ora.kernel(a, b, 0.4, ora.LAPLACIAN), math.exp(-0.4 * 7.0), rel_tol=1e-15)
    assert math.isclose(ora.kernel(a, b, 0.4, ora.EXPONENTIAL), math.exp(-0.4 * 5.0), rel_tol=1e-15)
    assert math.isclose(ora.kernel(a, b, 0.4, ora.GAUSSIAN), math.exp(-0.4 * 25.0), rel_tol=1e-15)
    for f in (ora.LAPLACIAN, ora.EXPONENTIAL):
        assert ora.kernel(a, a, 0.4, f) == 1.0


@pytest.mark.parametrize("family", [ora.LAPLACIAN, ora.EXPONENTIAL])
def test_family_degrees_match_bruteforce(family):
    rng = np.random.default_rng(11)
    X = rng.normal(size=(61, 5)).astype(np.float32)
    c = 0.9
    K = _family_matrix(X, c, family)
    np.fill_diagonal(K, 0.0)
    np.testing.assert_allclose(ora.degrees(X, c, kernel=family), K.sum(1), rtol=1e-13)


@pytest.mark.parametrize("family", [ora.LAPLACIAN, ora.EXPONENTIAL])
@pytest.mark.parametrize("n", [3, 8, 13])
def test_family_path_probability_telescopes_to_target(family, n):
    # Lemma 1's telescoping holds for any non-negative kernel: the path product
    # is k(x_i, x_j) / deg(x_i) for every (i, j)
    rng = np.random.default_rng(100 + n)
    X = (rng.normal(size=(n, 3)) * 0.8).astype(np.float32)
    c = 1.1
    perm = rng.permutation(n)
    pos = np.empty(n, dtype=np.int64)
    pos[perm] = np.arange(n)
    K = _family_matrix(X, c, family)
    np.fill_diagonal(K, 0.0)
    for i in range(n):
        want = K[i] / K[i].sum()
        got = np.array([ora.path_prob(X, c, i, pos[j], perm=perm, kernel=family) for j in range(n)])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("family", [ora.LAPLACIAN, ora.EXPONENTIAL])
def test_family_weights_and_graph(family):
    # Eq. 2 with the family's k; two points: p_hat = 1, w = k
    X = np.array([[0.0, 0.0], [0.6, -0.8]], np.float32)  # l1 1.4, l2 1.0
    c = 0.5
    g = ora.build_graph(X, c, 4, 0, kernel=family)
    k = math.exp(-c * (1.4 if family == ora.LAPLACIAN else 1.0))
    assert len(g["w"]) == 1 and math.isclose(g["w"][0], k, rel_tol=1e-7)
    np.testing.assert_allclose(g["deg"], [k, k], rtol=1e-7)
