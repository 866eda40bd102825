"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (derived from the FP32 arithmetic of each path):
  * KDE / degree:  |g_gpu - g_ora| <= 1e-5 g_ora + n 2^-126 (FP32 evaluations
    with direct differences, ex2.approx, runs of <= 64 terms, pairwise bins);
  * samples: identical to the oracle's unless the GPU flagged the sample (a
    decision within its error bound of the ratio);
  * weights: relative 1e-4 (k and both degrees each within ~1e-5).
"""
import math

import numpy as np
import pytest

import oracle as ora
from paper_2310_13870_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEG_RTOL = 1e-5
W_RTOL = 1e-4
TINY = 2.0 ** -126


@pytest.fixture(scope="module")
def fsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_13870_gb300 import fsg as _fsg
    import os
    if not os.path.exists(_fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    _fsg.load()
    return _fsg


def gpu_graph(fsg, X, sigma, L, seed, edge_mode=0, perm=None, leaf_max=0, **pk):
    pts = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    pt = None if perm is None else torch.from_numpy(np.asarray(perm, np.int32)).cuda()
    tree = fsg.fsg_build_tree(pts, perm=pt, leaf_max=leaf_max)
    bufs = fsg.fsg_build_graph(tree, fsg.params(sigma, **pk), L, seed, edge_mode=edge_mode)
    assert fsg.fsg_sync(tree) == 0
    torch.cuda.synchronize()
    m = int(bufs.m.item())
    out = dict(deg=bufs.deg.cpu().numpy(), samples=bufs.samples.cpu().numpy(), flags=bufs.flags.cpu().numpy(),
               src=bufs.src[:m].cpu().numpy(), dst=bufs.dst[:m].cpu().numpy(), w=bufs.w[:m].cpu().numpy(),
               stats=fsg.stats_dict(bufs), m=m)
    tree.close()
    return out


def check_degrees(deg_gpu, deg_ora, n):
    err = np.abs(deg_gpu - deg_ora)
    bound = DEG_RTOL * deg_ora + n * TINY
    assert (err <= bound).all(), f"max rel err {np.max(err / np.maximum(deg_ora, 1e-300)):.3e}"


def check_samples(smp_gpu, flags, smp_ora):
    bad = (smp_gpu != smp_ora) & (flags == 0)
    assert not bad.any(), f"{int(bad.sum())} unflagged mismatches of {smp_gpu.size}"


def edge_set(src, dst):
    return set(zip(np.minimum(src, dst).tolist(), np.maximum(src, dst).tolist()))


# ----------------------------------------------------------------------------
# Small full-graph cases: every output against the oracle
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,sigma,L,seed", [
    (2000, 2, 0.1, 32, 0),     # two-moons workload, the small configuration
    (777, 2, 0.1, 7, 3),       # ragged n, odd L
    (1500, 5, 0.6, 64, 1),     # L = 64 (full sample mask)
    (300, 10, 1.5, 33, 2),     # L just above one warp
    (1001, 3, 0.3, 1, 4),      # L = 1: one sample per point
])
def test_full_graph_matches_oracle(fsg, n, d, sigma, L, seed):
    if d == 2:
        X = inputs.two_moons(n=n, seed=seed)
    else:
        X = inputs.gaussian_mixture(n=n, d=d, k=5, box=3.0, seed=seed)
    gam = ora.gamma(sigma)
    g = gpu_graph(fsg, X, sigma, L, seed)
    o = ora.build_graph(X, gam, L, seed)
    check_degrees(g["deg"], o["deg"], n)
    check_samples(g["samples"], g["flags"], o["samples"])
    flagged = (g["flags"] != 0).sum()
    assert flagged <= 0.01 * n * L
    assert g["stats"]["n_flagged"] == flagged
    assert g["stats"]["n_samples"] == n * L
    assert g["stats"]["status"] == 0
    # edges: the same set up to pairs touched by flagged samples
    eg, eo = edge_set(g["src"], g["dst"]), edge_set(o["src"], o["dst"])
    assert len(eg) == g["m"]  # SET: no duplicate pair
    fl_pts = set(np.nonzero((g["flags"] != 0).any(1))[0].tolist())
    for (a, b) in eg ^ eo:
        assert a in fl_pts or b in fl_pts
    # weights of common edges
    wo = {(a, b): w for a, b, w in zip(o["src"].tolist(), o["dst"].tolist(), o["w"].tolist())}
    for a, b, w in zip(g["src"].tolist(), g["dst"].tolist(), g["w"].tolist()):
        key = (min(a, b), max(a, b))
        if key in wo:
            assert math.isclose(w, wo[key], rel_tol=W_RTOL), (key, w, wo[key])
    assert (g["src"] != g["dst"]).all()


def test_multi_edges_and_include_self(fsg):
    X = inputs.two_moons(n=500, seed=7)
    gam = ora.gamma(0.1)
    g = gpu_graph(fsg, X, 0.1, 12, 5, edge_mode=1, self_mode=1)
    o = ora.build_graph(X, gam, 12, 5, self_mode=ora.SELF_INCLUDE, edge_mode=ora.EDGES_MULTI)
    check_degrees(g["deg"], o["deg"], 500)
    check_samples(g["samples"], g["flags"], o["samples"])
    n_self = int((g["samples"] == np.arange(500)[:, None]).sum())
    assert g["stats"]["n_self"] == n_self
    assert g["m"] == 500 * 12 - n_self
    if not (g["flags"] != 0).any():
        assert g["m"] == len(o["src"])
        np.testing.assert_array_equal(g["src"], o["src"])
        np.testing.assert_array_equal(g["dst"], o["dst"])
        np.testing.assert_allclose(g["w"], o["w"], rtol=W_RTOL)


def test_sigma_sq_convention_and_given_order(fsg):
    X = inputs.gaussian_mixture(n=1200, d=3, k=4, box=2.0, seed=4)
    perm = np.random.default_rng(0).permutation(1200)
    gam = ora.gamma(0.5, ora.SIGMA_SQ)
    g = gpu_graph(fsg, X, 0.5, 16, 11, perm=perm, scale_conv=1)
    o = ora.build_graph(X, gam, 16, 11, perm=perm)
    check_degrees(g["deg"], o["deg"], 1200)
    check_samples(g["samples"], g["flags"], o["samples"])


@pytest.mark.parametrize("leaf_max", [64, 128, 1024])
def test_leaf_sizes_give_identical_samples(fsg, leaf_max):
    # The split between bin pass and leaf finish is a schedule choice only.
    X = inputs.two_moons(n=3001, seed=1)
    gam = ora.gamma(0.1)
    g = gpu_graph(fsg, X, 0.1, 8, 2, leaf_max=leaf_max)
    q = np.arange(0, 3001, 13)
    smp, _, _ = ora.sample(X, gam, 8, 2, queries=q)
    check_samples(g["samples"][q], g["flags"][q], smp)
    check_degrees(g["deg"][q], ora.degrees(X, gam, queries=q), 3001)


@pytest.mark.parametrize("d", [1, 4, 7, 16, 17, 33, 64])
def test_dimensions(fsg, d):
    X = inputs.gaussian_mixture(n=900, d=d, k=3, box=2.0, seed=d)
    sigma = 0.4 * math.sqrt(d)
    gam = ora.gamma(sigma)
    g = gpu_graph(fsg, X, sigma, 10, d)
    o = ora.build_graph(X, gam, 10, d)
    check_degrees(g["deg"], o["deg"], 900)
    check_samples(g["samples"], g["flags"], o["samples"])


@pytest.mark.parametrize("n,d", [(700, 100), (601, 1000), (500, 4096)])
def test_wide_dimensions(fsg, n, d):
    # the FP32 generic passes up to the widest d the library takes (FP32
    # data, so AUTO keeps FP32): many 32-coordinate chunks, ragged n.  The
    # squared distance sums d rounded terms, so a term with exponent a (log2
    # units) is within ln2 a (d + 3) 2^-24 relative (plus ex2's 2^-22 and the
    # sums' roundings); the degrees are checked against that bound over each
    # query's terms where it exceeds 1e-5.  sigma = sqrt(d) keeps a near 1.5,
    # where the typical error stays far inside the 2^-13 decision flags.
    from scipy.spatial.distance import cdist
    X = inputs.gaussian_mixture(n=n, d=d, k=3, box=2.0, seed=d)
    sigma = math.sqrt(d)
    gam = ora.gamma(sigma)
    g = gpu_graph(fsg, X, sigma, 8, d)
    o = ora.build_graph(X, gam, 8, d)
    Xd = X.astype(np.float64)
    a = gam * math.log2(math.e) * cdist(Xd, Xd, "sqeuclidean")
    kv = np.exp2(-a)
    np.fill_diagonal(kv, 0.0)
    bound = (kv * a).sum(1) * math.log(2) * (d + 3) * 2.0 ** -24 + o["deg"] * (2.0 ** -22 + 96 * 2.0 ** -24)
    err = np.abs(g["deg"] - o["deg"])
    assert (err <= np.maximum(bound, DEG_RTOL * o["deg"]) + n * TINY).all(), float((err / o["deg"]).max())
    check_samples(g["samples"], g["flags"], o["samples"])


def test_digit_like_d784(fsg):
    # 784-dimensional 8-bit images, sigma = median pairwise distance / 2.
    X = inputs.digit_like(n=2500, seed=3)
    sigma = inputs.median_pair_distance(X, m=1024) / 2
    gam = ora.gamma(sigma)
    g = gpu_graph(fsg, X, sigma, 16, 5)
    q = np.arange(0, 2500, 11)
    check_degrees(g["deg"][q], ora.degrees(X, gam, queries=q), 2500)
    smp, _, _ = ora.sample(X, gam, 16, 5, queries=q)
    check_samples(g["samples"][q], g["flags"][q], smp)


# ----------------------------------------------------------------------------
# Degenerate inputs
# ----------------------------------------------------------------------------
def test_single_point(fsg):
    X = np.zeros((1, 3), np.float32)
    g = gpu_graph(fsg, X, 1.0, 4, 0)
    assert (g["samples"] == -1).all() and g["m"] == 0 and g["deg"][0] == 0.0
    assert g["stats"]["n_empty"] == 4
    gi = gpu_graph(fsg, X, 1.0, 4, 0, self_mode=1)
    assert (gi["samples"] == 0).all() and gi["m"] == 0 and gi["deg"][0] == 1.0


def test_two_points_closed_form(fsg):
    X = np.array([[0.0, 0.0], [0.3, 0.4]], np.float32)
    g = gpu_graph(fsg, X, 0.5, 6, 1)
    k = math.exp(-ora.gamma(0.5) * (float(np.float32(0.3)) ** 2 + float(np.float32(0.4)) ** 2))
    np.testing.assert_allclose(g["deg"], [k, k], rtol=DEG_RTOL)
    assert (g["samples"][0] == 1).all() and (g["samples"][1] == 0).all()
    assert g["m"] == 1 and math.isclose(float(g["w"][0]), k, rel_tol=W_RTOL)


def test_identical_points(fsg):
    n, L = 37, 5
    X = np.full((n, 2), 0.25, np.float32)
    g = gpu_graph(fsg, X, 1.0, L, 3)
    np.testing.assert_allclose(g["deg"], n - 1, rtol=DEG_RTOL)
    assert (g["samples"] != np.arange(n)[:, None]).all()
    p = L / (n - 1)
    np.testing.assert_allclose(g["w"], 1.0 / (2 * p - p * p), rtol=W_RTOL)


def test_far_apart_points_have_no_samples(fsg):
    X = np.array([[0.0], [1.0e4], [2.0e4]], np.float32)
    g = gpu_graph(fsg, X, 0.1, 3, 0)
    assert (g["deg"] == 0).all() and (g["samples"] == -1).all() and g["m"] == 0


# ----------------------------------------------------------------------------
# Full-size Gaussian mixture (n = 100,000, d = 10, L = 64): sampled outputs
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def gmm_full(fsg):
    X = inputs.gaussian_mixture(n=100_000, d=10, seed=0)
    g = gpu_graph(fsg, X, 1.5, 64, 0)
    return X, g


def test_gmm_full_degrees_sampled(gmm_full):
    X, g = gmm_full
    gam = ora.gamma(1.5)
    q = np.random.default_rng(5).choice(100_000, size=512, replace=False)
    check_degrees(g["deg"][q], ora.degrees(X, gam, queries=q), 100_000)


def test_gmm_full_samples_and_weights_sampled(gmm_full):
    X, g = gmm_full
    gam = ora.gamma(1.5)
    q = np.random.default_rng(6).choice(100_000, size=48, replace=False)
    smp, _, _ = ora.sample(X, gam, 64, 0, queries=q)
    check_samples(g["samples"][q], g["flags"][q], smp)
    # weights of the oracle's own sampled pairs of these queries, against the GPU edge list
    src = np.repeat(q, 64)
    dst = smp.reshape(-1)
    keep = dst >= 0
    src, dst = src[keep], dst[keep]
    pts = np.unique(np.concatenate([src, dst]))
    deg = np.zeros(100_000)
    deg[pts] = ora.degrees(X, gam, queries=pts)
    _, w_ora = ora.weights(X, gam, 64, deg, src, dst)
    gkey = {}
    for a, b, w in zip(g["src"].tolist(), g["dst"].tolist(), g["w"].tolist()):
        gkey[(min(a, b), max(a, b))] = w
    found = 0
    for a, b, w in zip(src.tolist(), dst.tolist(), w_ora.tolist()):
        key = (min(a, b), max(a, b))
        if key in gkey:
            found += 1
            assert math.isclose(gkey[key], w, rel_tol=W_RTOL)
    assert found >= 0.99 * len(src)
    st = g["stats"]
    assert st["n_samples"] == 100_000 * 64 and st["status"] == 0
    assert st["n_flagged"] <= 0.01 * st["n_samples"]
    assert g["m"] <= 100_000 * 64


# ----------------------------------------------------------------------------
# Distribution: chi-square of GPU sample frequencies vs k(x_i,x_j)/deg(v_i)
# ----------------------------------------------------------------------------
def test_gpu_sampler_chi_square(fsg):
    from scipy.spatial.distance import cdist
    from scipy.stats import chi2
    n, L = 160, 64
    X = inputs.two_moons(n=n, seed=9)
    sigma = 0.15
    gam = ora.gamma(sigma)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    p = fsg.params(sigma)
    queries = [0, 40, 80, 159]
    counts = np.zeros((len(queries), n))
    for seed in range(1000, 1800):
        smp, _ = fsg.fsg_sample_edges(tree, p, L, seed)
        s = smp[queries].cpu().numpy()
        for r in range(len(queries)):
            counts[r] += np.bincount(s[r], minlength=n)
    K = np.exp(-gam * cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean"))
    np.fill_diagonal(K, 0.0)
    for r, i in enumerate(queries):
        probs = K[i] / K[i].sum()
        exp = probs * counts[r].sum()
        order = np.argsort(exp)
        oc, ec, ao, ae = [], [], 0.0, 0.0
        for t in order:
            ao += counts[r][t]
            ae += exp[t]
            if ae >= 5:
                oc.append(ao); ec.append(ae); ao = ae = 0.0
        oc[-1] += ao; ec[-1] += ae
        oc, ec = np.array(oc), np.array(ec)
        pval = chi2.sf(((oc - ec) ** 2 / ec).sum(), len(ec) - 1)
        assert pval > 0.01 / len(queries), (i, pval)
    tree.close()


@pytest.mark.parametrize("mode", ["split", "exact_int"])
def test_gpu_sampler_chi_square_tensor_core_modes(fsg, mode):
    # the sampled frequencies of the tensor-core bin passes against the exact
    # k(x_i, x_j) / deg(x_i) (FP64): split precision on a spatial order (d = 20,
    # bins of 100 points), exact 8-bit products (digit-like, d = 64)
    from scipy.spatial.distance import cdist
    from scipy.stats import chi2
    n, L = 200, 64
    if mode == "split":
        X = inputs.gaussian_mixture(n=n, d=20, k=3, box=1.5, seed=4)
        sigma, prec = 1.5, fsg.FSG_PREC_SPLIT_BF16
        perm = torch.from_numpy(fsg.fsg_spatial_order(X)).cuda()
    else:
        X = inputs.digit_like(n=n, d=64, seed=5)
        sigma, prec, perm = 1.2, fsg.FSG_PREC_EXACT_INT, None
    gam = ora.gamma(sigma)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda(), perm=perm)
    p = fsg.params(sigma, precision=prec)
    queries = [0, 77, 150, 199]
    counts = np.zeros((len(queries), n))
    for seed in range(2000, 2600):
        smp, _ = fsg.fsg_sample_edges(tree, p, L, seed)
        s = smp[queries].cpu().numpy()
        for r in range(len(queries)):
            counts[r] += np.bincount(s[r], minlength=n)
    assert fsg.fsg_sync(tree) == 0
    K = np.exp(-gam * cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean"))
    np.fill_diagonal(K, 0.0)
    for r, i in enumerate(queries):
        probs = K[i] / K[i].sum()
        exp = probs * counts[r].sum()
        order = np.argsort(exp)
        oc, ec, ao, ae = [], [], 0.0, 0.0
        for t in order:
            ao += counts[r][t]
            ae += exp[t]
            if ae >= 5:
                oc.append(ao); ec.append(ae); ao = ae = 0.0
        oc[-1] += ao; ec[-1] += ae
        oc, ec = np.array(oc), np.array(ec)
        pval = chi2.sf(((oc - ec) ** 2 / ec).sum(), len(ec) - 1)
        assert pval > 0.01 / len(queries), (mode, i, pval)
    tree.close()


def test_host_entry_point_matches_device_path(fsg):
    X = inputs.two_moons(n=1000, seed=2)
    src, dst, w = fsg.fsg_build_graph_host(X, fsg.params(0.1), 16, 4)
    g = gpu_graph(fsg, X, 0.1, 16, 4)
    np.testing.assert_array_equal(src, g["src"])
    np.testing.assert_array_equal(dst, g["dst"])
    np.testing.assert_array_equal(w, g["w"])
    # a second call reuses the cached tree and gives the same result
    src2, dst2, w2 = fsg.fsg_build_graph_host(X, fsg.params(0.1), 16, 4)
    np.testing.assert_array_equal(src2, src)


# ----------------------------------------------------------------------------
# Symmetric bin pass: bin sizes from 61 to 128 points (1..3 bins per warp,
# partial last block), d with 16- and 8-point mirror batches; against the
# oracle and against the plain pass (leaf_max 1024 gives bins > 128)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [100, 976, 1000, 3905, 4097, 8192, 12289])
@pytest.mark.parametrize("d", [3, 16, 20, 48])
def test_symmetric_pass_bin_sizes(fsg, n, d):
    # d <= 16: lane-aligned bins; d > 16: triangle of 128-position tiles
    X = inputs.gaussian_mixture(n=n, d=d, k=4, box=2.0, seed=n + d)
    sigma = {3: 1.0, 16: 2.0, 20: 2.0, 48: 3.0}[d]
    gam = ora.gamma(sigma)
    L, seed = 8, 11
    g = gpu_graph(fsg, X, sigma, L, seed)
    gp = gpu_graph(fsg, X, sigma, L, seed, leaf_max=1024)
    q = np.unique(np.linspace(0, n - 1, 97).astype(np.int64))
    check_degrees(g["deg"][q], ora.degrees(X, gam, queries=q), n)
    np.testing.assert_allclose(g["deg"], gp["deg"], rtol=2e-5)
    smp, _, _ = ora.sample(X, gam, L, seed, queries=q)
    check_samples(g["samples"][q], g["flags"][q], smp)
    both = (g["flags"] == 0) & (gp["flags"] == 0)
    np.testing.assert_array_equal(g["samples"][both], gp["samples"][both])


def test_bin_pass_evals(fsg):
    for n, d, sym in [(10_000, 10, True), (10_000, 17, True), (50, 3, False), (3000, 20, True)]:
        X = inputs.gaussian_mixture(n=n, d=d, seed=1)
        tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
        ev = fsg.fsg_bin_pass_evals(tree, fsg.params(1.5))
        if sym:
            assert n * n // 2 < ev < 0.62 * n * n
        else:
            assert ev == n * n
        assert fsg.fsg_bin_pass_evals(tree, fsg.params(1.5, schedule=fsg.FSG_SCHED_LEVELWISE)) == 0
        tree.close()


@pytest.mark.parametrize("n", [2, 3, 5, 64, 129])
def test_generic_d_small_n(fsg, n):
    X = inputs.gaussian_mixture(n=n, d=24, k=2, box=1.0, seed=n)
    gam = ora.gamma(3.0)
    g = gpu_graph(fsg, X, 3.0, 6, 4)
    o = ora.build_graph(X, gam, 6, 4)
    check_degrees(g["deg"], o["deg"], n)
    check_samples(g["samples"], g["flags"], o["samples"])


# ----------------------------------------------------------------------------
# Self term and edge semantics on the d > 16 FP32 path and the tensor-core path
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("path", ["generic", "tc"])
def test_include_self_and_multi_edges_large_d(fsg, path):
    if path == "generic":
        X = inputs.gaussian_mixture(n=900, d=24, k=3, box=1.5, seed=21)
        sigma = 2.5
    else:
        X = inputs.digit_like(n=900, d=784, seed=21)
        sigma = inputs.median_pair_distance(X, m=900) / 2
    gam = ora.gamma(sigma)
    g = gpu_graph(fsg, X, sigma, 10, 6, edge_mode=1, self_mode=1)
    o = ora.build_graph(X, gam, 10, 6, self_mode=ora.SELF_INCLUDE, edge_mode=ora.EDGES_MULTI)
    check_degrees(g["deg"], o["deg"], 900)
    check_samples(g["samples"], g["flags"], o["samples"])
    n_self = int((g["samples"] == np.arange(900)[:, None]).sum())
    assert g["stats"]["n_self"] == n_self
    assert g["m"] == 900 * 10 - n_self
    e = ora.build_graph(X, gam, 10, 6)  # SET semantics, EXCLUDE, on the same path
    ge = gpu_graph(fsg, X, sigma, 10, 6)
    check_samples(ge["samples"], ge["flags"], e["samples"])
    assert (ge["src"] != ge["dst"]).all()


# ----------------------------------------------------------------------------
# The paper's largest two-moons size: n = 1,000,000 (bins of ~488 points, the
# non-symmetric bin pass and the general leaf finish), sampled against the oracle
# ----------------------------------------------------------------------------
def test_two_moons_one_million(fsg):
    n = 1_000_000
    X = inputs.two_moons(n=n, seed=11)
    g = gpu_graph(fsg, X, 0.02, 8, 3)
    assert g["stats"]["status"] == 0 and g["stats"]["n_samples"] == n * 8
    assert g["stats"]["n_evals"] >= n * n  # int64 counts past 2^31
    q = np.random.default_rng(1).choice(n, size=6, replace=False)
    gam = ora.gamma(0.02)
    check_degrees(g["deg"][q], ora.degrees(X, gam, queries=q), n)
    smp, _, _ = ora.sample(X, gam, 8, 3, queries=q)
    check_samples(g["samples"][q], g["flags"][q], smp)
    assert g["stats"]["n_flagged"] <= 0.01 * n * 8
