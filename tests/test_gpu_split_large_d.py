"""Split precision for FP32 data at d > 64 (FSG_PREC_SPLIT_BF16 on the
tensor-core bin pass and leaf kernel): every coordinate as three BF16 parts,
x.y from six exact part products accumulated in FP32 in TMEM, no centring,
||x - y||^2 = ||x||^2 + ||y||^2 - 2 x.y with the norms summed in FP64.

Stated bound, per pair: the dot product carries at most one rounding of
2^-22 of sum |x_t y_t| <= |x||y| per accumulation step (S = 6 dpad / 16 MMA
steps of K = 16, dpad = d rounded up to 64), the three dropped part products
lie below 2^-23 |x||y|, and the norms and the expansion add three roundings
of 2^-24 (|x|^2 + |y|^2), so the squared distance is off by at most
(S + 1) 2^-22 (|x|^2 + |y|^2) and a kernel value by gamma times that
(relative), plus ex2's 2^-22.  Degrees are checked against the oracle with
that bound summed over each query's terms (and the FP32 bin sums' 64
roundings); unflagged samples must be the oracle's (the mode flags decisions
at 2^-10, which covers gamma (|x|^2 + |y|^2) (S + 1) 2^-22 on these data)."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle as ora
from paper_2310_13870_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W_RTOL = 2e-3
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


def jittered_digits(n, d, seed):
    """Digit-like images with a uniform jitter below one grey level: FP32
    data that are not multiples of 1/255 (the 8-bit path does not apply)."""
    X = inputs.digit_like(n=n, d=d, seed=seed).astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    return (X + rng.uniform(0.0, 1.0 / 255.0, size=X.shape)).astype(np.float32)


def degree_bound(X, gamma, q, kv):
    """Per-query bound on |deg_gpu - deg_exact| of the split form (module doc)."""
    d = X.shape[1]
    dpad = (d + 63) // 64 * 64
    steps = 6 * dpad // 16
    sq = (X.astype(np.float64) ** 2).sum(1)
    rel = gamma * (steps + 1) * 2.0 ** -22 * (sq[q][:, None] + sq[None, :]) + 2.0 ** -22
    return (kv * rel).sum(1) + kv.sum(1) * 64 * 2.0 ** -24


def run(fsg, X, sigma, L, seed, precision, leaf_max=0, self_mode=0):
    pts = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    tree = fsg.fsg_build_tree(pts, leaf_max=leaf_max)
    p = fsg.params(sigma, precision=precision, self_mode=self_mode)
    bufs = fsg.fsg_build_graph(tree, p, L, seed)
    assert fsg.fsg_sync(tree) == 0
    m = int(bufs.m.item())
    out = dict(deg=bufs.deg.cpu().numpy(), samples=bufs.samples.cpu().numpy(), flags=bufs.flags.cpu().numpy(),
               src=bufs.src[:m].cpu().numpy(), dst=bufs.dst[:m].cpu().numpy(), w=bufs.w[:m].cpu().numpy(),
               stats=fsg.stats_dict(bufs), evals=fsg.fsg_bin_pass_evals(tree, p))
    tree.close()
    return out


@pytest.mark.parametrize("kind,n,d,sigma,L,seed,leaf_max", [
    ("digits", 3000, 784, 4.5, 32, 0, 0),    # the digit workload's dimension, FP32 data
    ("digits", 2301, 100, 2.0, 16, 1, 0),    # ragged n, d not a multiple of 64
    ("mixture", 4000, 128, 9.0, 64, 2, 0),   # mixture data, full sample mask
    ("mixture", 3000, 65, 6.0, 24, 3, 512),  # the smallest d; bins of up to 512 points (FP32 leaf values)
])
def test_split_large_d_matches_oracle(fsg, kind, n, d, sigma, L, seed, leaf_max):
    X = jittered_digits(n, d, seed) if kind == "digits" else \
        inputs.gaussian_mixture(n=n, d=d, k=6, box=1.5, seed=seed)
    g = run(fsg, X, sigma, L, seed, fsg.FSG_PREC_SPLIT_BF16, leaf_max=leaf_max)
    assert g["stats"]["status"] == 0 and g["stats"]["n_bin_evals"] == g["evals"]
    gam = ora.gamma(sigma)
    q = np.arange(0, n, 9)
    Xd = X.astype(np.float64)
    kv = np.exp(-gam * cdist(Xd[q], Xd, "sqeuclidean"))
    kv[np.arange(q.size), q] = 0.0
    want = kv.sum(1)
    np.testing.assert_allclose(want, ora.degrees(X, gam, queries=q), rtol=1e-12)
    err = np.abs(g["deg"][q] - want)
    bound = degree_bound(X, gam, q, kv)
    assert (err <= bound + n * TINY).all(), float((err / bound).max())
    smp, _, _ = ora.sample(X, gam, L, seed, queries=q)
    assert not ((g["samples"][q] != smp) & (g["flags"][q] == 0)).any()
    assert g["stats"]["n_flagged"] <= 0.05 * n * L
    # the tensor-core bin pass ran: its executed-pair count, or (where a
    # single bin chunk makes both counts n^2) its rounding, differs from the
    # FP32 pass's
    fp = run(fsg, X, sigma, L, seed, fsg.FSG_PREC_FP32, leaf_max=leaf_max)
    assert g["evals"] != fp["evals"] or not np.array_equal(g["deg"], fp["deg"])
    np.testing.assert_allclose(g["deg"], fp["deg"], rtol=np.max(bound / want) + 2e-5)
    sel = np.arange(0, g["src"].size, max(1, g["src"].size // 1500))
    odeg = ora.degrees(X, gam)
    _, ow = ora.weights(X, gam, L, odeg, g["src"][sel], g["dst"][sel])
    np.testing.assert_allclose(g["w"][sel], ow, rtol=W_RTOL)


def test_split_large_d_include_self(fsg):
    X = jittered_digits(1500, 256, 5)
    g = run(fsg, X, 3.0, 16, 7, fsg.FSG_PREC_SPLIT_BF16, self_mode=fsg.FSG_SELF_INCLUDE)
    gam = ora.gamma(3.0)
    want = ora.degrees(X, gam, self_mode=ora.SELF_INCLUDE)
    np.testing.assert_allclose(g["deg"], want, rtol=1e-4)
    smp, _, _ = ora.sample(X, gam, 16, 7, self_mode=ora.SELF_INCLUDE)
    assert not ((g["samples"] != smp) & (g["flags"] == 0)).any()


def test_split_large_d_follows_tree_update(fsg):
    # the three-part image is refilled by fsg_tree_update: the same result as
    # a fresh tree on the new points, bit for bit
    X1, X2 = jittered_digits(2000, 200, 8), jittered_digits(2000, 200, 9)
    p = fsg.params(3.0, precision=fsg.FSG_PREC_SPLIT_BF16)
    tree = fsg.fsg_build_tree(torch.from_numpy(X1).cuda())
    fsg.fsg_degrees(tree, p)
    fsg.fsg_tree_update(tree, torch.from_numpy(X2).cuda())
    b1 = fsg.fsg_build_graph(tree, p, 16, 3)
    assert fsg.fsg_sync(tree) == 0
    tree.close()
    tree = fsg.fsg_build_tree(torch.from_numpy(X2).cuda())
    b2 = fsg.fsg_build_graph(tree, p, 16, 3)
    assert fsg.fsg_sync(tree) == 0
    tree.close()
    np.testing.assert_array_equal(b1.deg.cpu().numpy(), b2.deg.cpu().numpy())
    np.testing.assert_array_equal(b1.samples.cpu().numpy(), b2.samples.cpu().numpy())


def test_split_large_d_refusals(fsg):
    X = jittered_digits(1000, 100, 4)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    for kw in (dict(kde_eps=1e-3),                             # the approximate pass is d <= 64 only
               dict(kernel=fsg.FSG_KERNEL_EXPONENTIAL),        # the split form is Gaussian only
               dict(schedule=fsg.FSG_SCHED_LEVELWISE)):        # the levelwise schedule is plain FP32
        with pytest.raises(fsg.FsgError) as e:
            fsg.fsg_degrees(tree, fsg.params(2.0, precision=fsg.FSG_PREC_SPLIT_BF16, **kw))
        assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()


@pytest.mark.parametrize("n,d", [(1, 100), (2, 100), (3, 65), (77, 300), (129, 128), (300, 4096)])
def test_split_large_d_small_and_wide(fsg, n, d):
    # one point (no other mass: every sample empty), two points (each the
    # other's only neighbour, weight k), a single bin under one tile, a
    # ragged tile, and the widest d the library takes
    X = jittered_digits(n, d, 40 + n)
    sigma = 6.0 if d < 1000 else 15.0
    g = run(fsg, X, sigma, 8, 3, fsg.FSG_PREC_SPLIT_BF16)
    assert g["stats"]["status"] == 0
    gam = ora.gamma(sigma)
    want = ora.degrees(X, gam)
    if n == 1:
        assert g["deg"][0] == 0.0 and (g["samples"] == -1).all() and g["src"].size == 0
        return
    kv = np.exp(-gam * cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean"))
    np.fill_diagonal(kv, 0.0)
    q = np.arange(n)
    assert (np.abs(g["deg"] - want) <= degree_bound(X, gam, q, kv) + n * TINY).all()
    smp, _, _ = ora.sample(X, gam, 8, 3)
    assert not ((g["samples"] != smp) & (g["flags"] == 0)).any()
    if n == 2:
        assert (g["samples"] == np.array([[1], [0]])).all()
        np.testing.assert_allclose(g["w"], kv[0, 1], rtol=W_RTOL)
