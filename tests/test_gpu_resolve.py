"""High-precision re-decision of flagged descents (fsg_params.resolve) and FP64
weights (fsg_params.weight_f64), through the C ABI against the FP64 oracle.

* Re-decision: every sample the FP32 path flagged is taken again; after it,
  every sample that is not flagged equals the oracle's descent (Algorithm 1),
  the re-decided ones included, and n_resolved counts the samples flagged
  without it.  Only decisions within 2^-20 of the threshold in high precision
  may stay flagged, so the residual is a small fraction of the FP32 flags.
* FP64 weights (Eq. 2): w = k / p_hat formed in FP64 from a kernel value
  within relative error 2^-20 and the FP32-accumulated degrees.  p_hat is
  monotone in both inclusion probabilities, so its relative error is at most
  the larger of theirs (k's plus a degree's, or 0 when capped at 1); the
  weight's is at most 2 x 2^-20 plus the larger endpoint degree error (taken
  twice, for margin).
"""
import numpy as np
import pytest

import oracle as ora
from paper_2310_13870_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HP_ETA = 2.0 ** -20


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


def run(fsg, X, p, L, seed, perm=None, edge_mode=0):
    pts = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    pt = None if perm is None else torch.from_numpy(np.asarray(perm, np.int32)).cuda()
    tree = fsg.fsg_build_tree(pts, perm=pt)
    bufs = fsg.fsg_build_graph(tree, p, L, seed, edge_mode=edge_mode)
    assert fsg.fsg_sync(tree) == 0
    m = int(bufs.m.item())
    out = dict(deg=bufs.deg.cpu().numpy(), samples=bufs.samples.cpu().numpy(), flags=bufs.flags.cpu().numpy(),
               src=bufs.src[:m].cpu().numpy(), dst=bufs.dst[:m].cpu().numpy(), w=bufs.w[:m].cpu().numpy(),
               stats=fsg.stats_dict(bufs))
    tree.close()
    return out


CASES = {
    # name: (points, sigma, L, seed, extra params, spatial order)
    "two_moons": (lambda: inputs.two_moons(n=2000, seed=0), 0.1, 32, 0, {}, False),
    "mixture_d10": (lambda: inputs.gaussian_mixture(n=20_000, d=10, seed=3), 1.5, 64, 1, {}, False),
    "mixture_include": (lambda: inputs.gaussian_mixture(n=6_000, d=5, k=4, box=3.0, seed=4), 1.0, 48, 2,
                        {"self_mode": 1}, False),
    "generic_d40": (lambda: inputs.gaussian_mixture(n=5_000, d=40, k=5, box=3.0, seed=5), 2.5, 32, 3, {}, False),
    "split_d24": (lambda: inputs.gaussian_mixture(n=6_000, d=24, k=6, box=5.0, seed=6), 1.5, 32, 4,
                  {"precision": 2}, True),
    "approx_d10": (lambda: inputs.gaussian_mixture(n=6_000, d=10, seed=7), 1.5, 32, 5,
                   {"precision": 2, "kde_eps": 1.0 / (6.0 * np.log(6000))}, True),
    "digits_tc": (lambda: inputs.digit_like(n=3_000, seed=8), None, 16, 6, {}, False),
    # the split form above d = 64 on FP32 data (digit images with a jitter
    # below one grey level); its flagged samples take the per-sample walker
    "split_d200": (lambda: (inputs.digit_like(n=2_000, d=200, seed=10).astype(np.float64) +
                            np.random.Generator(np.random.PCG64(10)).uniform(0.0, 1.0 / 255.0, (2_000, 200))
                            ).astype(np.float32), 3.0, 16, 8, {"precision": 2}, False),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_resolved_samples_equal_the_oracle(fsg, case):
    make, sigma, L, seed, extra, spatial = CASES[case]
    X = make()
    n = X.shape[0]
    if sigma is None:
        sigma = inputs.median_pair_distance(X, m=1024) / 2
    perm = fsg.fsg_spatial_order(X) if spatial else None
    base = run(fsg, X, fsg.params(sigma, **extra), L, seed, perm=perm)
    res = run(fsg, X, fsg.params(sigma, resolve=True, **extra), L, seed, perm=perm)
    before = (base["flags"] & 1) != 0
    after = (res["flags"] & 1) != 0
    assert res["stats"]["status"] == 0
    assert res["stats"]["n_resolved"] == int(before.sum())
    assert before.sum() > 0, "no flagged sample to re-decide in this case"
    assert after.sum() <= max(2, before.sum() // 20), (int(after.sum()), int(before.sum()))
    # samples never flagged are untouched
    np.testing.assert_array_equal(res["samples"][~before], base["samples"][~before])
    # every query with a re-decided sample, plus a spread of others, against the oracle
    q = np.unique(np.concatenate([np.nonzero(before.any(1))[0], np.arange(0, n, max(1, n // 64))]))
    if case == "digits_tc":
        q = q[:96]
    osmp, _, _ = ora.sample(X, ora.gamma(sigma), L, seed, queries=q, perm=perm,
                            self_mode=extra.get("self_mode", 0))
    bad = (res["samples"][q] != osmp) & ~after[q]
    assert not bad.any(), f"{int(bad.sum())} unflagged samples differ from the oracle"
    redecided = before[q] & ~after[q]
    assert (res["samples"][q][redecided] == osmp[redecided]).all()


@pytest.mark.parametrize("edge_mode", [0, 1])
def test_f64_weights_within_the_bound(fsg, edge_mode):
    X = inputs.gaussian_mixture(n=8_000, d=6, k=5, box=4.0, seed=9)
    sigma, L, seed = 1.2, 32, 7
    gam = ora.gamma(sigma)
    g = run(fsg, X, fsg.params(sigma, weight_f64=True), L, seed, edge_mode=edge_mode)
    g32 = run(fsg, X, fsg.params(sigma), L, seed, edge_mode=edge_mode)
    assert g["w"].dtype == np.float64
    np.testing.assert_array_equal(g["src"], g32["src"])
    np.testing.assert_array_equal(g["dst"], g32["dst"])
    deg_o = ora.degrees(X, gam)
    _, w_o = ora.weights(X, gam, L, deg_o, g["src"], g["dst"])
    ed = np.abs(g["deg"] - deg_o) / deg_o
    bound = 2.0 * HP_ETA + 2.0 * np.maximum(ed[g["src"]], ed[g["dst"]]) + 1e-12
    rel = np.abs(g["w"] - w_o) / w_o
    assert (rel <= bound).all(), float((rel / bound).max())
    # pairs whose two inclusion probabilities are capped at 1 carry w = k: 2^-20
    k_o, _ = ora.weights(X, gam, L, deg_o, g["src"], g["dst"])
    capped = (L * k_o >= deg_o[g["src"]] * (1 + 1e-4)) & (L * k_o >= deg_o[g["dst"]] * (1 + 1e-4))
    assert capped.any()
    assert (np.abs(g["w"][capped] - k_o[capped]) <= HP_ETA * k_o[capped]).all()
    # the FP32 weights are within their own 1e-4 of the FP64 ones
    np.testing.assert_allclose(g32["w"], g["w"], rtol=1e-4)


def test_resolve_and_f64_refused_where_unsupported(fsg):
    X = inputs.two_moons(n=500, seed=1)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    for extra in ({"schedule": fsg.FSG_SCHED_LEVELWISE, "resolve": True},
                  {"kernel": fsg.FSG_KERNEL_LAPLACIAN, "resolve": True},
                  {"kernel": fsg.FSG_KERNEL_EXPONENTIAL, "weight_f64": True}):
        with pytest.raises(fsg.FsgError) as e:
            fsg.fsg_build_graph(tree, fsg.params(0.1, **extra), 8, 0)
        assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()
    with pytest.raises(fsg.FsgError) as e:  # host buffers are float32
        fsg.fsg_build_graph_host(X, fsg.params(0.1, weight_f64=True), 8, 0)
    assert e.value.status == fsg.FSG_ERR_INVALID_ARG
