"""Split-precision bin pass (FSG_PREC_SPLIT_BF16: centred tiles, three-part
BF16 split, six tensor-core products, FP32 accumulation) against the FP64
oracle on the same spatial tree order.  Its stated bound: every degree within
SPLIT_DEG_RTOL of the oracle's, and every sample the oracle's unless a
decision was flagged under the mode's default tolerance (2^-10).  For d in
17..64 the leaf phase uses the same arithmetic (the bin's points and the
items' queries centred at the bin's centre), so leaf values and edge weights
share the bound; for d <= 16 the leaf phase runs in FP32."""
import math

import numpy as np
import pytest

import oracle as ora
from paper_2310_13870_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT_DEG_RTOL = 1e-3  # measured: <= 4e-4 (d = 64, n = 20,000 and 100,000)
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


def run(fsg, X, perm, sigma, L, seed, precision, edge_mode=0, self_mode=0):
    pts = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    tree = fsg.fsg_build_tree(pts, perm=torch.from_numpy(perm).cuda())
    bufs = fsg.fsg_build_graph(tree, fsg.params(sigma, precision=precision, self_mode=self_mode), L, seed,
                               edge_mode=edge_mode)
    assert fsg.fsg_sync(tree) == 0
    m = int(bufs.m.item())
    out = dict(deg=bufs.deg.cpu().numpy(), samples=bufs.samples.cpu().numpy(), flags=bufs.flags.cpu().numpy(),
               src=bufs.src[:m].cpu().numpy(), dst=bufs.dst[:m].cpu().numpy(), w=bufs.w[:m].cpu().numpy(),
               stats=fsg.stats_dict(bufs), m=m)
    tree.close()
    return out


@pytest.mark.parametrize("n,d,sigma,L,seed", [
    (3000, 64, 1.5, 32, 0),    # the mixture workload's dimension
    (5000, 10, 1.5, 64, 3),    # d <= 16: the FP32 leaf finish of that range behind it
    (2000, 2, 0.1, 32, 4),     # two moons's dimension
    (2777, 33, 1.5, 24, 1),    # ragged n, padded coordinates
    (4100, 17, 1.0, 64, 2),    # the smallest split dimension, full sample mask
])
def test_split_matches_oracle(fsg, n, d, sigma, L, seed):
    X = inputs.gaussian_mixture(n=n, d=d, k=6, box=4.0, seed=seed)
    perm = fsg.fsg_spatial_order(X)
    gam = ora.gamma(sigma)
    g = run(fsg, X, perm, sigma, L, seed, fsg.FSG_PREC_SPLIT_BF16)
    assert g["stats"]["status"] == 0
    q = np.arange(0, n, 7)
    want = ora.degrees(X, gam, queries=q)
    err = np.abs(g["deg"][q] - want)
    assert (err <= SPLIT_DEG_RTOL * want + n * TINY).all(), float((err / want).max())
    osmp, oflg, _ = ora.sample(X, gam, L, seed, queries=q, perm=perm)
    assert not ((g["samples"][q] != osmp) & (g["flags"][q] == 0)).any()
    assert g["stats"]["n_flagged"] <= 0.05 * n * L
    # edge weights: leaf values and degrees of the two end points, each within the bound
    o = ora.build_graph(X, gam, L, seed, perm=perm)
    wo = {(min(s, t), max(s, t)): w for s, t, w in zip(o["src"].tolist(), o["dst"].tolist(), o["w"].tolist())}
    for s, t, w in zip(g["src"].tolist(), g["dst"].tolist(), g["w"].tolist()):
        key = (min(s, t), max(s, t))
        if key in wo:
            assert math.isclose(w, wo[key], rel_tol=2 * SPLIT_DEG_RTOL), (key, w, wo[key])


@pytest.mark.parametrize("n,d", [(40, 20), (129, 64), (300, 48)])
def test_split_small_point_sets(fsg, n, d):
    # one bin, a ragged second query tile, bins of 75 points
    X = inputs.gaussian_mixture(n=n, d=d, k=2, box=2.0, seed=n)
    perm = fsg.fsg_spatial_order(X)
    gam = ora.gamma(1.5)
    g = run(fsg, X, perm, 1.5, 16, 7, fsg.FSG_PREC_SPLIT_BF16)
    want = ora.degrees(X, gam)
    assert (np.abs(g["deg"] - want) <= SPLIT_DEG_RTOL * want + n * TINY).all()
    osmp, _, _ = ora.sample(X, gam, 16, 7, perm=perm)
    assert not ((g["samples"] != osmp) & (g["flags"] == 0)).any()


def test_split_against_fp32_path(fsg):
    # same tree, same draws: degrees within the stated bound of the FP32 path's,
    # samples equal wherever neither path flagged
    X = inputs.gaussian_mixture(n=6000, d=48, seed=4)
    perm = fsg.fsg_spatial_order(X)
    a = run(fsg, X, perm, 1.5, 32, 5, fsg.FSG_PREC_FP32)
    b = run(fsg, X, perm, 1.5, 32, 5, fsg.FSG_PREC_SPLIT_BF16)
    np.testing.assert_allclose(b["deg"], a["deg"], rtol=SPLIT_DEG_RTOL)
    both = (a["flags"] == 0) & (b["flags"] == 0)
    np.testing.assert_array_equal(a["samples"][both], b["samples"][both])


def test_split_include_self_and_multi(fsg):
    X = inputs.gaussian_mixture(n=2500, d=24, seed=6)
    perm = fsg.fsg_spatial_order(X)
    g = run(fsg, X, perm, 1.5, 16, 3, fsg.FSG_PREC_SPLIT_BF16, edge_mode=1, self_mode=1)
    o = ora.build_graph(X, ora.gamma(1.5), 16, 3, perm=perm, self_mode=ora.SELF_INCLUDE,
                        edge_mode=ora.EDGES_MULTI)
    assert not ((g["samples"] != o["samples"]) & (g["flags"] == 0)).any()
    n_self = int((g["samples"] == np.arange(2500)[:, None]).sum())
    assert g["stats"]["n_self"] == n_self and g["m"] == 2500 * 16 - n_self


def test_split_refused_outside_its_range(fsg):
    # (d > 64 takes the tensor-core kernels on three-part images: tested in
    # test_gpu_split_large_d.py)
    X = inputs.gaussian_mixture(n=1000, d=32, seed=1)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    with pytest.raises(fsg.FsgError) as e:  # the levelwise schedule is the plain FP32 path only
        fsg.fsg_degrees(tree, fsg.params(1.5, precision=fsg.FSG_PREC_SPLIT_BF16, schedule=fsg.FSG_SCHED_LEVELWISE))
    assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()


def test_split_skips_zero_tiles_exactly(fsg):
    # four clusters far apart (box 60, sigma 1.5): on the spatial order most
    # tile pairs have every value below 2^-126 and are skipped, which must not
    # change any sum: every degree within the stated bound of the oracle, the
    # oracle's samples wherever no decision was flagged
    X = inputs.gaussian_mixture(n=4096, d=32, k=4, box=60.0, seed=11)
    perm = fsg.fsg_spatial_order(X)
    gam = ora.gamma(1.5)
    g = run(fsg, X, perm, 1.5, 16, 3, fsg.FSG_PREC_SPLIT_BF16)
    st = g["stats"]
    assert st["status"] == 0 and 0 < st["n_bin_evals"] < 0.6 * 4096 * 4096
    want = ora.degrees(X, gam)
    assert (np.abs(g["deg"] - want) <= SPLIT_DEG_RTOL * want + 4096 * TINY).all()
    q = np.arange(0, 4096, 5)
    osmp, _, _ = ora.sample(X, gam, 16, 3, queries=q, perm=perm)
    assert not ((g["samples"][q] != osmp) & (g["flags"][q] == 0)).any()
