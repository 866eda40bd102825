"""The plain FP32 levelwise schedule (FSG_SCHED_LEVELWISE: Algorithm 1 run
literally, both halves' KDEs summed afresh at every level) against the FP64
oracle, and against the fused schedule: both must give the oracle's samples
except where they flag a decision, the same degrees to FP32 accuracy, and the
same edge list wherever neither flagged."""
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


def run(fsg, X, sigma, L, seed, schedule, edge_mode=0, **pk):
    pts = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    tree = fsg.fsg_build_tree(pts)
    bufs = fsg.fsg_build_graph(tree, fsg.params(sigma, schedule=schedule, **pk), L, seed, edge_mode=edge_mode)
    assert fsg.fsg_sync(tree) == 0
    m = int(bufs.m.item())
    out = dict(deg=bufs.deg.cpu().numpy(), samples=bufs.samples.cpu().numpy(), flags=bufs.flags.cpu().numpy(),
               src=bufs.src[:m].cpu().numpy(), dst=bufs.dst[:m].cpu().numpy(), w=bufs.w[:m].cpu().numpy(),
               stats=fsg.stats_dict(bufs), m=m)
    tree.close()
    return out


def wmap(g):
    return {(min(a, b), max(a, b)): w for a, b, w in zip(g["src"].tolist(), g["dst"].tolist(), g["w"].tolist())}


@pytest.mark.parametrize("n,d,sigma,L,seed", [
    (2000, 2, 0.1, 32, 0),    # two-moons workload
    (1500, 10, 1.5, 64, 1),   # Gaussian mixture, full sample mask
    (777, 17, 1.5, 7, 2),     # runtime-d kernels, ragged n
    (333, 33, 2.0, 40, 3),
])
def test_levelwise_matches_oracle_and_fused(fsg, n, d, sigma, L, seed):
    X = inputs.two_moons(n=n, seed=seed) if d == 2 else inputs.gaussian_mixture(n=n, d=d, k=5, box=3.0, seed=seed)
    gam = ora.gamma(sigma)
    lw = run(fsg, X, sigma, L, seed, fsg.FSG_SCHED_LEVELWISE)
    fu = run(fsg, X, sigma, L, seed, fsg.FSG_SCHED_FUSED)
    o = ora.build_graph(X, gam, L, seed)
    err = np.abs(lw["deg"] - o["deg"])
    assert (err <= DEG_RTOL * o["deg"] + n * TINY).all()
    assert not ((lw["samples"] != o["samples"]) & (lw["flags"] == 0)).any()
    both = (lw["flags"] == 0) & (fu["flags"] == 0)
    np.testing.assert_array_equal(lw["samples"][both], fu["samples"][both])
    st = lw["stats"]
    assert st["status"] == 0 and st["n_samples"] == n * L
    assert st["n_flagged"] == int((lw["flags"] != 0).sum()) <= 0.01 * n * L
    # the plain schedule runs at least one full pass (the degrees) and at most depth passes
    assert n * n <= st["n_evals"] <= n * n * max(1, math.ceil(math.log2(n)))
    # edges: identical weights on common pairs, differences only at flagged points
    fl = set(np.nonzero((lw["flags"] != 0).any(1) | (fu["flags"] != 0).any(1))[0].tolist())
    a, b = wmap(lw), wmap(fu)
    for key in set(a) ^ set(b):
        assert key[0] in fl or key[1] in fl
    for key in set(a) & set(b):
        assert math.isclose(a[key], b[key], rel_tol=W_RTOL)
    wo = {(min(s, t), max(s, t)): w for s, t, w in zip(o["src"].tolist(), o["dst"].tolist(), o["w"].tolist())}
    for key in set(a) & set(wo):
        assert math.isclose(a[key], wo[key], rel_tol=W_RTOL)


def test_levelwise_multi_include(fsg):
    X = inputs.two_moons(n=400, seed=4)
    lw = run(fsg, X, 0.1, 12, 9, fsg.FSG_SCHED_LEVELWISE, edge_mode=1, self_mode=1)
    o = ora.build_graph(X, ora.gamma(0.1), 12, 9, self_mode=ora.SELF_INCLUDE, edge_mode=ora.EDGES_MULTI)
    assert not ((lw["samples"] != o["samples"]) & (lw["flags"] == 0)).any()
    n_self = int((lw["samples"] == np.arange(400)[:, None]).sum())
    assert lw["stats"]["n_self"] == n_self and lw["m"] == 400 * 12 - n_self


def test_levelwise_degrees_entry(fsg):
    X = inputs.gaussian_mixture(n=3000, d=10, seed=8)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    dl = fsg.fsg_degrees(tree, fsg.params(1.5, schedule=fsg.FSG_SCHED_LEVELWISE)).cpu().numpy()
    df = fsg.fsg_degrees(tree, fsg.params(1.5)).cpu().numpy()
    assert fsg.fsg_sync(tree) == 0
    tree.close()
    q = np.arange(0, 3000, 29)
    want = ora.degrees(X, ora.gamma(1.5), queries=q)
    assert (np.abs(dl[q] - want) <= DEG_RTOL * want + 3000 * TINY).all()
    np.testing.assert_allclose(dl, df, rtol=2e-5)


def test_levelwise_degenerate(fsg):
    one = np.zeros((1, 3), np.float32)
    g = run(fsg, one, 1.0, 4, 0, fsg.FSG_SCHED_LEVELWISE)
    assert (g["samples"] == -1).all() and g["m"] == 0 and g["deg"][0] == 0.0
    g = run(fsg, one, 1.0, 4, 0, fsg.FSG_SCHED_LEVELWISE, self_mode=1)
    assert (g["samples"] == 0).all() and g["m"] == 0 and g["deg"][0] == 1.0
    two = np.array([[0.0, 0.0], [0.3, 0.4]], np.float32)
    g = run(fsg, two, 0.5, 6, 1, fsg.FSG_SCHED_LEVELWISE)
    assert (g["samples"][0] == 1).all() and (g["samples"][1] == 0).all() and g["m"] == 1
    same = np.full((37, 2), 0.25, np.float32)
    g = run(fsg, same, 1.0, 5, 3, fsg.FSG_SCHED_LEVELWISE)
    np.testing.assert_allclose(g["deg"], 36, rtol=DEG_RTOL)
    assert (g["samples"] != np.arange(37)[:, None]).all()
    far = np.array([[0.0], [1.0e4], [2.0e4]], np.float32)
    g = run(fsg, far, 0.1, 3, 0, fsg.FSG_SCHED_LEVELWISE)
    assert (g["deg"] == 0).all() and (g["samples"] == -1).all() and g["m"] == 0


def test_levelwise_refuses_tensor_core_precision(fsg):
    X = inputs.digit_like(n=300, d=64, seed=1)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    with pytest.raises(fsg.FsgError) as e:
        fsg.fsg_degrees(tree, fsg.params(1.0, precision=fsg.FSG_PREC_EXACT_INT, schedule=fsg.FSG_SCHED_LEVELWISE))
    assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()


@pytest.mark.parametrize("n,d,sigma,L,seed", [
    (2000, 2, 0.1, 32, 0),
    (1500, 10, 1.5, 64, 1),
    (777, 17, 1.5, 7, 2),
])
def test_carried_denominator_variant(fsg, n, d, sigma, L, seed):
    # only the left half is summed below the root; g_R = g_node - g_L is
    # carried, and its error bound widens the flag tolerance: the oracle's
    # samples wherever no decision was flagged, with fewer evaluations
    X = inputs.two_moons(n=n, seed=seed) if d == 2 else inputs.gaussian_mixture(n=n, d=d, k=5, box=3.0, seed=seed)
    gam = ora.gamma(sigma)
    cv = run(fsg, X, sigma, L, seed, fsg.FSG_SCHED_CARRIED)
    lw = run(fsg, X, sigma, L, seed, fsg.FSG_SCHED_LEVELWISE)
    o = ora.build_graph(X, gam, L, seed)
    err = np.abs(cv["deg"] - o["deg"])
    assert (err <= DEG_RTOL * o["deg"] + n * TINY).all()
    assert not ((cv["samples"] != o["samples"]) & (cv["flags"] == 0)).any()
    both = (cv["flags"] == 0) & (lw["flags"] == 0)
    np.testing.assert_array_equal(cv["samples"][both], lw["samples"][both])
    st = cv["stats"]
    assert st["status"] == 0 and st["n_samples"] == n * L
    assert st["n_flagged"] <= 0.05 * n * L
    assert n * n <= st["n_evals"] < lw["stats"]["n_evals"]
