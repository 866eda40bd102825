"""GPU spatial tree order (FSG_ORDER_SPATIAL): a permutation, the same on
every build; every node above 32 points split at the tree's midpoint along
its widest coordinate, the left part not above the right part by more than
one histogram bucket (1/256 of the node's spread); compact blocks like the
host order's; recomputed by fsg_tree_update; and the sampled graph of such a
tree equals the oracle's on the same permutation wherever no decision was
flagged."""
import numpy as np
import pytest

import oracle as ora
from paper_2310_13870_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def gpu_order(fsg, X):
    tree = fsg.fsg_build_tree(torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda(),
                              order=fsg.FSG_ORDER_SPATIAL)
    perm = fsg.fsg_tree_perm(tree).cpu().numpy()
    tree.close()
    return perm


def node_split_violations(X, perm, leaf=32):
    """Nodes (midpoint rule) whose left part exceeds the right part along the
    node's widest coordinate by more than one bucket of its spread."""
    n = len(perm)
    Y = X[perm].astype(np.float64)
    bad, nodes = 0, [(0, n)]
    while nodes:
        nxt = []
        for lo, hi in nodes:
            if hi - lo <= leaf:
                continue
            P = Y[lo:hi]
            spread = P.max(0) - P.min(0)
            t = int(np.argmax(spread))
            mid = lo + (hi - lo) // 2
            if Y[lo:mid, t].max() - Y[mid:hi, t].min() > spread[t] / 256 * 1.001 + 1e-6:
                bad += 1
            nxt += [(lo, mid), (mid, hi)]
        nodes = nxt
    return bad


def block_spread(X, perm, B=128):
    Y = X[perm].astype(np.float64)
    nb = len(Y) // B
    Z = Y[: nb * B].reshape(nb, B, -1)
    return float(((Z - Z.mean(1, keepdims=True)) ** 2).sum(-1).mean())


@pytest.mark.parametrize("n,d", [(1, 3), (33, 2), (1000, 10), (20011, 10), (6000, 64)])
def test_gpu_order_is_a_deterministic_permutation(fsg, n, d):
    X = inputs.gaussian_mixture(n=n, d=d, seed=n)
    a = gpu_order(fsg, X)
    np.testing.assert_array_equal(np.sort(a), np.arange(n))
    np.testing.assert_array_equal(gpu_order(fsg, X), a)
    assert node_split_violations(X, a) == 0


def test_gpu_order_is_as_compact_as_the_host_order(fsg):
    X = inputs.gaussian_mixture(n=30000, d=10, seed=2)
    g = block_spread(X, gpu_order(fsg, X))
    h = block_spread(X, fsg.fsg_spatial_order(X))
    ident = block_spread(X, np.arange(len(X)))
    assert g <= 1.25 * h and g < 0.2 * ident, (g, h, ident)


def test_gpu_order_identical_points(fsg):
    X = np.ones((500, 4), np.float32)  # zero spread: split by position
    np.testing.assert_array_equal(np.sort(gpu_order(fsg, X)), np.arange(500))


def test_tree_update_recomputes_the_order(fsg):
    X1 = inputs.gaussian_mixture(n=5000, d=10, seed=1)
    X2 = inputs.gaussian_mixture(n=5000, d=10, seed=2)
    tree = fsg.fsg_build_tree(torch.from_numpy(X1).cuda(), order=fsg.FSG_ORDER_SPATIAL)
    fsg.fsg_tree_update(tree, torch.from_numpy(X2).cuda())
    got = fsg.fsg_tree_perm(tree).cpu().numpy()
    tree.close()
    np.testing.assert_array_equal(got, gpu_order(fsg, X2))


def test_spatial_order_refuses_a_caller_permutation(fsg):
    X = torch.from_numpy(inputs.gaussian_mixture(n=100, d=3, seed=0)).cuda()
    with pytest.raises(fsg.FsgError) as e:
        fsg.fsg_build_tree(X, perm=torch.arange(100, dtype=torch.int32).cuda(), order=fsg.FSG_ORDER_SPATIAL)
    assert e.value.status == fsg.FSG_ERR_INVALID_ARG


@pytest.mark.parametrize("precision,kde_eps", [(0, 0.0), (2, 0.0), (2, 1e-3)])
def test_graph_on_the_gpu_order_matches_the_oracle(fsg, precision, kde_eps):
    n, d, L, seed = 4000, 10, 16, 5
    X = inputs.gaussian_mixture(n=n, d=d, seed=7)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda(), order=fsg.FSG_ORDER_SPATIAL)
    perm = fsg.fsg_tree_perm(tree).cpu().numpy()
    bufs = fsg.fsg_build_graph(tree, fsg.params(1.5, precision=precision, kde_eps=kde_eps), L, seed)
    assert fsg.fsg_sync(tree) == 0
    samples, flags = bufs.samples.cpu().numpy(), bufs.flags.cpu().numpy()
    tree.close()
    q = np.arange(0, n, 3)
    osmp, _, _ = ora.sample(X, ora.gamma(1.5), L, seed, queries=q, perm=perm)
    assert not ((samples[q] != osmp) & (flags[q] == 0)).any()
