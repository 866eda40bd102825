"""fsg_spatial_order (host, no GPU): the tree order under which every node is
a compact group.  It must be a permutation, deterministic, split each node
where the tree of Sec. 4.1 splits it (left = floor(|X|/2) positions) along the
coordinate of largest spread, keep well-separated clusters whole, and refuse
bad input."""
import ctypes
import os

import numpy as np
import pytest

from paper_2310_13870_gb300 import fsg, inputs


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return fsg.load()


def test_permutation_and_determinism(lib):
    X = inputs.gaussian_mixture(n=5003, d=12, seed=3)
    p1 = fsg.fsg_spatial_order(X)
    p2 = fsg.fsg_spatial_order(X.copy())
    assert p1.dtype == np.int32 and p1.shape == (5003,)
    np.testing.assert_array_equal(np.sort(p1), np.arange(5003))
    np.testing.assert_array_equal(p1, p2)


def _check_node(X, perm, lo, hi, leaf):
    """The node's split is at lo + floor((hi-lo)/2) along its widest coordinate."""
    if hi - lo <= leaf:
        np.testing.assert_array_equal(perm[lo:hi], np.sort(perm[lo:hi]))  # leaves keep index order
        return
    P = X[perm[lo:hi]]
    axis = int(np.argmax(P.max(0) - P.min(0)))
    mid = lo + (hi - lo) // 2
    left, right = X[perm[lo:mid], axis], X[perm[mid:hi], axis]
    assert left.max() <= right.min()
    _check_node(X, perm, lo, mid, leaf)
    _check_node(X, perm, mid, hi, leaf)


@pytest.mark.parametrize("n,d,leaf", [(1000, 3, 32), (777, 20, 8), (64, 2, 1), (1, 5, 32), (2, 1, 1)])
def test_nodes_split_where_the_tree_splits(lib, n, d, leaf):
    rng = np.random.default_rng(n + d)
    X = rng.random((n, d), dtype=np.float32) * np.arange(1, d + 1, dtype=np.float32)  # distinct spreads
    perm = fsg.fsg_spatial_order(X, leaf=leaf)
    _check_node(X, perm, 0, n, leaf)


def test_separated_clusters_become_subtrees(lib):
    # 8 clusters of 512 points at the corners of a cube, 100 apart, radius < 1:
    # each depth-3 node (512 positions) holds exactly one cluster
    rng = np.random.default_rng(0)
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float32) * 100.0
    label = np.repeat(np.arange(8), 512)
    X = (corners[label] + rng.uniform(-0.5, 0.5, (4096, 3))).astype(np.float32)
    order = rng.permutation(4096)
    X, label = X[order], label[order]
    perm = fsg.fsg_spatial_order(X)
    for node in range(8):
        assert len(set(label[perm[512 * node:512 * (node + 1)]].tolist())) == 1


def test_blocks_are_compact(lib):
    X = inputs.gaussian_mixture(n=8192, d=32, seed=5)
    perm = fsg.fsg_spatial_order(X)

    def spread(p):
        Y = X[p].reshape(-1, 128, 32)
        return float(((Y - Y.mean(1, keepdims=True)) ** 2).sum(-1).mean())

    assert spread(perm) < 0.2 * spread(np.arange(8192))


def test_bad_input_is_refused(lib):
    X = np.zeros((4, 2), np.float32)
    out = np.empty(4, np.int32)
    assert lib.fsg_spatial_order(None, 4, 2, 32, out.ctypes.data) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_spatial_order(X.ctypes.data, 4, 2, 32, None) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_spatial_order(X.ctypes.data, 0, 2, 32, out.ctypes.data) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_spatial_order(X.ctypes.data, 4, 0, 32, out.ctypes.data) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_spatial_order(X.ctypes.data, 4, 2, 0, out.ctypes.data) == fsg.FSG_ERR_INVALID_ARG
    X[1, 1] = np.nan
    assert lib.fsg_spatial_order(X.ctypes.data, 4, 2, 32, out.ctypes.data) == fsg.FSG_ERR_INVALID_ARG
    X[1, 1] = np.inf
    assert lib.fsg_spatial_order(X.ctypes.data, 4, 2, 32, out.ctypes.data) == fsg.FSG_ERR_INVALID_ARG
