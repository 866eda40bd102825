"""Autotuner (fsg_autotune): the launch shapes it picks are valid, applied to
the tree and cached per shape; results with the tuned shapes still match the
oracle, and unflagged samples equal those of the heuristic shapes."""
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


def _graph(fsg, tree, p, L, seed):
    bufs = fsg.fsg_build_graph(tree, p, L, seed)
    assert fsg.fsg_sync(tree) == 0
    return bufs.samples.cpu().numpy(), bufs.flags.cpu().numpy(), bufs.deg.cpu().numpy()


@pytest.mark.parametrize("n,d,maker", [(6000, 10, "gmm"), (3000, 784, "digits"), (4000, 40, "gmm")])
def test_autotune_valid_and_consistent(fsg, n, d, maker):
    X = inputs.gaussian_mixture(n=n, d=d, seed=3) if maker == "gmm" else inputs.digit_like(n=n, d=d, seed=3)
    sigma = 1.5 if maker == "gmm" else inputs.median_pair_distance(X, m=1024) / 2
    p = fsg.params(sigma)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    s0, f0, d0 = _graph(fsg, tree, p, 16, 5)
    tun = fsg.fsg_autotune(tree, p, 16, 5, reps=2)
    assert fsg.fsg_tree_tuning(tree) == tun
    assert tun["leaf_splits"] >= 1
    if d <= 16:
        assert 4 <= tun["sym_bins"] <= 16
    if maker == "digits":
        assert 8 <= tun["tc_bins"] <= 24
    s1, f1, d1 = _graph(fsg, tree, p, 16, 5)
    np.testing.assert_allclose(d1, d0, rtol=2e-5)
    both = (f0 == 0) & (f1 == 0)
    np.testing.assert_array_equal(s1[both], s0[both])
    q = np.arange(0, n, max(1, n // 100))
    smp, _, _ = ora.sample(X, ora.gamma(sigma), 16, 5, queries=q)
    assert not ((s1[q] != smp) & (f1[q] == 0)).any()
    # the same shape is served from the cache, and a second tree takes it too
    tree2 = fsg.fsg_build_tree(pts)
    assert fsg.fsg_autotune(tree2, p, 16, 5, reps=2) == tun
    tree2.close()
    tree.close()


def test_tuning_set_and_refuse(fsg):
    X = inputs.gaussian_mixture(n=2000, d=5, seed=1)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    assert fsg.fsg_tree_tuning(tree, {"sym_bins": 6, "leaf_splits": 3}) == {"sym_bins": 6, "tc_bins": 0,
                                                                          "leaf_splits": 3}
    with pytest.raises(fsg.FsgError):
        fsg.fsg_tree_tuning(tree, {"sym_bins": -1})
    s, f, _ = _graph(fsg, tree, fsg.params(1.0), 8, 2)
    q = np.arange(0, 2000, 37)
    smp, _, _ = ora.sample(X, ora.gamma(1.0), 8, 2, queries=q)
    assert not ((s[q] != smp) & (f[q] == 0)).any()
    tree.close()
