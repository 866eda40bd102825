"""Stepped graph build (fsg_graph_begin / fsg_graph_step / fsg_graph_end):
Algorithm 2 over ranges of query positions, checkpointed and resumed.  Every
per-query computation after the bin pass reads only the bin sums and the
query's own draws, so for any split of the positions into steps, taken in
any order, repeated or resumed after a refused step, the outputs equal
fsg_build_graph's bit for bit; the whole build itself is checked against the
oracle elsewhere, and here its unflagged samples once more on a subset."""
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


def arrays(fsg, b):
    m = int(b.m.item())
    return dict(deg=b.deg.cpu().numpy(), samples=b.samples.cpu().numpy(), flags=b.flags.cpu().numpy(),
                src=b.src[:m].cpu().numpy(), dst=b.dst[:m].cpu().numpy(), w=b.w[:m].cpu().numpy(),
                stats=fsg.stats_dict(b))


def whole(fsg, tree, p, L, seed, edge_mode):
    b = fsg.fsg_build_graph(tree, p, L, seed, edge_mode=edge_mode)
    assert fsg.fsg_sync(tree) == 0
    return arrays(fsg, b)


def stepped(fsg, tree, p, L, seed, edge_mode, ranges):
    fsg.fsg_graph_begin(tree, p, L, seed)
    for a, b in ranges:
        fsg.fsg_graph_step(tree, a, b)
    assert fsg.fsg_graph_cursor(tree) == tree.n
    out = fsg.fsg_graph_end(tree, L, edge_mode=edge_mode, weight_f64=bool(p.weight_f64))
    assert fsg.fsg_sync(tree) == 0
    return arrays(fsg, out)


def assert_same(a, b, counts=True):
    for k in ("deg", "samples", "flags", "src", "dst", "w"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    keys = ("n_samples", "n_flagged", "n_self", "n_empty", "n_edges", "n_bin_evals", "n_resolved", "status")
    if counts:
        keys += ("n_items", "n_evals")
    for k in keys:
        assert a["stats"][k] == b["stats"][k], k


CASES = {
    "d10": (lambda: inputs.gaussian_mixture(n=20000, d=10, seed=1), dict(sigma=1.5), 32),
    "d10_resolve_f64": (lambda: inputs.gaussian_mixture(n=12000, d=10, seed=2),
                        dict(sigma=1.5, resolve=True, weight_f64=True), 64),
    "d24": (lambda: inputs.gaussian_mixture(n=9001, d=24, k=6, box=4.0, seed=3), dict(sigma=2.5), 16),
    "digits": (lambda: inputs.digit_like(n=3000, seed=4), dict(sigma=4.5), 16),
    "split_d64": (lambda: inputs.gaussian_mixture(n=6000, d=64, k=6, box=4.0, seed=5),
                  dict(sigma=3.0, precision=2), 16),
    "laplacian": (lambda: inputs.gaussian_mixture(n=5000, d=6, seed=6), dict(sigma=1.0, kernel=1), 24),
}


@pytest.mark.parametrize("name", list(CASES))
def test_steps_equal_the_whole_build(fsg, name):
    make, kw, L = CASES[name]
    X = make()
    n = X.shape[0]
    sigma = kw.pop("sigma") if "sigma" in kw else 1.5
    p = fsg.params(sigma, **kw)
    kw["sigma"] = sigma
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    edge_mode = fsg.FSG_EDGES_MULTI if name == "d24" else fsg.FSG_EDGES_SET
    ref = whole(fsg, tree, p, L, 11, edge_mode)
    a, b = n // 3, 2 * n // 3
    # out of order, one single-query step, uneven sizes
    got = stepped(fsg, tree, p, L, 11, edge_mode, [(b, n), (0, a), (a, a + 1), (a + 1, b)])
    tree.close()
    assert_same(ref, got)
    if name == "d10":
        q = np.arange(0, n, 97)
        smp, _, _ = ora.sample(X, ora.gamma(sigma), L, 11, queries=q)
        assert not ((got["samples"][q] != smp) & (got["flags"][q] == 0)).any()


def test_resume_after_refused_and_repeated_steps(fsg):
    X = inputs.gaussian_mixture(n=15000, d=10, seed=7)
    n, L = X.shape[0], 48
    p = fsg.params(1.5)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    ref = whole(fsg, tree, p, L, 5, fsg.FSG_EDGES_SET)
    fsg.fsg_graph_begin(tree, p, L, 5)
    assert fsg.fsg_graph_cursor(tree) == 0
    fsg.fsg_graph_step(tree, 0, 4000)
    fsg.fsg_graph_step(tree, 4000, 9000)
    assert fsg.fsg_graph_cursor(tree) == 9000
    for bad in ((9000, n + 1), (-1, 10), (50, 50)):  # refused on the host: nothing enqueued
        with pytest.raises(fsg.FsgError) as e:
            fsg.fsg_graph_step(tree, *bad)
        assert e.value.status == fsg.FSG_ERR_INVALID_ARG
    with pytest.raises(fsg.FsgError) as e:  # not every position stepped yet
        fsg.fsg_graph_end(tree, L)
    assert e.value.status == fsg.FSG_ERR_INVALID_ARG
    assert fsg.fsg_graph_cursor(tree) == 9000
    fsg.fsg_graph_step(tree, 4000, 9000)   # a step repeated, as after a failed sync
    fsg.fsg_graph_step(tree, 12000, n)     # a gap: the cursor stays at its start
    assert fsg.fsg_graph_cursor(tree) == 9000
    fsg.fsg_graph_step(tree, 9000, 12000)  # resumed from the cursor
    assert fsg.fsg_graph_cursor(tree) == n
    got = arrays(fsg, fsg.fsg_graph_end(tree, L))
    assert fsg.fsg_sync(tree) == 0
    assert_same(ref, got, counts=False)  # the repeated step's work is counted twice
    assert got["stats"]["n_items"] > ref["stats"]["n_items"]


def test_other_calls_end_the_run(fsg):
    X = inputs.gaussian_mixture(n=5000, d=10, seed=8)
    p = fsg.params(1.5)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    fsg.fsg_graph_begin(tree, p, 16, 1)
    fsg.fsg_graph_step(tree, 0, 2500)
    fsg.fsg_degrees(tree, p)  # reuses the workspace that holds the run
    for call in (lambda: fsg.fsg_graph_step(tree, 2500, 5000), lambda: fsg.fsg_graph_cursor(tree)):
        with pytest.raises(fsg.FsgError) as e:
            call()
        assert e.value.status == fsg.FSG_ERR_INVALID_ARG
    with pytest.raises(fsg.FsgError) as e:  # the levelwise schedules have no bin pass to keep
        fsg.fsg_graph_begin(tree, fsg.params(1.5, schedule=fsg.FSG_SCHED_LEVELWISE), 16, 1)
    assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    assert fsg.fsg_sync(tree) == 0
    tree.close()
