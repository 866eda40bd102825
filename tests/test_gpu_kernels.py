"""The Laplacian and exponential kernels of Sec. 2.1 (fsg_params.kernel) on
the fused FP32 path for d <= 16, against the FP64 oracle of the same family:
degrees within the FP32 tolerance, unflagged samples equal to the oracle's,
edge weights within 1e-4; refused where the path does not offer them."""
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


def family_pair(fsg, name):
    return {"laplacian": (fsg.FSG_KERNEL_LAPLACIAN, ora.LAPLACIAN),
            "exponential": (fsg.FSG_KERNEL_EXPONENTIAL, ora.EXPONENTIAL)}[name]


@pytest.mark.parametrize("name", ["laplacian", "exponential"])
@pytest.mark.parametrize("n,d,sigma,L,seed", [
    (6000, 10, 3.0, 32, 1),      # the mixture workload's dimension
    (5003, 2, 0.2, 16, 2),       # ragged n, two dimensions
    (9000, 16, 4.0, 64, 3),      # the largest d of the path, full sample mask
])
def test_family_matches_oracle(fsg, name, n, d, sigma, L, seed):
    fam, ofam = family_pair(fsg, name)
    X = inputs.gaussian_mixture(n=n, d=d, k=8, box=6.0, seed=seed)
    c = ora.scale(sigma, ofam)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    bufs = fsg.fsg_build_graph(tree, fsg.params(sigma, kernel=fam), L, seed)
    assert fsg.fsg_sync(tree) == 0
    m = int(bufs.m.item())
    deg, samples, flags = bufs.deg.cpu().numpy(), bufs.samples.cpu().numpy(), bufs.flags.cpu().numpy()
    src, dst, w = bufs.src[:m].cpu().numpy(), bufs.dst[:m].cpu().numpy(), bufs.w[:m].cpu().numpy()
    st = fsg.stats_dict(bufs)
    tree.close()
    assert st["status"] == 0
    q = np.arange(0, n, 7)
    want = ora.degrees(X, c, queries=q, kernel=ofam)
    assert (np.abs(deg[q] - want) <= DEG_RTOL * want + n * TINY).all(), float((np.abs(deg[q] - want) / want).max())
    osmp, _, _ = ora.sample(X, c, L, seed, queries=q, kernel=ofam)
    assert not ((samples[q] != osmp) & (flags[q] == 0)).any()
    assert st["n_flagged"] <= 0.01 * n * L
    # weights of the GPU's own edges against Eq. 2 with the oracle's k and degrees
    sel = np.arange(0, m, max(1, m // 2000))
    odeg = ora.degrees(X, c, kernel=ofam)
    _, ow = ora.weights(X, c, L, odeg, src[sel], dst[sel], kernel=ofam)
    np.testing.assert_allclose(w[sel], ow, rtol=W_RTOL)


@pytest.mark.parametrize("name", ["laplacian", "exponential"])
def test_family_include_self(fsg, name):
    fam, ofam = family_pair(fsg, name)
    X = inputs.gaussian_mixture(n=4000, d=5, seed=4)
    c = ora.scale(2.0, ofam)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    bufs = fsg.fsg_build_graph(tree, fsg.params(2.0, kernel=fam, self_mode=fsg.FSG_SELF_INCLUDE), 16, 9)
    assert fsg.fsg_sync(tree) == 0
    deg = bufs.deg.cpu().numpy()
    tree.close()
    want = ora.degrees(X, c, self_mode=ora.SELF_INCLUDE, kernel=ofam)
    np.testing.assert_allclose(deg, want, rtol=DEG_RTOL)


def test_families_differ_from_the_gaussian(fsg):
    # the same input under the three kernels gives three different degree vectors
    X = torch.from_numpy(inputs.gaussian_mixture(n=3000, d=4, seed=5)).cuda()
    tree = fsg.fsg_build_tree(X)
    out = []
    for fam in (fsg.FSG_KERNEL_GAUSSIAN, fsg.FSG_KERNEL_LAPLACIAN, fsg.FSG_KERNEL_EXPONENTIAL):
        out.append(fsg.fsg_degrees(tree, fsg.params(1.5, kernel=fam)).cpu().numpy())
    tree.close()
    assert not np.allclose(out[0], out[1]) and not np.allclose(out[1], out[2]) and not np.allclose(out[0], out[2])


def test_family_refused_outside_the_fused_fp32_path(fsg):
    X = inputs.gaussian_mixture(n=6000, d=20, seed=1)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    with pytest.raises(fsg.FsgError) as e:  # d > 16
        fsg.fsg_degrees(tree, fsg.params(1.5, kernel=fsg.FSG_KERNEL_LAPLACIAN))
    assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()
    X = inputs.gaussian_mixture(n=6000, d=8, seed=1)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    for kw in (dict(schedule=fsg.FSG_SCHED_LEVELWISE), dict(precision=fsg.FSG_PREC_SPLIT_BF16)):
        with pytest.raises(fsg.FsgError) as e:
            fsg.fsg_degrees(tree, fsg.params(1.5, kernel=fsg.FSG_KERNEL_EXPONENTIAL, **kw))
        assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()
