"""Tensor-core (tcgen05) bin pass for d >= 64 on 8-bit data: degrees and
samples against the FP64 oracle and against the FP32 path of the same
library (which must agree to FP32 accuracy), on sizes that span several
128-query blocks, several 256-point tiles and ragged tails."""
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


def _deg(fsg, X, sigma, precision):
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    d = fsg.fsg_degrees(tree, fsg.params(sigma, precision=precision)).cpu().numpy()
    assert fsg.fsg_sync(tree) == 0
    tree.close()
    return d


@pytest.mark.parametrize("n,d", [(300, 64), (1000, 64), (777, 784), (2600, 784)])
def test_tc_degrees_match_oracle_and_fp32(fsg, n, d):
    X = inputs.digit_like(n=n, d=d, seed=n + d)
    sigma = inputs.median_pair_distance(X, m=min(n, 1024)) / 2
    gam = ora.gamma(sigma)
    tc = _deg(fsg, X, sigma, fsg.FSG_PREC_EXACT_INT)
    fp = _deg(fsg, X, sigma, fsg.FSG_PREC_FP32)
    q = np.arange(0, n, max(1, n // 200))
    want = ora.degrees(X, gam, queries=q)
    np.testing.assert_allclose(tc[q], want, rtol=1e-5, atol=n * 2.0 ** -126)
    np.testing.assert_allclose(tc, fp, rtol=2e-5)


def test_tc_samples_match_oracle(fsg):
    X = inputs.digit_like(n=3000, d=784, seed=9)
    sigma = inputs.median_pair_distance(X, m=1024) / 2
    gam = ora.gamma(sigma)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    bufs = fsg.fsg_build_graph(tree, fsg.params(sigma, precision=fsg.FSG_PREC_EXACT_INT), 16, 3)
    assert fsg.fsg_sync(tree) == 0
    smp = bufs.samples.cpu().numpy()
    flg = bufs.flags.cpu().numpy()
    q = np.arange(0, 3000, 17)
    osmp, _, _ = ora.sample(X, gam, 16, 3, queries=q)
    bad = (osmp != smp[q]) & (flg[q] == 0)
    assert not bad.any()
    tree.close()


def test_non_8bit_data_refuse_exact_int(fsg):
    X = inputs.gaussian_mixture(n=500, d=64, seed=2)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    with pytest.raises(fsg.FsgError) as e:
        fsg.fsg_degrees(tree, fsg.params(1.5, precision=fsg.FSG_PREC_EXACT_INT))
    assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()
