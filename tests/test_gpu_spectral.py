"""The downstream consumer (spectral clustering, Rand index; Sec. 5) on graphs
the library builds on the GPU: two moons, a segmentation image against the
complete kernel graph's clustering, a Gaussian mixture, and the mixture at
d = 64 in split precision."""
import numpy as np
import pytest

import oracle as ora
from paper_2310_13870_gb300 import inputs, spectral

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")
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


def test_two_moons(fsg):
    n = 2000
    X = inputs.two_moons(n=n, seed=4)
    src, dst, w = fsg.fsg_build_graph_host(X, fsg.params(0.1), 16, 5)
    lab = spectral.spectral_clustering(n, src, dst, w, 2)
    assert spectral.rand_index(lab, inputs.two_moons_labels(n)) >= 0.99


def test_segmentation_image(fsg):
    X, reg = inputs.segmentation_image(48, 72, seed=7, return_labels=True)
    k = len(np.unique(reg))
    src, dst, w = fsg.fsg_build_graph_host(X, fsg.params(0.05), 16, 1)
    ri_sparse = spectral.rand_index(spectral.spectral_clustering(len(X), src, dst, w, k), reg)
    gam = ora.gamma(0.05)
    K = np.exp(-gam * ((X[:, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(K, 0.0)
    i, j = np.nonzero(np.triu(K, 1))
    ri_dense = spectral.rand_index(spectral.spectral_clustering(len(X), i, j, K[i, j], k), reg)
    assert ri_sparse >= 0.85 and ri_sparse >= ri_dense - 0.05, (ri_sparse, ri_dense)


@pytest.mark.parametrize("d,split", [(10, False), (64, True)])
def test_gaussian_mixture(fsg, d, split):
    X, truth = inputs.gaussian_mixture(n=5000, d=d, k=8, seed=3, return_labels=True)
    p = fsg.params(1.5, precision=fsg.FSG_PREC_SPLIT_BF16 if split else fsg.FSG_PREC_AUTO)
    src, dst, w = fsg.fsg_build_graph_host(X, p, 16, 2)
    lab = spectral.spectral_clustering(len(X), src, dst, w, 8)
    assert spectral.rand_index(lab, truth) >= 0.99
