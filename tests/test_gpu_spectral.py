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
    # The Rand index of one sampled graph's clustering varies with the seed
    # (the exact method's own graphs of this image span 0.87..0.93 over seeds
    # 1..8 at L = 16), so the check takes the median over five seeds and
    # compares it with the oracle's graphs on the same seeds, and with the
    # complete kernel graph's clustering.
    X, reg = inputs.segmentation_image(48, 72, seed=7, return_labels=True)
    k = len(np.unique(reg))
    gam = ora.gamma(0.05)
    ri_gpu, ri_ora = [], []
    for seed in range(1, 6):
        src, dst, w = fsg.fsg_build_graph_host(X, fsg.params(0.05), 16, seed)
        ri_gpu.append(spectral.rand_index(spectral.spectral_clustering(len(X), src, dst, w, k), reg))
        o = ora.build_graph(X, gam, 16, seed)
        ri_ora.append(spectral.rand_index(spectral.spectral_clustering(len(X), o["src"], o["dst"], o["w"], k), reg))
    K = np.exp(-gam * ((X[:, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(K, 0.0)
    i, j = np.nonzero(np.triu(K, 1))
    ri_dense = spectral.rand_index(spectral.spectral_clustering(len(X), i, j, K[i, j], k), reg)
    med_gpu, med_ora = float(np.median(ri_gpu)), float(np.median(ri_ora))
    assert med_gpu >= 0.85 and abs(med_gpu - med_ora) <= 0.03, (ri_gpu, ri_ora)
    assert med_gpu >= ri_dense - 0.06, (med_gpu, ri_dense)


# At d = 64 the bandwidth is 3: with sigma = 1.5 the kernel values inside a
# blob span about nine orders of magnitude, some vertices hang on by edges
# many orders lighter than the rest, and the normalised spectral embedding is
# ill-conditioned for any graph of this data (the oracle's own graph, whose
# components are exactly the 8 blobs, scores a Rand index of 0.96, and 1e-4
# relative noise on its weights moves it between 0.96 and 0.997).  At sigma =
# 3 the weights span two orders and the oracle's graph scores 1.0 under 1e-3
# noise, so the check measures the graph, not the eigensolver.
@pytest.mark.parametrize("d,split,sigma", [(10, False, 1.5), (64, True, 3.0)])
def test_gaussian_mixture(fsg, d, split, sigma):
    X, truth = inputs.gaussian_mixture(n=5000, d=d, k=8, seed=3, return_labels=True)
    p = fsg.params(sigma, precision=fsg.FSG_PREC_SPLIT_BF16 if split else fsg.FSG_PREC_AUTO)
    src, dst, w = fsg.fsg_build_graph_host(X, p, 16, 2)
    lab = spectral.spectral_clustering(len(X), src, dst, w, 8)
    assert spectral.rand_index(lab, truth) >= 0.99
