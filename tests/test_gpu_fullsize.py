"""Parity at the full sizes of the digit-image and segmentation workloads.

Both run through the C ABI in the launch configuration the benchmark times and
are compared with the FP64 oracle on sampled outputs the oracle computes one
by one:

* digit-image-shaped data, n = 70,000, d = 784, L = 64, sigma = median pairwise
  distance / 2, on the exact 8-bit tensor-core path (FSG_PREC_AUTO selects it:
  every coordinate is k/255): degrees at 1e-5 on 256 points, samples of 32
  points equal to the oracle's descent (Algorithm 1) unless flagged, weights
  (Eq. 2) of their edges at 1e-4;
* two segmentation-shaped images at the ends of the batch's size range,
  160 x 240 and 321 x 481 pixels (38,400 and 154,401 points, d = 5,
  sigma = 0.05, L = 48), built together through the batch entry point with
  CUDA-graph replay: degrees at 1e-5 on 256 points per image, samples of
  32 points per image.
"""
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


def check_degrees(got, want, n):
    err = np.abs(got - want)
    assert (err <= DEG_RTOL * want + n * TINY).all(), float(np.max(err / np.maximum(want, 1e-300)))


def check_samples(smp_gpu, flags, smp_ora):
    bad = (smp_gpu != smp_ora) & (flags == 0)
    assert not bad.any(), f"{int(bad.sum())} unflagged mismatches of {smp_gpu.size}"


def test_digits_full_size(fsg):
    n, L, seed = 70_000, 64, 0
    X = inputs.digit_like(n=n, seed=0)
    sigma = inputs.median_pair_distance(X, m=4096, seed=0) / 2
    gam = ora.gamma(sigma)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    bufs = fsg.fsg_build_graph(tree, fsg.params(sigma), L, seed)
    assert fsg.fsg_sync(tree) == 0
    torch.cuda.synchronize()
    st = fsg.stats_dict(bufs)
    assert st["status"] == 0 and st["n_samples"] == n * L
    assert st["n_flagged"] <= 0.01 * n * L
    deg = bufs.deg.cpu().numpy()
    smp = bufs.samples.cpu().numpy()
    flg = bufs.flags.cpu().numpy()
    m = int(bufs.m.item())
    src, dst, w = (bufs.src[:m].cpu().numpy(), bufs.dst[:m].cpu().numpy(), bufs.w[:m].cpu().numpy())
    tree.close()
    rng = np.random.Generator(np.random.PCG64(21))
    q = rng.choice(n, size=256, replace=False)
    check_degrees(deg[q], ora.degrees(X, gam, queries=q), n)
    qs = q[:32]
    osmp, _, _ = ora.sample(X, gam, L, seed, queries=qs)
    check_samples(smp[qs], flg[qs], osmp)
    # weights of the oracle's sampled pairs of these points, found in the GPU's SET edge list
    s_o = np.repeat(qs, L)
    d_o = osmp.reshape(-1)
    keep = d_o >= 0
    s_o, d_o = s_o[keep], d_o[keep]
    ends = np.unique(np.concatenate([s_o, d_o]))
    dg = np.zeros(n)
    dg[ends] = ora.degrees(X, gam, queries=ends)
    _, w_ora = ora.weights(X, gam, L, dg, s_o, d_o)
    gw = {(min(a, b), max(a, b)): x for a, b, x in zip(src.tolist(), dst.tolist(), w.tolist())}
    found = 0
    for a, b, x in zip(s_o.tolist(), d_o.tolist(), w_ora.tolist()):
        key = (min(a, b), max(a, b))
        if key in gw:
            found += 1
            assert math.isclose(gw[key], x, rel_tol=W_RTOL), (key, gw[key], x)
    assert found >= 0.99 * len(s_o)


def test_segmentation_full_size_batch(fsg):
    L, sigma = 48, 0.05
    gam = ora.gamma(sigma)
    imgs = [inputs.segmentation_image(160, 240, seed=0), inputs.segmentation_image(321, 481, seed=63)]
    sets = [(torch.from_numpy(X).cuda(), fsg.params(sigma), L, 1000 + k) for k, X in enumerate(imgs)]
    batch = fsg.Batch(sets, streams=2, capture=True)
    batch.run()
    batch.run()  # the captured graph's replay
    torch.cuda.synchronize()
    for k, (X, b) in enumerate(zip(imgs, batch.bufs)):
        n = X.shape[0]
        st = fsg.stats_dict(b)
        assert st["status"] == 0 and st["n_samples"] == n * L
        rng = np.random.Generator(np.random.PCG64(30 + k))
        q = rng.choice(n, size=256, replace=False)
        check_degrees(b.deg.cpu().numpy()[q], ora.degrees(X, gam, queries=q), n)
    batch.close()
    # samples: the same sets built one at a time expose the per-sample outputs
    for k, X in enumerate(imgs):
        n = X.shape[0]
        tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
        bufs = fsg.fsg_build_graph(tree, fsg.params(sigma), L, 1000 + k)
        assert fsg.fsg_sync(tree) == 0
        rng = np.random.Generator(np.random.PCG64(40 + k))
        qs = rng.choice(n, size=32, replace=False)
        osmp, _, _ = ora.sample(X, gam, L, 1000 + k, queries=qs)
        check_samples(bufs.samples.cpu().numpy()[qs], bufs.flags.cpu().numpy()[qs], osmp)
        assert fsg.stats_dict(bufs)["n_flagged"] <= 0.01 * n * L
        tree.close()
