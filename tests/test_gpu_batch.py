"""Batched graph construction (fsg_batch_*): several independent point sets of
different sizes, dimensions, L and parameters in one run (several streams,
CUDA-graph replay) give exactly the single-set results, and match the oracle
on sampled queries."""
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


def _sets(fsg):
    imgs = [inputs.segmentation_image(h, w, seed=s) for h, w, s in ((40, 60, 0), (57, 85, 1), (33, 49, 2))]
    out = [(torch.from_numpy(X).cuda(), fsg.params(0.05), 12, 7 + k) for k, X in enumerate(imgs)]
    out.append((torch.from_numpy(inputs.two_moons(n=1500, seed=3)).cuda(), fsg.params(0.1), 32, 1))
    out.append((torch.from_numpy(inputs.gaussian_mixture(n=2500, d=10, k=4, box=4.0, seed=5)).cuda(),
                fsg.params(1.5, self_mode=1), 64, 2))
    # the d > 16 FP32 path, the tensor-core path (8-bit data) and the levelwise schedule in the same batch
    out.append((torch.from_numpy(inputs.gaussian_mixture(n=1700, d=40, k=4, box=3.0, seed=6)).cuda(),
                fsg.params(2.5), 16, 3))
    dig = inputs.digit_like(n=1300, d=784, seed=7)
    out.append((torch.from_numpy(dig).cuda(), fsg.params(inputs.median_pair_distance(dig, m=1024) / 2), 16, 4))
    out.append((torch.from_numpy(inputs.two_moons(n=900, seed=8)).cuda(),
                fsg.params(0.1, schedule=fsg.FSG_SCHED_LEVELWISE), 16, 5))
    return out


def _single(fsg, pts, p, L, seed):
    tree = fsg.fsg_build_tree(pts)
    b = fsg.fsg_build_graph(tree, p, L, seed)
    torch.cuda.synchronize()
    m = int(b.m.item())
    r = (b.src[:m].cpu().numpy(), b.dst[:m].cpu().numpy(), b.w[:m].cpu().numpy(), b.deg.cpu().numpy(),
         b.samples.cpu().numpy(), b.flags.cpu().numpy())
    tree.close()
    return r


@pytest.mark.parametrize("capture", [False, True])
def test_batch_equals_single_sets(fsg, capture):
    sets = _sets(fsg)
    batch = fsg.Batch(sets, streams=3, capture=capture)
    for rep in range(3):  # first run plain, then captured graph replays
        batch.run()
        torch.cuda.synchronize()
        for (pts, p, L, seed), b in zip(sets, batch.bufs):
            src, dst, w, deg, _, _ = _single(fsg, pts, p, L, seed)
            m = int(b.m.item())
            np.testing.assert_array_equal(b.src[:m].cpu().numpy(), src)
            np.testing.assert_array_equal(b.dst[:m].cpu().numpy(), dst)
            np.testing.assert_array_equal(b.w[:m].cpu().numpy(), w)
            np.testing.assert_array_equal(b.deg.cpu().numpy(), deg)
    # new point values of the same shapes are picked up by the replay
    pts0 = sets[0][0]
    pts0.mul_(0.5)
    batch.run()
    torch.cuda.synchronize()
    src, dst, w, deg, _, _ = _single(fsg, *sets[0])
    b = batch.bufs[0]
    np.testing.assert_array_equal(b.deg.cpu().numpy(), deg)
    np.testing.assert_array_equal(b.src[:int(b.m.item())].cpu().numpy(), src)
    batch.close()


def test_batch_matches_oracle_on_sampled_queries(fsg):
    sets = _sets(fsg)
    batch = fsg.Batch(sets, streams=2, capture=True)
    batch.run()
    batch.run()
    torch.cuda.synchronize()
    for (pts, p, L, seed), b in zip(sets, batch.bufs):
        X = pts.cpu().numpy()
        gam = ora.gamma(p.sigma)
        q = np.arange(0, X.shape[0], max(1, X.shape[0] // 40))
        deg = ora.degrees(X, gam, queries=q, self_mode=p.self_mode)
        np.testing.assert_allclose(b.deg.cpu().numpy()[q], deg, rtol=1e-5, atol=X.shape[0] * 2.0 ** -126)
    batch.close()


def test_packed_batch_equals_single_sets(fsg):
    # every set takes the symmetric d = 5 FP32 pass, so the batch computes all
    # bin sums in one launch: the results must equal each set built alone,
    # whatever the sets' sizes, bandwidths, L and self modes
    imgs = [inputs.segmentation_image(h, w, seed=s) for h, w, s in ((40, 60, 0), (64, 96, 1), (33, 49, 2),
                                                                     (80, 120, 3))]
    sets = [(torch.from_numpy(X).cuda(), fsg.params(sig, self_mode=sm), L, 11 + k)
            for k, (X, sig, sm, L) in enumerate(zip(imgs, (0.05, 0.08, 0.05, 0.1), (0, 1, 0, 0), (12, 48, 7, 64)))]
    for capture in (False, True):
        batch = fsg.Batch(sets, streams=3, capture=capture)
        for _ in range(2):
            batch.run()
            torch.cuda.synchronize()
            for (pts, p, L, seed), b in zip(sets, batch.bufs):
                src, dst, w, deg, _, _ = _single(fsg, pts, p, L, seed)
                m = int(b.m.item())
                np.testing.assert_array_equal(b.deg.cpu().numpy(), deg)
                np.testing.assert_array_equal(b.src[:m].cpu().numpy(), src)
                np.testing.assert_array_equal(b.dst[:m].cpu().numpy(), dst)
                np.testing.assert_array_equal(b.w[:m].cpu().numpy(), w)
        batch.close()
    X = imgs[1]
    q = np.arange(0, X.shape[0], 37)
    want = ora.degrees(X, ora.gamma(0.08), queries=q, self_mode=1)
    np.testing.assert_allclose(_single(fsg, *sets[1])[3][q], want, rtol=1e-5, atol=X.shape[0] * 2.0 ** -126)
