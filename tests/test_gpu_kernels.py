"""The Laplacian and exponential kernels of Sec. 2.1 (fsg_params.kernel) on
the fused schedule's FP32 paths (d <= 16: the symmetric bin pass and the
128-point leaf kernel; d > 16: the generic passes and leaf kernels, also for
8-bit data under the Laplacian, where AUTO means FP32) and, for the
exponential, the exact 8-bit tensor-core path, against the FP64 oracle of the
same family: degrees within the FP32 tolerance, unflagged samples equal to
the oracle's, edge weights within 1e-4; refused where the path does not
offer them."""
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
    (9000, 16, 4.0, 64, 3),      # the largest d of the d <= 16 path, full sample mask
    (5000, 24, 6.0, 32, 4),      # generic symmetric pass, fused generic leaf (bins <= 128)
    (3001, 40, 8.0, 16, 5),      # ragged n at d = 40
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


@pytest.mark.parametrize("name", ["laplacian", "exponential"])
def test_family_on_8bit_data_and_large_bins(fsg, name):
    # digit-like 8-bit data (AUTO takes the FP32 generic passes for the
    # Laplacian, the tensor-core form for the exponential) and a tree with
    # bins of up to 512 points (the two-kernel generic leaf phase: values in
    # HBM, then the leaf finish)
    fam, ofam = family_pair(fsg, name)
    for X, sigma, leaf_max in ((inputs.digit_like(n=2500, d=784, seed=6), 9.0, 0),
                               (inputs.gaussian_mixture(n=6000, d=20, k=5, box=4.0, seed=7), 5.0, 512)):
        c = ora.scale(sigma, ofam)
        tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda(), leaf_max=leaf_max)
        bufs = fsg.fsg_build_graph(tree, fsg.params(sigma, kernel=fam), 16, 8)
        assert fsg.fsg_sync(tree) == 0
        q = np.arange(0, X.shape[0], 11)
        want = ora.degrees(X, c, queries=q, kernel=ofam)
        deg = bufs.deg.cpu().numpy()[q]
        # FP32 bound of the degree at large d: a term with exponent a (log2
        # units) computed from d rounded differences and sums carries
        # ln2 a (d + 3) 2^-24 relative error, plus ex2's 2^-22 and the
        # accumulation's (at most 96 roundings of 2^-24 on the way)
        d = X.shape[1]
        Xd = X.astype(np.float64)
        if ofam == ora.LAPLACIAN:
            dist = np.abs(Xd[q][:, None, :] - Xd[None, :, :]).sum(-1)
        else:
            dist = np.sqrt(((Xd[q][:, None, :] - Xd[None, :, :]) ** 2).sum(-1))
        a = c * np.log2(np.e) * dist
        kv = np.exp2(-a)
        kv[np.arange(q.size), q] = 0.0
        bound = (kv * a).sum(1) * np.log(2) * (d + 3) * 2.0 ** -24 + want * (2.0 ** -22 + 96 * 2.0 ** -24)
        assert (np.abs(deg - want) <= np.maximum(bound, DEG_RTOL * want) + X.shape[0] * TINY).all()
        osmp, _, _ = ora.sample(X, c, 16, 8, queries=q, kernel=ofam)
        assert not ((bufs.samples.cpu().numpy()[q] != osmp) & (bufs.flags.cpu().numpy()[q] == 0)).any()
        tree.close()


@pytest.mark.parametrize("n,d,sigma,L,seed", [
    (3000, 784, 9.0, 32, 1),     # the digit workload's dimension
    (2311, 64, 4.0, 16, 2),      # ragged n, the smallest d of the tensor-core path
])
def test_exponential_on_the_tensor_core_path(fsg, n, d, sigma, L, seed):
    # 8-bit data: AUTO takes the exact tensor-core path for the exponential
    # kernel (the square root of the exact integer squared distance), the
    # same result as FSG_PREC_EXACT_INT, near the FP32 path's and the oracle's
    fam, ofam = family_pair(fsg, "exponential")
    X = inputs.digit_like(n=n, d=d, seed=seed)
    c = ora.scale(sigma, ofam)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    p_auto = fsg.params(sigma, kernel=fam)
    p_int = fsg.params(sigma, kernel=fam, precision=fsg.FSG_PREC_EXACT_INT)
    p_fp32 = fsg.params(sigma, kernel=fam, precision=fsg.FSG_PREC_FP32)
    assert fsg.fsg_bin_pass_evals(tree, p_auto) == fsg.fsg_bin_pass_evals(tree, p_int)
    assert fsg.fsg_bin_pass_evals(tree, p_auto) != fsg.fsg_bin_pass_evals(tree, p_fp32)
    out = {}
    for name, p in (("auto", p_auto), ("int", p_int), ("fp32", p_fp32)):
        b = fsg.fsg_build_graph(tree, p, L, seed)
        assert fsg.fsg_sync(tree) == 0
        m = int(b.m.item())
        out[name] = (b.deg.cpu().numpy(), b.samples.cpu().numpy(), b.flags.cpu().numpy(),
                     b.src[:m].cpu().numpy(), b.dst[:m].cpu().numpy(), b.w[:m].cpu().numpy(), fsg.stats_dict(b))
    tree.close()
    deg, samples, flags, src, dst, w, st = out["auto"]
    assert st["status"] == 0
    np.testing.assert_array_equal(deg, out["int"][0])
    np.testing.assert_array_equal(samples, out["int"][1])
    np.testing.assert_allclose(deg, out["fp32"][0], rtol=2 * DEG_RTOL)
    q = np.arange(0, n, 5)
    want = ora.degrees(X, c, queries=q, kernel=ofam)
    assert (np.abs(deg[q] - want) <= DEG_RTOL * want + n * TINY).all(), float((np.abs(deg[q] - want) / want).max())
    osmp, _, _ = ora.sample(X, c, L, seed, queries=q, kernel=ofam)
    assert not ((samples[q] != osmp) & (flags[q] == 0)).any()
    assert st["n_flagged"] <= 0.01 * n * L
    sel = np.arange(0, src.size, max(1, src.size // 2000))
    odeg = ora.degrees(X, c, kernel=ofam)
    _, ow = ora.weights(X, c, L, odeg, src[sel], dst[sel], kernel=ofam)
    np.testing.assert_allclose(w[sel], ow, rtol=W_RTOL)


def test_family_refused_outside_the_fused_fp32_path(fsg):
    X = inputs.gaussian_mixture(n=6000, d=8, seed=1)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    for kw in (dict(schedule=fsg.FSG_SCHED_LEVELWISE), dict(precision=fsg.FSG_PREC_SPLIT_BF16)):
        with pytest.raises(fsg.FsgError) as e:
            fsg.fsg_degrees(tree, fsg.params(1.5, kernel=fsg.FSG_KERNEL_EXPONENTIAL, **kw))
        assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()
    # the Laplacian's l1 distance has no dot-product form: no tensor-core path
    tree = fsg.fsg_build_tree(torch.from_numpy(inputs.digit_like(n=2000, d=784, seed=2)).cuda())
    with pytest.raises(fsg.FsgError) as e:
        fsg.fsg_degrees(tree, fsg.params(9.0, kernel=fsg.FSG_KERNEL_LAPLACIAN, precision=fsg.FSG_PREC_EXACT_INT))
    assert e.value.status == fsg.FSG_ERR_UNSUPPORTED
    tree.close()
