"""The allocation-free degree entry point, fsg_degrees_noalloc.

It exists for callers that must not allocate device memory -- an application
whose pool allocator owns the whole GPU, or a latency-critical caller that
cannot pay for cudaMalloc/cudaFree -- and keeps its scratch in one fixed
array inside the library.  This file checks, through the C ABI:

* that it gives the degrees of the tree-based entry point (fsg_degrees) within
  the degree tolerance of the other GPU tests, and the FP64 oracle's degrees
  of Algorithm 2 on sampled points, on two calls in a row;
* that the second call is not disturbed by what an earlier call left in the
  shared scratch: between the two compared calls another call runs on a
  different problem (more points, another dimension, the other self mode), so
  stale position maps, partial sums or status words would show;
* that a problem too large for the scratch is refused before any GPU work.

The file is named to be collected last, and it builds the library itself, so
it passes alone in a fresh process as well as after the other tests.
"""
import ctypes
import os

import numpy as np
import pytest

from paper_2310_13870_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEG_RTOL = 1e-5
TINY = 2.0 ** -126


@pytest.fixture(scope="module")
def fsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_13870_gb300 import fsg as _fsg
    if not os.path.exists(_fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    _fsg.load()
    return _fsg


def _noalloc(fsg, pts, p):
    lib = fsg.load()
    out = torch.full((pts.shape[0],), -1.0, dtype=torch.float64, device="cuda")
    rc = lib.fsg_degrees_noalloc(ctypes.c_void_p(pts.data_ptr()), pts.shape[0], pts.shape[1], ctypes.byref(p),
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == fsg.FSG_OK, fsg.load().fsg_error_string(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _tree_degrees(fsg, pts, p):
    tree = fsg.fsg_build_tree(pts)
    ref = fsg.fsg_degrees(tree, p).cpu().numpy()
    fsg.fsg_sync(tree)
    tree.close()
    return ref


def _close(got, want, n):
    err = np.abs(got - want)
    ok = np.isfinite(got).all() and (err <= DEG_RTOL * want + n * TINY).all()
    return ok, float(np.max(err / np.maximum(want, 1e-300)))


CASES = {
    "two_moons": lambda fsg: (inputs.two_moons(n=3001, seed=4), fsg.params(0.1), 0.1, 0),
    "mixture_d10": lambda fsg: (inputs.gaussian_mixture(n=60_000, d=10, seed=2), fsg.params(1.5), 1.5, 0),
    "mixture_d3_include": lambda fsg: (inputs.gaussian_mixture(n=7_777, d=3, k=4, box=2.0, seed=1),
                                       fsg.params(0.5, self_mode=1), 0.5, 1),
}
# the call placed between the two compared ones: more points, another d, the other self mode
OTHER = {
    "two_moons": lambda fsg: (inputs.gaussian_mixture(n=90_001, d=7, seed=9), fsg.params(1.2, self_mode=1)),
    "mixture_d10": lambda fsg: (inputs.gaussian_mixture(n=80_000, d=16, seed=3), fsg.params(2.0, self_mode=1)),
    "mixture_d3_include": lambda fsg: (inputs.two_moons(n=100_000, seed=5), fsg.params(0.1)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_tree_entry_point_and_oracle_on_two_calls(fsg, case):
    import oracle as ora
    X, p, sigma, self_mode = CASES[case](fsg)
    n = X.shape[0]
    pts = torch.from_numpy(X).cuda()
    ref = _tree_degrees(fsg, pts, p)
    q = np.random.Generator(np.random.PCG64(11)).choice(n, size=min(n, 256), replace=False)
    want = ora.degrees(X, ora.gamma(sigma), queries=q, self_mode=self_mode)
    ok, worst = _close(ref[q], want, n)
    assert ok, f"tree entry point vs oracle: {worst}"

    Xo, po = OTHER[case](fsg)
    for call in range(2):
        got = _noalloc(fsg, pts, p)
        ok, worst = _close(got, ref, n)
        assert ok, f"call {call}: vs fsg_degrees {worst}"
        ok, worst = _close(got[q], want, n)
        assert ok, f"call {call}: vs the oracle {worst}"
        if call == 0:
            # a different problem in between, itself checked against the tree entry point
            other = torch.from_numpy(Xo).cuda()
            got_o = _noalloc(fsg, other, po)
            ok, worst = _close(got_o, _tree_degrees(fsg, other, po), Xo.shape[0])
            assert ok, f"intervening call: {worst}"


def test_noalloc_refuses_problems_beyond_its_scratch(fsg):
    lib = fsg.load()
    p = fsg.params(1.0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    rc = lib.fsg_degrees_noalloc(fake, 2_000_000, 16, ctypes.byref(p), fake, None)
    assert rc == fsg.FSG_ERR_SCRATCH
    assert b"scratch" in lib.fsg_error_string(rc)
    assert lib.fsg_degrees_noalloc(fake, 1000, 17, ctypes.byref(p), fake, None) == fsg.FSG_ERR_UNSUPPORTED
