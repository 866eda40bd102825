"""The allocation-free degree entry point, fsg_degrees_noalloc.

It exists for callers that must not allocate device memory -- an application
whose pool allocator owns the whole GPU, or a latency-critical caller that
cannot pay for cudaMalloc/cudaFree -- and keeps its scratch in one fixed
array inside the library.  This file checks, through the C ABI, that it gives
the same degrees as the tree-based entry point (fsg_degrees) within the
degree tolerance of the other GPU tests, on two calls in a row (the second
call must not be disturbed by what the first left in the shared scratch), and
that a problem too large for the scratch is refused before any GPU work.

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


@pytest.mark.parametrize("case", ["two_moons", "mixture_d10", "mixture_d3_include"])
def test_noalloc_matches_tree_entry_point_on_two_calls(fsg, case):
    if case == "two_moons":
        X, p = inputs.two_moons(n=3001, seed=4), fsg.params(0.1)
    elif case == "mixture_d10":
        X, p = inputs.gaussian_mixture(n=60_000, d=10, seed=2), fsg.params(1.5)
    else:
        X, p = inputs.gaussian_mixture(n=7_777, d=3, k=4, box=2.0, seed=1), fsg.params(0.5, self_mode=1)
    n = X.shape[0]
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    ref = fsg.fsg_degrees(tree, p).cpu().numpy()
    tree.close()
    for _ in range(2):
        got = _noalloc(fsg, pts, p)
        err = np.abs(got - ref)
        assert (err <= DEG_RTOL * ref + n * TINY).all(), float(np.max(err / np.maximum(ref, 1e-300)))


def test_noalloc_refuses_problems_beyond_its_scratch(fsg):
    lib = fsg.load()
    p = fsg.params(1.0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    rc = lib.fsg_degrees_noalloc(fake, 2_000_000, 16, ctypes.byref(p), fake, None)
    assert rc == fsg.FSG_ERR_SCRATCH
    assert b"scratch" in lib.fsg_error_string(rc)
    assert lib.fsg_degrees_noalloc(fake, 1000, 17, ctypes.byref(p), fake, None) == fsg.FSG_ERR_UNSUPPORTED
