"""Failure detection on the GPU without a GPU fault: a device wait made to run
out (an mbarrier that nothing completes, a 0.2 s limit) reports
FSG_ERR_TIMEOUT through the status word, no kernel traps, and the context
keeps working for the next call."""
import time

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


def test_bounded_wait_reports_timeout_and_the_context_survives(fsg):
    t0 = time.time()
    assert fsg.load().fsg_selftest_wait_timeout(200_000_000, None) == fsg.FSG_ERR_TIMEOUT
    assert time.time() - t0 < 30
    X = inputs.gaussian_mixture(n=2000, d=4, seed=0)
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    deg = fsg.fsg_degrees(tree, fsg.params(1.5)).cpu().numpy()
    assert fsg.fsg_sync(tree) == 0
    tree.close()
    np.testing.assert_allclose(deg, ora.degrees(X, ora.gamma(1.5)), rtol=1e-5)
