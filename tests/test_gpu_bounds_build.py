"""The bounds-checking build (FSG_BOUNDS_CHECK): every kernel's index checks
compiled in, a failure recorded in device error words and reported by
fsg_sync (FSG_ERR_BOUNDS) and fsg_bounds_error instead of an out-of-bounds
access.  The test builds that library beside the normal one and runs graph
builds through it on every path it instruments (the symmetric FP32 and
plain bin passes, descend_top and the item scatter, the 128-point and
generic leaf kernels, the symmetric tensor-core pass, the high-precision
re-decision, the split form at d > 64 and a stepped build over uneven
ranges), each against the FP64 oracle or the whole build, with no check
failing."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, torch
import oracle as ora
from paper_2310_13870_gb300 import fsg, inputs
lib = fsg.load()
assert "_build_bounds" in fsg.LIB_PATH
cases = [
    (inputs.two_moons(n=2000, seed=0), 0.1, 32, {}),                       # symmetric FP32, leaf128
    (inputs.gaussian_mixture(n=9000, d=10, seed=1), 1.5, 64, {"resolve": True}),  # + re-decision
    (inputs.two_moons(n=777, seed=3), 0.1, 7, {}),                          # plain pass, generic leaf
    (inputs.digit_like(n=1500, seed=4), None, 16, {}),                      # symmetric tensor-core pass
]
for X, sigma, L, extra in cases:
    if sigma is None:
        sigma = inputs.median_pair_distance(X, m=1024) / 2
    tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
    b = fsg.fsg_build_graph(tree, fsg.params(sigma, **extra), L, 5)
    assert fsg.fsg_sync(tree) == 0
    out = (__import__("ctypes").c_int64 * 4)()
    assert lib.fsg_bounds_error(out) == 0 and list(out) == [0, 0, 0, 0], list(out)
    q = np.arange(0, X.shape[0], max(1, X.shape[0] // 64))
    want = ora.degrees(X, ora.gamma(sigma), queries=q)
    got = b.deg.cpu().numpy()[q]
    assert (np.abs(got - want) <= 1e-5 * want + X.shape[0] * 2.0 ** -126).all()
    smp, _, _ = ora.sample(X, ora.gamma(sigma), L, 5, queries=q)
    assert not ((b.samples.cpu().numpy()[q] != smp) & (b.flags.cpu().numpy()[q] == 0)).any()
    tree.close()
# the split form at d > 64 (three-part operands on the tensor-core kernels)
X = inputs.digit_like(n=1800, d=200, seed=5)
tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
b = fsg.fsg_build_graph(tree, fsg.params(3.0, precision=fsg.FSG_PREC_SPLIT_BF16), 16, 5)
assert fsg.fsg_sync(tree) == 0
out = (__import__("ctypes").c_int64 * 4)()
assert lib.fsg_bounds_error(out) == 0 and list(out) == [0, 0, 0, 0], list(out)
want = ora.degrees(X, ora.gamma(3.0))
assert (np.abs(b.deg.cpu().numpy() - want) <= 1e-4 * want).all()
tree.close()
# a stepped build over uneven ranges (descent and bucketing by range)
X = inputs.gaussian_mixture(n=7001, d=10, seed=6)
tree = fsg.fsg_build_tree(torch.from_numpy(X).cuda())
p = fsg.params(1.5, resolve=True)
whole = fsg.fsg_build_graph(tree, p, 32, 7)
fsg.fsg_graph_begin(tree, p, 32, 7)
for a, c in ((5000, 7001), (0, 1), (1, 5000)):
    fsg.fsg_graph_step(tree, a, c)
st = fsg.fsg_graph_end(tree, 32)
assert fsg.fsg_sync(tree) == 0
assert lib.fsg_bounds_error(out) == 0 and list(out) == [0, 0, 0, 0], list(out)
assert (st.samples.cpu().numpy() == whole.samples.cpu().numpy()).all()
tree.close()
print("bounds build ok")
'''


def test_bounds_checking_build_runs_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, FSG_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-m", "paper_2310_13870_gb300.build"], cwd=ROOT, env=env,
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, FSG_LIB_DIR="_build_bounds", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode == 0 and "bounds build ok" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])
