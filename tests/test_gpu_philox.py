"""Philox4x32-10 pinned to cuRAND: the library's device generator and the
oracle's C generator must both reproduce cuRAND's Philox4_32_10 blocks
bit for bit (three implementations, one published definition)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as ora

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = os.path.join(HERE, "cuda", "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "philox_check.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler",
                           "-fPIC", "-I", os.path.join(ROOT, "include"), "-I",
                           os.path.join(ROOT, "paper_2310_13870_gb300", "csrc"),
                           os.path.join(HERE, "cuda", "philox_check.cu"), "-o", so])
    lib = ctypes.CDLL(so)
    lib.philox_check.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF12345678])
def test_device_and_oracle_philox_equal_curand(checker, seed):
    nsub, nk, nl = 5, 9, 3
    cr = np.zeros((nsub, nl, nk, 4), np.uint32)
    fs = np.zeros_like(cr)
    assert checker.philox_check(seed, nsub, nk, nl, cr.ctypes.data, fs.ctypes.data) == 0
    np.testing.assert_array_equal(fs, cr)
    key = [seed & 0xffffffff, seed >> 32]
    for s in range(nsub):
        for l in range(nl):
            for k in range(nk):
                np.testing.assert_array_equal(ora.philox4x32_10([k, l, s, 0], key), cr[s, l, k])
