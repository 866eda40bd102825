"""CPU checks of the C ABI: the library loads, exports every function that
include/fsg.h declares, and refuses bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_2310_13870_gb300 import fsg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "fsg.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return fsg.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fsg_build_tree", "fsg_degrees", "fsg_sample_edges", "fsg_build_graph"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(fsg.EXPORTED) == _declared()


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.fsg_version()
    for code in range(0, 8):
        assert lib.fsg_error_string(code)
    assert lib.fsg_error_string(fsg.FSG_ERR_CAPACITY) == b"output buffer too small"


def test_bad_arguments_are_refused_without_gpu(lib):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    assert lib.fsg_build_tree(None, 10, 2, None, None, ctypes.byref(h)) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_build_tree(fake, 0, 2, None, None, ctypes.byref(h)) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_build_tree(fake, 10, 0, None, None, ctypes.byref(h)) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_build_tree(fake, 10, 4097, None, None, ctypes.byref(h)) == fsg.FSG_ERR_INVALID_ARG
    opts = fsg.fsg_tree_opts()
    opts.leaf_max = 100  # not a power of two
    assert lib.fsg_build_tree(fake, 10, 2, ctypes.byref(opts), None, ctypes.byref(h)) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_build_tree(fake, 10, 2, None, None, None) == fsg.FSG_ERR_INVALID_ARG
    opts = fsg.fsg_tree_opts()
    opts.order = 2  # no such order
    assert lib.fsg_build_tree(fake, 10, 2, ctypes.byref(opts), None, ctypes.byref(h)) == fsg.FSG_ERR_INVALID_ARG
    opts.order, opts.d_perm = fsg.FSG_ORDER_SPATIAL, 0x2000  # a computed order and a given one
    assert lib.fsg_build_tree(fake, 10, 2, ctypes.byref(opts), None, ctypes.byref(h)) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_tree_perm(None, fake, None) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_selftest_wait_timeout(10, None) == fsg.FSG_ERR_INVALID_ARG  # limit below 1 us
    p = fsg.params(0.1)
    assert lib.fsg_degrees(None, ctypes.byref(p), fake, None) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_sample_edges(None, ctypes.byref(p), 8, 0, fake, None, None) == fsg.FSG_ERR_INVALID_ARG
    tun = fsg.fsg_tuning()
    assert lib.fsg_autotune(None, ctypes.byref(p), 8, 0, 3, ctypes.byref(tun), None) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_tree_tuning(None, None, ctypes.byref(tun)) == fsg.FSG_ERR_INVALID_ARG
    ev = ctypes.c_int64()
    assert lib.fsg_bin_pass_evals(None, ctypes.byref(p), ctypes.byref(ev)) == fsg.FSG_ERR_INVALID_ARG
    # the stepped build: no tree, no run
    assert lib.fsg_graph_begin(None, ctypes.byref(p), 8, 0, None) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_graph_step(None, 0, 10, None) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_graph_cursor(None, ctypes.byref(ev)) == fsg.FSG_ERR_INVALID_ARG
    assert lib.fsg_graph_end(None, 0, fake, fake, fake, 100, fake, None, None, None, None,
                             None) == fsg.FSG_ERR_INVALID_ARG
    m = ctypes.c_int64()
    buf = (ctypes.c_float * 8)()
    for bad in (fsg.params(0.0), fsg.params(float("nan")), fsg.params(-1.0), fsg.params(0.1, self_mode=3),
                fsg.params(0.1, scale_conv=7), fsg.params(0.1, precision=9), fsg.params(0.1, flag_eps=-1.0),
                fsg.params(0.1, kde_eps=-1e-3), fsg.params(0.1, kde_eps=float("nan")), fsg.params(0.1, kde_eps=0.6),
                fsg.params(0.1, kernel=3), fsg.params(0.1, kernel=-1)):
        rc = lib.fsg_build_graph_host(buf, 4, 2, ctypes.byref(bad), 2, 0, 0, buf, buf, buf, 8, ctypes.byref(m), None)
        assert rc == fsg.FSG_ERR_INVALID_ARG
    # the allocation-free degree call is the exact FP32 pass: an approximate one is not offered
    deg = (ctypes.c_double * 4)()
    approx = fsg.params(0.1, kde_eps=1e-3)
    assert lib.fsg_degrees_noalloc(buf, 4, 2, ctypes.byref(approx), deg, None) == fsg.FSG_ERR_UNSUPPORTED
    # capacity below n*L is refused
    rc = lib.fsg_build_graph_host(buf, 4, 2, ctypes.byref(p), 4, 0, 0, buf, buf, buf, 8, ctypes.byref(m), None)
    assert rc == fsg.FSG_ERR_CAPACITY
    # L outside 1..64
    rc = lib.fsg_build_graph_host(buf, 4, 2, ctypes.byref(p), 65, 0, 0, buf, buf, buf, 1000, ctypes.byref(m), None)
    assert rc == fsg.FSG_ERR_INVALID_ARG
    # server options: budget, slots and admission order are checked before any device call
    sv = ctypes.c_void_p()
    for field, value in (("hbm_budget_bytes", 0), ("max_slots", 0), ("max_slots", 65), ("queue_cap", -1),
                         ("admission", 2), ("admission", -1)):
        o = fsg.fsg_server_opts()
        o.hbm_budget_bytes, o.max_slots = 1 << 30, 4
        setattr(o, field, value)
        assert lib.fsg_server_create(ctypes.byref(o), ctypes.byref(sv)) == fsg.FSG_ERR_INVALID_ARG


def test_struct_layouts_match_header():
    assert ctypes.sizeof(fsg.fsg_batch_item) == 144
    assert ctypes.sizeof(fsg.fsg_server_opts) == 40
    assert ctypes.sizeof(fsg.fsg_request) == 120
    assert ctypes.sizeof(fsg.fsg_result) == 48
    assert ctypes.sizeof(fsg.fsg_params) == 48
    assert fsg.fsg_params.flag_eps.offset == 24 and fsg.fsg_params.kde_eps.offset == 28
    assert fsg.fsg_params.kernel.offset == 32
    assert ctypes.sizeof(fsg.fsg_tree_opts) == 32 and fsg.fsg_tree_opts.order.offset == 12
    assert ctypes.sizeof(fsg.fsg_stats) == 80
