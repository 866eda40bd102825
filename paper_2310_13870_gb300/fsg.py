"""Python binding of libfsg.so (include/fsg.h): argument marshalling only.

Every step of the path runs in the library's sm_103a kernels; this module
allocates output tensors with PyTorch, passes raw device pointers and the
current CUDA stream, and turns status codes into exceptions.  There is no
fallback: if libfsg.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FSG_LIB_DIR=_build_bounds selects the bounds-checking build (see build.py)
LIB_PATH = os.path.join(_HERE, os.environ.get("FSG_LIB_DIR", "_build"), "libfsg.so")

FSG_OK = 0
FSG_ERR_INVALID_ARG = 1
FSG_ERR_OOM = 2
FSG_ERR_CUDA = 3
FSG_ERR_TIMEOUT = 4
FSG_ERR_UNSUPPORTED = 5
FSG_ERR_BUSY = 6
FSG_ERR_CAPACITY = 7
FSG_ERR_SCRATCH = 8
FSG_ERR_CANCELLED = 9
FSG_ERR_BOUNDS = 10

FSG_TWO_SIGMA_SQ, FSG_SIGMA_SQ = 0, 1
FSG_SELF_EXCLUDE, FSG_SELF_INCLUDE = 0, 1
FSG_PREC_AUTO, FSG_PREC_FP32, FSG_PREC_SPLIT_BF16, FSG_PREC_EXACT_INT = 0, 1, 2, 3
FSG_EDGES_SET, FSG_EDGES_MULTI = 0, 1
FSG_SCHED_FUSED, FSG_SCHED_LEVELWISE, FSG_SCHED_CARRIED = 0, 1, 2
FSG_ADMIT_ARRIVAL, FSG_ADMIT_RESPONSE_RATIO = 0, 1
FSG_ORDER_IDENTITY, FSG_ORDER_SPATIAL = 0, 1
FSG_KERNEL_GAUSSIAN, FSG_KERNEL_LAPLACIAN, FSG_KERNEL_EXPONENTIAL = 0, 1, 2

# Names every build of the library must export (checked by the CPU tests
# against include/fsg.h).
EXPORTED = [
    "fsg_version", "fsg_error_string", "fsg_build_tree", "fsg_free_tree", "fsg_tree_info", "fsg_bin_pass_evals",
    "fsg_spatial_order", "fsg_tree_perm",
    "fsg_autotune", "fsg_tree_tuning",
    "fsg_degrees", "fsg_sample_edges", "fsg_build_graph", "fsg_sync", "fsg_build_graph_host",
    "fsg_tree_update", "fsg_profile", "fsg_profile_read", "fsg_degrees_noalloc",
    "fsg_batch_create", "fsg_batch_run", "fsg_batch_destroy",
    "fsg_server_create", "fsg_server_submit", "fsg_server_poll", "fsg_server_cancel", "fsg_server_info",
    "fsg_server_destroy", "fsg_selftest_wait_timeout", "fsg_bounds_error",
    "fsg_graph_begin", "fsg_graph_step", "fsg_graph_cursor", "fsg_graph_end",
]
FSG_NUM_PHASES = 8
PHASES = ["tree", "kde_bins", "descend_top", "bucket", "leaf_finish", "edges", "outputs", "resolve"]


class FsgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib_or_none().fsg_error_string(status).decode() if _lib_or_none() else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class fsg_params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("scale_conv", ctypes.c_int32), ("self_mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("schedule", ctypes.c_int32), ("flag_eps", ctypes.c_float),
                ("kde_eps", ctypes.c_float), ("kernel", ctypes.c_int32), ("resolve", ctypes.c_int32),
                ("weight_f64", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class fsg_tree_opts(ctypes.Structure):
    _fields_ = [("d_perm", ctypes.c_void_p), ("leaf_max", ctypes.c_int32), ("order", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class fsg_batch_item(ctypes.Structure):
    _fields_ = [("d_points", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("L", ctypes.c_int32),
                ("params", fsg_params), ("seed", ctypes.c_uint64), ("edge_mode", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("d_src", ctypes.c_void_p), ("d_dst", ctypes.c_void_p),
                ("d_w", ctypes.c_void_p), ("cap", ctypes.c_int64), ("d_m_out", ctypes.c_void_p),
                ("d_deg", ctypes.c_void_p), ("d_stats", ctypes.c_void_p)]


class fsg_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("queue_cap", ctypes.c_int32),
                ("inject_alloc_fail_every", ctypes.c_int32), ("admission", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class fsg_request(ctypes.Structure):
    _fields_ = [("h_points", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("L", ctypes.c_int32),
                ("params", fsg_params), ("seed", ctypes.c_uint64), ("edge_mode", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("h_src", ctypes.c_void_p), ("h_dst", ctypes.c_void_p),
                ("h_w", ctypes.c_void_p), ("cap", ctypes.c_int64)]


class fsg_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("n_edges", ctypes.c_int64), ("n_flagged", ctypes.c_int64), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double)]


STATS_FIELDS = ["n_samples", "n_flagged", "n_self", "n_empty", "n_evals", "n_items", "n_edges", "status",
                "n_bin_evals", "n_resolved"]


class fsg_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in STATS_FIELDS]


_lib = None


def _lib_or_none():
    return _lib


def load(path: str = LIB_PATH):
    """Loads libfsg.so (built by paper_2310_13870_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    lib.fsg_version.restype = ctypes.c_char_p
    lib.fsg_version.argtypes = []
    lib.fsg_error_string.restype = ctypes.c_char_p
    lib.fsg_error_string.argtypes = [ctypes.c_int]
    lib.fsg_build_tree.argtypes = [P, I64, I32, P, P, ctypes.POINTER(P)]
    lib.fsg_free_tree.argtypes = [P]
    lib.fsg_free_tree.restype = None
    lib.fsg_tree_info.argtypes = [P, P, P, P]
    lib.fsg_bin_pass_evals.argtypes = [P, P, P]
    lib.fsg_autotune.argtypes = [P, P, I32, U64, I32, P, P]
    lib.fsg_tree_tuning.argtypes = [P, P, P]
    lib.fsg_degrees.argtypes = [P, P, P, P]
    lib.fsg_sample_edges.argtypes = [P, P, I32, U64, P, P, P]
    lib.fsg_build_graph.argtypes = [P, P, I32, U64, I32, P, P, P, I64, P, P, P, P, P, P]
    lib.fsg_sync.argtypes = [P, P]
    lib.fsg_build_graph_host.argtypes = [P, I64, I32, P, I32, U64, I32, P, P, P, I64, P, P]
    lib.fsg_tree_update.argtypes = [P, P, P]
    lib.fsg_profile.argtypes = [P, ctypes.c_int]
    lib.fsg_profile_read.argtypes = [P, P, P]
    lib.fsg_degrees_noalloc.argtypes = [P, I64, I32, P, P, P]
    lib.fsg_batch_create.argtypes = [P, I32, I32, I32, P, ctypes.POINTER(P)]
    lib.fsg_batch_run.argtypes = [P, P]
    lib.fsg_batch_destroy.argtypes = [P]
    lib.fsg_batch_destroy.restype = None
    lib.fsg_server_create.argtypes = [P, ctypes.POINTER(P)]
    lib.fsg_server_submit.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint64)]
    lib.fsg_server_poll.argtypes = [P, P, I32, ctypes.POINTER(ctypes.c_int32), I32]
    lib.fsg_server_cancel.argtypes = [P, ctypes.c_uint64]
    lib.fsg_server_info.argtypes = [P, P, P, P]
    lib.fsg_server_destroy.argtypes = [P]
    lib.fsg_server_destroy.restype = None
    lib.fsg_spatial_order.argtypes = [P, ctypes.c_int64, I32, I32, P]
    lib.fsg_tree_perm.argtypes = [P, P, P]
    lib.fsg_selftest_wait_timeout.argtypes = [ctypes.c_int64, P]
    lib.fsg_bounds_error.argtypes = [P]
    lib.fsg_graph_begin.argtypes = [P, P, I32, U64, P]
    lib.fsg_graph_step.argtypes = [P, I64, I64, P]
    lib.fsg_graph_cursor.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.fsg_graph_end.argtypes = [P, I32, P, P, P, I64, P, P, P, P, P, P]
    for name in EXPORTED:
        if name not in ("fsg_version", "fsg_error_string", "fsg_free_tree", "fsg_batch_destroy", "fsg_server_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != FSG_OK:
        raise FsgError(rc, where)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def params(sigma: float, scale_conv: int = FSG_TWO_SIGMA_SQ, self_mode: int = FSG_SELF_EXCLUDE,
           precision: int = FSG_PREC_AUTO, schedule: int = FSG_SCHED_FUSED, flag_eps: float = 0.0,
           kde_eps: float = 0.0, kernel: int = 0, resolve: bool = False, weight_f64: bool = False) -> fsg_params:
    p = fsg_params()
    p.sigma = float(sigma)
    p.scale_conv = scale_conv
    p.self_mode = self_mode
    p.precision = precision
    p.schedule = schedule
    p.flag_eps = float(flag_eps)
    p.kde_eps = float(kde_eps)
    p.kernel = int(kernel)
    p.resolve = int(bool(resolve))
    p.weight_f64 = int(bool(weight_f64))
    return p


class Tree:
    """Owns an fsg_tree*; freed on close() or garbage collection."""

    def __init__(self, handle: ctypes.c_void_p, n: int, d: int):
        self.handle = handle
        self.n = n
        self.d = d

    def close(self):
        if self.handle is not None and _lib is not None:
            _lib.fsg_free_tree(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def depth(self) -> int:
        n, d, dep = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().fsg_tree_info(self.handle, ctypes.byref(n), ctypes.byref(d), ctypes.byref(dep)), "fsg_tree_info")
        return int(dep.value)


def fsg_build_tree(points, perm=None, leaf_max: int = 0, stream=None, order: int = 0) -> Tree:
    """points: CUDA float32 [n][d] contiguous; perm: optional CUDA int32 [n];
    order: FSG_ORDER_IDENTITY or FSG_ORDER_SPATIAL (computed on the GPU)."""
    import torch
    lib = load()
    if not (points.is_cuda and points.dtype == torch.float32 and points.dim() == 2):
        raise ValueError("points must be a CUDA float32 [n][d] tensor")
    points = points.contiguous()
    opts = fsg_tree_opts()
    opts.d_perm = None if perm is None else perm.contiguous().data_ptr()
    opts.leaf_max = leaf_max
    opts.order = order
    h = ctypes.c_void_p()
    _check(lib.fsg_build_tree(_dptr(points), points.shape[0], points.shape[1], ctypes.byref(opts),
                              _stream_ptr(stream), ctypes.byref(h)), "fsg_build_tree")
    return Tree(h, points.shape[0], points.shape[1])


def fsg_tree_perm(tree: Tree, stream=None):
    """The tree's order as a CUDA int32 [n] tensor (position -> original index)."""
    import torch
    out = torch.empty(tree.n, dtype=torch.int32, device="cuda")
    _check(load().fsg_tree_perm(tree.handle, _dptr(out), _stream_ptr(stream)), "fsg_tree_perm")
    return out


def fsg_spatial_order(points: np.ndarray, leaf: int = 32) -> np.ndarray:
    """Host spatial tree order (see fsg.h): int32 [n], position -> original index."""
    X = np.ascontiguousarray(points, dtype=np.float32)
    n, d = X.shape
    perm = np.empty(n, np.int32)
    _check(load().fsg_spatial_order(X.ctypes.data, n, d, leaf, perm.ctypes.data), "fsg_spatial_order")
    return perm


def fsg_tree_update(tree: Tree, points, stream=None):
    """Refills the tree with new points of the same shape (no allocation)."""
    import torch
    if not (points.is_cuda and points.dtype == torch.float32 and tuple(points.shape) == (tree.n, tree.d)):
        raise ValueError("points must be a CUDA float32 tensor of the tree's shape")
    points = points.contiguous()
    _check(load().fsg_tree_update(tree.handle, _dptr(points), _stream_ptr(stream)), "fsg_tree_update")


def fsg_bin_pass_evals(tree: Tree, p: fsg_params) -> int:
    """Kernel evaluations the fused schedule's bin pass executes (see fsg.h)."""
    v = ctypes.c_int64()
    _check(load().fsg_bin_pass_evals(tree.handle, ctypes.byref(p), ctypes.byref(v)), "fsg_bin_pass_evals")
    return int(v.value)


class fsg_tuning(ctypes.Structure):
    _fields_ = [("sym_bins", ctypes.c_int32), ("tc_bins", ctypes.c_int32), ("leaf_splits", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


def _tuning_dict(t: fsg_tuning) -> dict:
    return {"sym_bins": t.sym_bins, "tc_bins": t.tc_bins, "leaf_splits": t.leaf_splits}


def fsg_autotune(tree: Tree, p: fsg_params, L: int, seed: int = 0, reps: int = 3, stream=None) -> dict:
    """Times the launch shapes of the bin pass and leaf finish, keeps the fastest (see fsg.h)."""
    out = fsg_tuning()
    _check(load().fsg_autotune(tree.handle, ctypes.byref(p), int(L), int(seed), int(reps), ctypes.byref(out),
                               _stream_ptr(stream)), "fsg_autotune")
    return _tuning_dict(out)


def fsg_tree_tuning(tree: Tree, tuning: dict | None = None) -> dict:
    """Sets (if given) and returns the tree's launch shapes (0 = heuristic)."""
    t = None
    if tuning is not None:
        t = fsg_tuning()
        t.sym_bins = int(tuning.get("sym_bins", 0))
        t.tc_bins = int(tuning.get("tc_bins", 0))
        t.leaf_splits = int(tuning.get("leaf_splits", 0))
    out = fsg_tuning()
    _check(load().fsg_tree_tuning(tree.handle, ctypes.byref(t) if t is not None else None, ctypes.byref(out)),
           "fsg_tree_tuning")
    return _tuning_dict(out)


def fsg_profile(tree: Tree, enable: bool = True):
    _check(load().fsg_profile(tree.handle, int(enable)), "fsg_profile")


def fsg_profile_read(tree: Tree):
    """Returns ({phase: ms} of the last profiled call, total kernel launches)."""
    ms = (ctypes.c_float * FSG_NUM_PHASES)()
    launches = ctypes.c_int64()
    _check(load().fsg_profile_read(tree.handle, ms, ctypes.byref(launches)), "fsg_profile_read")
    return dict(zip(PHASES, list(ms))), int(launches.value)


def fsg_degrees(tree: Tree, p: fsg_params, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty(tree.n, dtype=torch.float64, device="cuda")
    _check(load().fsg_degrees(tree.handle, ctypes.byref(p), _dptr(out), _stream_ptr(stream)), "fsg_degrees")
    return out


def fsg_degrees_noalloc(points, p: fsg_params, out=None, stream=None):
    """Degrees through the allocation-free entry point (no tree object; the
    library's fixed device scratch is used; see include/fsg.h)."""
    import torch
    if not (points.is_cuda and points.dtype == torch.float32 and points.dim() == 2):
        raise ValueError("points must be a CUDA float32 [n][d] tensor")
    points = points.contiguous()
    if out is None:
        out = torch.empty(points.shape[0], dtype=torch.float64, device=points.device)
    _check(load().fsg_degrees_noalloc(_dptr(points), points.shape[0], points.shape[1], ctypes.byref(p), _dptr(out),
                                      _stream_ptr(stream)), "fsg_degrees_noalloc")
    return out


def fsg_sample_edges(tree: Tree, p: fsg_params, L: int, seed: int, samples=None, flags=None, stream=None):
    import torch
    if samples is None:
        samples = torch.empty((tree.n, L), dtype=torch.int32, device="cuda")
    if flags is None:
        flags = torch.empty((tree.n, L), dtype=torch.uint8, device="cuda")
    _check(load().fsg_sample_edges(tree.handle, ctypes.byref(p), L, ctypes.c_uint64(seed), _dptr(samples),
                                   _dptr(flags), _stream_ptr(stream)), "fsg_sample_edges")
    return samples, flags


class GraphBuffers:
    """Device output buffers of fsg_build_graph, reusable across calls."""

    def __init__(self, n: int, L: int, with_aux: bool = True, weight_f64: bool = False):
        import torch
        cap = n * L
        self.cap = cap
        self.src = torch.empty(cap, dtype=torch.int32, device="cuda")
        self.dst = torch.empty(cap, dtype=torch.int32, device="cuda")
        self.w = torch.empty(cap, dtype=torch.float64 if weight_f64 else torch.float32, device="cuda")
        self.m = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.stats = torch.zeros(len(STATS_FIELDS), dtype=torch.int64, device="cuda")
        self.deg = torch.empty(n, dtype=torch.float64, device="cuda") if with_aux else None
        self.samples = torch.empty((n, L), dtype=torch.int32, device="cuda") if with_aux else None
        self.flags = torch.empty((n, L), dtype=torch.uint8, device="cuda") if with_aux else None


def fsg_build_graph(tree: Tree, p: fsg_params, L: int, seed: int, edge_mode: int = FSG_EDGES_SET,
                    bufs: Optional[GraphBuffers] = None, stream=None) -> GraphBuffers:
    import torch
    if bufs is None:
        bufs = GraphBuffers(tree.n, L, weight_f64=bool(p.weight_f64))
    if bufs.w.dtype != (torch.float64 if p.weight_f64 else torch.float32):
        raise ValueError("the weight buffer's dtype does not match params.weight_f64")
    _check(load().fsg_build_graph(tree.handle, ctypes.byref(p), L, ctypes.c_uint64(seed), edge_mode,
                                  _dptr(bufs.src), _dptr(bufs.dst), _dptr(bufs.w), bufs.cap, _dptr(bufs.m),
                                  _dptr(bufs.deg), _dptr(bufs.samples), _dptr(bufs.flags), _dptr(bufs.stats),
                                  _stream_ptr(stream)), "fsg_build_graph")
    return bufs


def fsg_graph_begin(tree: Tree, p: fsg_params, L: int, seed: int, stream=None):
    """Stepped build: the bin pass of every query (kept in the tree)."""
    _check(load().fsg_graph_begin(tree.handle, ctypes.byref(p), L, ctypes.c_uint64(seed), _stream_ptr(stream)),
           "fsg_graph_begin")


def fsg_graph_step(tree: Tree, q_begin: int, q_end: int, stream=None):
    """Stepped build: sampling of the queries at tree positions [q_begin, q_end)."""
    _check(load().fsg_graph_step(tree.handle, q_begin, q_end, _stream_ptr(stream)), "fsg_graph_step")


def fsg_graph_cursor(tree: Tree) -> int:
    c = ctypes.c_int64()
    _check(load().fsg_graph_cursor(tree.handle, ctypes.byref(c)), "fsg_graph_cursor")
    return int(c.value)


def fsg_graph_end(tree: Tree, L: int, edge_mode: int = FSG_EDGES_SET, bufs: Optional[GraphBuffers] = None,
                  weight_f64: bool = False, stream=None) -> GraphBuffers:
    """Stepped build: edge list and outputs once every position was stepped."""
    if bufs is None:
        bufs = GraphBuffers(tree.n, L, weight_f64=weight_f64)
    _check(load().fsg_graph_end(tree.handle, edge_mode, _dptr(bufs.src), _dptr(bufs.dst), _dptr(bufs.w), bufs.cap,
                                _dptr(bufs.m), _dptr(bufs.deg), _dptr(bufs.samples), _dptr(bufs.flags),
                                _dptr(bufs.stats), _stream_ptr(stream)), "fsg_graph_end")
    return bufs


def stats_dict(bufs: GraphBuffers) -> dict:
    v = bufs.stats.cpu().tolist()
    return dict(zip(STATS_FIELDS, v))


def fsg_sync(tree: Tree, stream=None) -> int:
    rc = load().fsg_sync(tree.handle, _stream_ptr(stream))
    _check(rc, "fsg_sync")
    return rc


def fsg_build_graph_host(points: np.ndarray, p: fsg_params, L: int, seed: int, edge_mode: int = FSG_EDGES_SET,
                         out=None, stream=None):
    """End to end on host arrays: returns (src, dst, w) numpy views of `out`.
    `out` = (src int32 [cap], dst int32 [cap], w float32 [cap]) host arrays
    (pinned recommended) with cap >= n*L."""
    X = np.ascontiguousarray(points, dtype=np.float32)
    n, d = X.shape
    if out is None:
        cap = n * L
        out = (np.empty(cap, np.int32), np.empty(cap, np.int32), np.empty(cap, np.float32))
    src, dst, w = out
    m = ctypes.c_int64()
    _check(load().fsg_build_graph_host(X.ctypes.data_as(ctypes.c_void_p), n, d, ctypes.byref(p), L,
                                       ctypes.c_uint64(seed), edge_mode, src.ctypes.data_as(ctypes.c_void_p),
                                       dst.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                       src.shape[0], ctypes.byref(m), _stream_ptr(stream)), "fsg_build_graph_host")
    k = int(m.value)
    return src[:k], dst[:k], w[:k]


class Batch:
    """Graph builds of many point sets (fsg_batch_*).  `sets` is a list of
    (points CUDA float32 [n][d], fsg_params, L, seed); output buffers are
    allocated here and reused by every run()."""

    def __init__(self, sets, edge_mode: int = FSG_EDGES_SET, streams: int = 4, capture: bool = True, stream=None):
        lib = load()
        self.sets = sets
        self.bufs = []
        arr = (fsg_batch_item * len(sets))()
        for i, (pts, p, L, seed) in enumerate(sets):
            b = GraphBuffers(pts.shape[0], L, with_aux=False)
            b.deg = __import__("torch").empty(pts.shape[0], dtype=__import__("torch").float64, device="cuda")
            self.bufs.append(b)
            it = arr[i]
            it.d_points = pts.data_ptr()
            it.n = pts.shape[0]
            it.d = pts.shape[1]
            it.L = L
            it.params = p
            it.seed = seed
            it.edge_mode = edge_mode
            it.d_src, it.d_dst, it.d_w = b.src.data_ptr(), b.dst.data_ptr(), b.w.data_ptr()
            it.cap = b.cap
            it.d_m_out = b.m.data_ptr()
            it.d_deg = b.deg.data_ptr()
            it.d_stats = b.stats.data_ptr()
        self._items = arr
        h = ctypes.c_void_p()
        _check(lib.fsg_batch_create(arr, len(sets), streams, int(capture), _stream_ptr(stream), ctypes.byref(h)),
               "fsg_batch_create")
        self.handle = h

    def run(self, stream=None):
        _check(load().fsg_batch_run(self.handle, _stream_ptr(stream)), "fsg_batch_run")

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.fsg_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The library's request loop (fsg_server_*).  submit() takes host numpy
    points and returns an id; the edge list lands in host buffers allocated
    here (pinned) and is returned by poll() with the result record."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 8, queue_cap: int = 0,
                 inject_alloc_fail_every: int = 0, admission: int = 0):
        o = fsg_server_opts()
        o.admission = admission
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        o.max_slots = max_slots
        o.queue_cap = queue_cap
        o.inject_alloc_fail_every = inject_alloc_fail_every
        h = ctypes.c_void_p()
        _check(load().fsg_server_create(ctypes.byref(o), ctypes.byref(h)), "fsg_server_create")
        self.handle = h
        self.live = {}  # id -> (points, src, dst, w) kept alive until polled

    def submit(self, points: np.ndarray, p: fsg_params, L: int, seed: int, edge_mode: int = FSG_EDGES_SET,
               pinned: bool = True, out=None) -> int:
        """out: optional (src, dst, w) host arrays of >= n*L elements (e.g.
        pinned buffers reused by the caller); points are then used as given."""
        import torch
        X = np.ascontiguousarray(points, dtype=np.float32)
        n, d = X.shape
        cap = n * L
        if out is not None:
            src, dst, w = out
            cap = min(src.shape[0], dst.shape[0], w.shape[0])
        elif pinned:
            Xt = torch.from_numpy(X).pin_memory()
            X = Xt.numpy()
            src = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
            dst = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
            w = torch.empty(cap, dtype=torch.float32).pin_memory().numpy()
        else:
            src, dst, w = np.empty(cap, np.int32), np.empty(cap, np.int32), np.empty(cap, np.float32)
        r = fsg_request()
        r.h_points = X.ctypes.data
        r.n, r.d, r.L = n, d, L
        r.params = p
        r.seed = seed
        r.edge_mode = edge_mode
        r.h_src, r.h_dst, r.h_w = src.ctypes.data, dst.ctypes.data, w.ctypes.data
        r.cap = cap
        rid = ctypes.c_uint64()
        _check(load().fsg_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)), "fsg_server_submit")
        self.live[rid.value] = (X, src, dst, w)
        return rid.value

    def poll(self, max_results: int = 256, wait_ms: int = 0):
        """Returns a list of (result dict, (src, dst, w) numpy views)."""
        arr = (fsg_result * max_results)()
        cnt = ctypes.c_int32()
        _check(load().fsg_server_poll(self.handle, arr, max_results, ctypes.byref(cnt), wait_ms), "fsg_server_poll")
        out = []
        for k in range(cnt.value):
            r = arr[k]
            rec = dict(id=r.id, status=r.status, n_edges=r.n_edges, n_flagged=r.n_flagged, latency_ms=r.latency_ms,
                       queue_ms=r.queue_ms)
            X, src, dst, w = self.live.pop(r.id, (None, None, None, None))
            m = r.n_edges if r.status == FSG_OK else 0
            out.append((rec, (src[:m], dst[:m], w[:m]) if src is not None else None))
        return out

    def cancel(self, rid: int):
        _check(load().fsg_server_cancel(self.handle, ctypes.c_uint64(rid)), "fsg_server_cancel")

    def info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().fsg_server_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "fsg_server_info")
        return dict(pending=a.value, in_flight=b.value, bytes_in_use=c.value)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.fsg_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
