"""FP64 CPU oracle for the FastSimilarityGraph hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
import this package.  It wraps the plain C implementation in ``fsg_oracle.c``
(compiled by :func:`build`) with ctypes and numpy; it shares no code with the
CUDA library.  What each routine follows in the paper (Macgregor & Sun,
NeurIPS 2023) is stated beside it in ``fsg_oracle.c``:

* ``kernel``/``kde``      -- Gaussian kernel (Sec. 2.1) and the KDE of Eq. 1;
* ``degrees``             -- g_[1,n](x_i) of Algorithm 2;
* ``sample``              -- the halving descent of Algorithm 1 / Sec. 4.1;
* ``weights``             -- the re-weighting of Eq. 2 / Algorithm 2;
* ``build_graph``         -- the whole of Algorithm 2 (small n);
* ``philox4x32_10``       -- the counter-based generator (Salmon et al., SC'11).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsg_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

TWO_SIGMA_SQ, SIGMA_SQ = 0, 1
SELF_EXCLUDE, SELF_INCLUDE = 0, 1
EDGES_SET, EDGES_MULTI = 0, 1
GAUSSIAN, LAPLACIAN, EXPONENTIAL = 0, 1, 2  # kernel families of Sec. 2.1

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64, no fast-math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fsg_oracle.h"))
    ):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
             _SRC, "-o", tmp, "-lm", "-lpthread"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64, i32, u32, u64, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    P = ctypes.c_void_p
    lib.ora_philox4x32_10.argtypes = [P, P, P]
    lib.ora_philox4x32_10.restype = None
    lib.ora_draw_u32.argtypes = [u64, u32, u32, u32]
    lib.ora_draw_u32.restype = u32
    lib.ora_uniform.argtypes = [u64, u32, u32, u32]
    lib.ora_uniform.restype = f64
    lib.ora_gamma.argtypes = [f64, i32]
    lib.ora_gamma.restype = f64
    lib.ora_scale.argtypes = [f64, i32, i32]
    lib.ora_scale.restype = f64
    lib.ora_kernel.argtypes = [P, P, i32, f64, i32]
    lib.ora_kernel.restype = f64
    lib.ora_split.argtypes = [i64, i64]
    lib.ora_split.restype = i64
    lib.ora_kde.argtypes = [P, i64, i32, P, f64, i32, i32, i64, i64, i64]
    lib.ora_kde.restype = f64
    lib.ora_num_threads.argtypes = [i32]
    lib.ora_num_threads.restype = i32
    lib.ora_degrees.argtypes = [P, i64, i32, f64, i32, i32, P, i64, P, i32]
    lib.ora_degrees.restype = i32
    lib.ora_sample.argtypes = [P, i64, i32, P, f64, i32, i32, i32, u64, P, i64, P, P, P, i32]
    lib.ora_sample.restype = i32
    lib.ora_path_prob.argtypes = [P, i64, i32, P, f64, i32, i32, i64, i64]
    lib.ora_path_prob.restype = f64
    lib.ora_weights.argtypes = [P, i64, i32, f64, i32, i32, P, i64, P, P, P, P]
    lib.ora_weights.restype = i32
    lib.ora_build_graph.argtypes = [P, i64, i32, P, f64, i32, i32, i32, u64, i32, P, P, P, i64, P, P, P, P, i32]
    lib.ora_build_graph.restype = i32
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _points(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("points must be [n][d]")
    return X


def _perm(perm):
    return None if perm is None else np.ascontiguousarray(perm, dtype=np.int64)


def num_threads(requested: int = 0) -> int:
    return int(_load().ora_num_threads(int(requested)))


def gamma(sigma: float, scale_conv: int = TWO_SIGMA_SQ) -> float:
    return float(_load().ora_gamma(float(sigma), int(scale_conv)))


def scale(sigma: float, kernel: int = GAUSSIAN, scale_conv: int = TWO_SIGMA_SQ) -> float:
    """The family's scale: gamma for the Gaussian, 1/sigma for the Laplacian
    and exponential kernels."""
    return float(_load().ora_scale(float(sigma), int(scale_conv), int(kernel)))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().ora_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw_u32(seed: int, i: int, l: int, level: int) -> int:
    return int(_load().ora_draw_u32(seed, i, l, level))


def uniform(seed: int, i: int, l: int, level: int) -> float:
    return float(_load().ora_uniform(seed, i, l, level))


def split(lo: int, hi: int) -> int:
    return int(_load().ora_split(lo, hi))


def kernel(a, b, gam: float, kernel: int = GAUSSIAN) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().ora_kernel(_ptr(a), _ptr(b), a.shape[0], gam, kernel))


def kde(X, gam, i, lo, hi, perm=None, self_mode=SELF_EXCLUDE, kernel=GAUSSIAN) -> float:
    X = _points(X)
    p = _perm(perm)
    return float(_load().ora_kde(_ptr(X), X.shape[0], X.shape[1], _ptr(p), gam, kernel, self_mode, i, lo, hi))


def degrees(X, gam, queries=None, self_mode=SELF_EXCLUDE, nthreads=0, kernel=GAUSSIAN):
    X = _points(X)
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = X.shape[0] if q is None else q.shape[0]
    out = np.zeros(nq, dtype=np.float64)
    rc = _load().ora_degrees(_ptr(X), X.shape[0], X.shape[1], gam, kernel, self_mode, _ptr(q), nq, _ptr(out),
                             nthreads)
    if rc != 0:
        raise ValueError(f"ora_degrees failed ({rc})")
    return out


def sample(X, gam, L, seed, queries=None, perm=None, self_mode=SELF_EXCLUDE, nthreads=0, kernel=GAUSSIAN):
    """Returns (samples[nq][L] int64, margin[nq][L] f64, levels[nq][L] i32)."""
    X = _points(X)
    p = _perm(perm)
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = X.shape[0] if q is None else q.shape[0]
    smp = np.zeros((nq, L), dtype=np.int64)
    mrg = np.zeros((nq, L), dtype=np.float64)
    lev = np.zeros((nq, L), dtype=np.int32)
    rc = _load().ora_sample(_ptr(X), X.shape[0], X.shape[1], _ptr(p), gam, kernel, self_mode, L, seed,
                            _ptr(q), nq, _ptr(smp), _ptr(mrg), _ptr(lev), nthreads)
    if rc != 0:
        raise ValueError(f"ora_sample failed ({rc})")
    return smp, mrg, lev


def path_prob(X, gam, i, p, perm=None, self_mode=SELF_EXCLUDE, kernel=GAUSSIAN) -> float:
    X = _points(X)
    pp = _perm(perm)
    return float(_load().ora_path_prob(_ptr(X), X.shape[0], X.shape[1], _ptr(pp), gam, kernel, self_mode, i, p))


def weights(X, gam, L, deg, src, dst, kernel=GAUSSIAN):
    """Returns (k, w) for the given pairs; deg indexed by original index."""
    X = _points(X)
    deg = np.ascontiguousarray(deg, dtype=np.float64)
    s = np.ascontiguousarray(src, dtype=np.int64)
    t = np.ascontiguousarray(dst, dtype=np.int64)
    k = np.zeros(s.shape[0], dtype=np.float64)
    w = np.zeros(s.shape[0], dtype=np.float64)
    rc = _load().ora_weights(_ptr(X), X.shape[0], X.shape[1], gam, kernel, L, _ptr(deg), s.shape[0],
                             _ptr(s), _ptr(t), _ptr(k), _ptr(w))
    if rc != 0:
        raise ValueError(f"ora_weights failed ({rc})")
    return k, w


def build_graph(X, gam, L, seed, perm=None, self_mode=SELF_EXCLUDE, edge_mode=EDGES_SET, nthreads=0,
                kernel=GAUSSIAN):
    """Whole of Algorithm 2.  Returns dict(src, dst, w, deg, samples, n_self)."""
    X = _points(X)
    n = X.shape[0]
    p = _perm(perm)
    cap = n * L
    src = np.zeros(cap, dtype=np.int64)
    dst = np.zeros(cap, dtype=np.int64)
    w = np.zeros(cap, dtype=np.float64)
    m = np.zeros(1, dtype=np.int64)
    deg = np.zeros(n, dtype=np.float64)
    smp = np.zeros((n, L), dtype=np.int64)
    nself = np.zeros(1, dtype=np.int64)
    rc = _load().ora_build_graph(_ptr(X), n, X.shape[1], _ptr(p), gam, kernel, self_mode, L, seed, edge_mode,
                                 _ptr(src), _ptr(dst), _ptr(w), cap, _ptr(m), _ptr(deg), _ptr(smp),
                                 _ptr(nself), nthreads)
    if rc != 0:
        raise ValueError(f"ora_build_graph failed ({rc})")
    mm = int(m[0])
    return dict(src=src[:mm], dst=dst[:mm], w=w[:mm], deg=deg, samples=smp, n_self=int(nself[0]))
