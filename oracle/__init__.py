"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python access to ``oracle.c``: plain, single-threaded reference computations of BFS
levels, shortest-path distances, FP64 PageRank, the two-way partition, betweenness
centrality and connected components, plus validators.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg (and its
``--impl reference`` arm) may import this package. The CUDA library never calls it, and it
shares no code with the CUDA sources; the two meet only in the seeded inputs of ``synth``.

Pinned against closed forms, brute force and library routines in
``tests/test_oracle_pins.py``. Every function here is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

INF = 0xFFFFFFFF
REMOTE = 0x80000000
NCLASS = 34

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, -O2, no vectorisation pragmas, single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    vp, u32, i32, dbl, i64 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int,
                              ctypes.c_double, ctypes.c_int64)
    lib.orc_bfs.restype = i32
    lib.orc_bfs.argtypes = [u32, vp, vp, u32, vp, vp]
    lib.orc_sssp.restype = i32
    lib.orc_sssp.argtypes = [u32, vp, vp, vp, u32, vp]
    lib.orc_pagerank.restype = i32
    lib.orc_pagerank.argtypes = [u32, vp, vp, dbl, i32, dbl, i32, vp, vp, vp]
    lib.orc_partition.restype = i32
    lib.orc_partition.argtypes = [u32, vp, vp, vp, vp] + [vp] * 6 + [vp, vp, vp, vp]
    lib.orc_check_bfs.restype = i32
    lib.orc_check_bfs.argtypes = [u32, vp, vp, u32, vp, vp]
    lib.orc_check_sssp.restype = i32
    lib.orc_check_sssp.argtypes = [u32, vp, vp, vp, u32, vp]
    lib.orc_traversed.restype = i64
    lib.orc_traversed.argtypes = [u32, vp, vp]
    lib.orc_bc.restype = i32
    lib.orc_bc.argtypes = [u32, vp, vp, u32, vp, vp, vp]
    lib.orc_cc.restype = i32
    lib.orc_cc.argtypes = [u32, vp, vp, vp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


def bfs(n, offsets, cols, source, want_parents=True):
    """Levels (uint32, INF unreached) and one valid parent array (parent[source]=source)."""
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    level = np.empty(max(n, 1), np.uint32)
    parent = np.empty(max(n, 1), np.uint32) if want_parents else None
    rc = _load().orc_bfs(n, _p(off), _p(col), int(source), _p(level), _p(parent))
    if rc:
        raise OracleError(f"orc_bfs rc={rc}")
    return level[:n], (parent[:n] if want_parents else None)


def sssp(n, offsets, cols, weights, source):
    """Shortest-path distances (uint32, INF unreached). Raises if a distance overflows."""
    off, col, w = _c(offsets, np.int64), _c(cols, np.uint32), _c(weights, np.uint32)
    dist = np.empty(max(n, 1), np.uint32)
    rc = _load().orc_sssp(n, _p(off), _p(col), _p(w), int(source), _p(dist))
    if rc:
        raise OracleError(f"orc_sssp rc={rc}")
    return dist[:n]


def pagerank(n, offsets, cols, damping=0.85, max_iter=20, tol=0.0, dangling=1):
    """FP64 ranks after the iterations run, residual history, iteration count."""
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    r = np.empty(max(n, 1), np.float64)
    res = np.zeros(max(max_iter, 1), np.float64)
    it = ctypes.c_int(0)
    rc = _load().orc_pagerank(n, _p(off), _p(col), float(damping), int(max_iter), float(tol),
                              int(dangling), _p(r), _p(res), ctypes.addressof(it))
    if rc:
        raise OracleError(f"orc_pagerank rc={rc}")
    return r[:n], res[:it.value], it.value


def partition(n, offsets, cols, assign, weights=None):
    """Two-way partition (see oracle.c). Returns a dict of numpy arrays per partition."""
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    asg = _c(assign, np.uint8)
    w = None if weights is None else _c(weights, np.uint32)
    deg = np.diff(off)
    nvp = [int((asg == p).sum()) for p in (0, 1)]
    nep = [int(deg[asg == p].sum()) for p in (0, 1)]
    l2g = [np.zeros(max(nvp[p], 1), np.uint32) for p in (0, 1)]
    poff = [np.zeros(nvp[p] + 1, np.int64) for p in (0, 1)]
    pE = [np.zeros(max(nep[p], 1), np.uint32) for p in (0, 1)]
    pW = [np.zeros(max(nep[p], 1), np.uint32) for p in (0, 1)]
    outb = [np.zeros(max(nvp[1 - p], 1), np.uint32) for p in (0, 1)]
    cls = [np.zeros(NCLASS, np.uint32) for p in (0, 1)]
    g2l = np.zeros(max(n, 1), np.uint32)
    nv = np.zeros(2, np.uint32)
    ne = np.zeros(2, np.int64)
    nout = np.zeros(2, np.uint32)

    def arr(lst):
        a = (ctypes.c_void_p * 2)(*[x.ctypes.data for x in lst])
        return a

    A = [arr(l2g), arr(poff), arr(pE), arr(pW), arr(outb), arr(cls)]
    rc = _load().orc_partition(n, _p(off), _p(col), _p(w), _p(asg),
                               *[ctypes.cast(a, ctypes.c_void_p) for a in A],
                               _p(g2l), _p(nv), _p(ne), _p(nout))
    if rc:
        raise OracleError(f"orc_partition rc={rc}")
    parts = []
    for p in (0, 1):
        parts.append(dict(nv=int(nv[p]), ne=int(ne[p]), l2g=l2g[p][:nv[p]], off=poff[p],
                          E=pE[p][:ne[p]], W=(pW[p][:ne[p]] if w is not None else None),
                          outbox=outb[p][:nout[p]], cls_end=cls[p]))
    return dict(parts=parts, g2l=g2l[:n])


def check_bfs(n, offsets, cols, source, level, parent=None) -> int:
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    lv = _c(level, np.uint32)
    pa = None if parent is None else _c(parent, np.uint32)
    return _load().orc_check_bfs(n, _p(off), _p(col), int(source), _p(lv), _p(pa))


def check_sssp(n, offsets, cols, weights, source, dist) -> int:
    off, col, w = _c(offsets, np.int64), _c(cols, np.uint32), _c(weights, np.uint32)
    d = _c(dist, np.uint32)
    return _load().orc_check_sssp(n, _p(off), _p(col), _p(w), int(source), _p(d))


def traversed(n, offsets, value) -> int:
    """Sum of degrees of the vertices whose value is not INF (TEPS numerator, Section 5)."""
    off = _c(offsets, np.int64)
    v = _c(value, np.uint32)
    return int(_load().orc_traversed(n, _p(off), _p(v)))


def degree_assignment(offsets, threshold):
    """HIGH rule of Section 6.3.1 on one GPU: partition 0 holds vertices of degree >= T."""
    deg = np.diff(np.asarray(offsets, dtype=np.int64))
    return np.where(deg >= threshold, 0, 1).astype(np.uint8)


def edge_share_threshold(offsets, share):
    """Largest T such that the vertices of degree >= T hold at least `share` of all edge
    entries: the HIGH strategy of Section 6.3.1, which places the highest-degree vertices
    in one partition until it holds a chosen share of the edges. share <= 0 gives a T above the maximum degree (no hubs)."""
    deg = np.diff(np.asarray(offsets, dtype=np.int64))
    m = int(deg.sum())
    if share <= 0 or m == 0:
        return int(deg.max(initial=0)) + 1
    need = share * m
    ds = np.sort(deg)[::-1]
    csum = np.cumsum(ds)
    # first prefix of the descending degree order that reaches the share; every vertex of
    # that prefix's last degree joins (ties included).
    k = min(int(np.searchsorted(csum, need, side="left")), len(ds) - 1)
    return int(ds[k])


def bc(n, offsets, cols, sources):
    """FP64 betweenness scores summed over the sources (Brandes), and the TEPS numerator
    (twice the degree sum of the reached vertices, per source)."""
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    src = _c(sources, np.uint32)
    out = np.zeros(max(n, 1), np.float64)
    trav = ctypes.c_int64(0)
    rc = _load().orc_bc(n, _p(off), _p(col), len(src), _p(src), _p(out), ctypes.addressof(trav))
    if rc:
        raise OracleError(f"orc_bc rc={rc}")
    return out[:n], trav.value


def cc(n, offsets, cols):
    """Component label of every vertex: the smallest vertex id of its component."""
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    out = np.empty(max(n, 1), np.uint32)
    rc = _load().orc_cc(n, _p(off), _p(col), _p(out))
    if rc:
        raise OracleError(f"orc_cc rc={rc}")
    return out[:n]
