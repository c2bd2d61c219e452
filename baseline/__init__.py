"""Timed CPU baseline (bench.py and tests only): the paper's CPU kernels with OpenMP.

``omp_graph.cpp`` implements top-down bitmap BFS (Figure 11), pull PageRank (Figure 14) and
Bellman-Ford SSSP (Figure 20) over all host cores. It is a baseline to time against, not
part of the library and not the oracle; tests check it against the oracle. Compiled with
g++ -fopenmp on first use (portable flags: x86-64 and aarch64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "omp_graph.cpp")
_LIB = os.path.join(_HERE, "libomp_graph.so")
_lock = threading.Lock()
_lib = None
INF = 0xFFFFFFFF


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, u32, i32, dbl = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
            lib.omp_threads.restype = i32
            lib.omp_threads.argtypes = []
            lib.omp_bfs.restype = i32
            lib.omp_bfs.argtypes = [u32, vp, vp, u32, vp]
            lib.omp_sssp.restype = i32
            lib.omp_sssp.argtypes = [u32, vp, vp, vp, u32, vp]
            lib.omp_pagerank.restype = dbl
            lib.omp_pagerank.argtypes = [u32, vp, vp, dbl, i32, i32, vp]
            _lib = lib
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def threads() -> int:
    """Threads the OpenMP runtime uses (all host cores unless OMP_NUM_THREADS says less)."""
    return int(_load().omp_threads())


def bfs(n, offsets, cols, source):
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    lv = np.empty(n, np.uint32)
    levels = _load().omp_bfs(n, off.ctypes.data, col.ctypes.data, int(source), lv.ctypes.data)
    return lv, int(levels)


def sssp(n, offsets, cols, weights, source):
    off, col, w = _c(offsets, np.int64), _c(cols, np.uint32), _c(weights, np.uint32)
    d = np.empty(n, np.uint32)
    rounds = _load().omp_sssp(n, off.ctypes.data, col.ctypes.data, w.ctypes.data, int(source),
                              d.ctypes.data)
    if rounds < 0:
        raise OverflowError("a distance reaches 2^32 - 1")
    return d, int(rounds)


def pagerank(n, offsets, cols, damping=0.85, iters=20, dangling=True):
    off, col = _c(offsets, np.int64), _c(cols, np.uint32)
    r = np.empty(n, np.float64)
    res = _load().omp_pagerank(n, off.ctypes.data, col.ctypes.data, float(damping), int(iters),
                               int(bool(dangling)), r.ctypes.data)
    return r, float(res)
