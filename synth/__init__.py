"""Seeded synthetic inputs shared by the oracle and the GPU path.

Holds no graph-algorithm arithmetic: RMAT edge generation (Table 2 parameters),
symmetrisation, deduplication, vertex relabelling, edge weights, source picking and
random vertex assignments. The C++ implementation lives in ``rmat.cpp``; this module
compiles it on first use (g++, no GPU needed) and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.cpp")
_LIB = os.path.join(_HERE, "librmat.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile librmat.so next to its source (portable flags: x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32, i64, u64, dbl, i32 = (ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_double, ctypes.c_int)
            vp = ctypes.c_void_p
            lib.synth_rmat_csr.restype = vp
            lib.synth_rmat_csr.argtypes = [i32, i32, dbl, dbl, dbl, u64, i32, u64, i32,
                                           ctypes.POINTER(u32), ctypes.POINTER(i64)]
            lib.synth_csr_offsets.restype = vp
            lib.synth_csr_offsets.argtypes = [vp]
            lib.synth_csr_cols.restype = vp
            lib.synth_csr_cols.argtypes = [vp]
            lib.synth_csr_free.restype = None
            lib.synth_csr_free.argtypes = [vp]
            lib.synth_weights.restype = None
            lib.synth_weights.argtypes = [u32, vp, vp, u64, u32, i32, vp]
            lib.synth_sources.restype = i64
            lib.synth_sources.argtypes = [u32, vp, i64, u64, vp]
            lib.synth_permutation.restype = None
            lib.synth_permutation.argtypes = [u32, u64, vp]
            lib.synth_random_assignment.restype = None
            lib.synth_random_assignment.argtypes = [u32, dbl, u64, vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Csr:
    """Symmetric CSR: int64 offsets[n+1], uint32 cols[m], optional uint32 weights[m]."""
    n: int
    offsets: np.ndarray
    cols: np.ndarray
    weights: np.ndarray | None = None
    recipe: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.offsets[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)


class _Owned:
    """Keeps the C++-owned CSR buffers alive while numpy views exist."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if self.handle:
            _load().synth_csr_free(self.handle)
            self.handle = None


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, permute: bool = True, perm_seed: int | None = None,
         threads: int = 0) -> Csr:
    """RMAT graph (Table 2 parameters by default), symmetrised, deduplicated, self-loops
    dropped, vertex ids relabelled by a seeded permutation (perm_seed defaults to seed)."""
    lib = _load()
    n = ctypes.c_uint32(0)
    m = ctypes.c_int64(0)
    ps = seed if perm_seed is None else perm_seed
    h = lib.synth_rmat_csr(scale, edge_factor, a, b, c, seed, int(permute), ps, threads,
                           ctypes.byref(n), ctypes.byref(m))
    if not h:
        raise MemoryError("synth_rmat_csr failed")
    owner = _Owned(h)
    nn, mm = n.value, m.value
    off = np.ctypeslib.as_array(ctypes.cast(lib.synth_csr_offsets(h),
                                            ctypes.POINTER(ctypes.c_int64)), shape=(nn + 1,))
    cols = np.ctypeslib.as_array(ctypes.cast(lib.synth_csr_cols(h),
                                             ctypes.POINTER(ctypes.c_uint32)),
                                 shape=(max(mm, 1),))[:mm]
    # numpy views do not own the memory; pin the owner to the arrays' lifetime.
    off = _attach(off, owner)
    cols = _attach(cols, owner)
    recipe = dict(generator="rmat", scale=scale, edge_factor=edge_factor, a=a, b=b, c=c,
                  seed=seed, permute=bool(permute), perm_seed=ps, symmetrised=True,
                  dedup=True, self_loops=False)
    return Csr(nn, off, cols, None, recipe)


class _View(np.ndarray):
    """ndarray view that keeps the C++ owner of its memory alive (slices included)."""

    def __array_finalize__(self, obj):
        self._owner = getattr(obj, "_owner", None)


def _attach(arr: np.ndarray, owner) -> np.ndarray:
    v = arr.view(_View)
    v._owner = owner
    return v


def weights(g: Csr, wmax: int, seed: int = 3, threads: int = 0) -> np.ndarray:
    """Symmetric uint32 weights uniform in [1, wmax], a seeded hash of the vertex pair."""
    w = np.empty(max(g.m, 1), dtype=np.uint32)
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    cols = np.ascontiguousarray(g.cols, dtype=np.uint32)
    _load().synth_weights(g.n, _ptr(off), _ptr(cols), seed, wmax, threads, _ptr(w))
    g.weights = w[:g.m]
    g.recipe.update(weight_max=wmax, weight_seed=seed)
    return g.weights


def sources(g: Csr, count: int, seed: int = 2) -> np.ndarray:
    """Distinct vertices of degree > 0 from a seeded stream."""
    out = np.empty(max(count, 1), dtype=np.uint32)
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    k = _load().synth_sources(g.n, _ptr(off), count, seed, _ptr(out))
    return out[:k]


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.uint32)
    _load().synth_permutation(n, seed, _ptr(out))
    return out[:n]


def random_assignment(n: int, share0: float, seed: int) -> np.ndarray:
    """uint8 partition id per vertex: 0 with probability share0, else 1."""
    out = np.empty(max(n, 1), dtype=np.uint8)
    _load().synth_random_assignment(n, share0, seed, _ptr(out))
    return out[:n]


def rmat_family(count: int, scales=(10, 17), edge_factors=(8, 32), seed: int = 7,
                threads: int = 0) -> list:
    """`count` independent RMAT graphs (Table 2 parameters) whose scale and edge factor are
    drawn uniformly from the inclusive ranges by a seeded generator; graph i uses RMAT seed
    seed * 1000 + i. The recipe of each graph records its draw."""
    rng = np.random.default_rng(seed)
    sc = rng.integers(scales[0], scales[1] + 1, size=count)
    ef = rng.integers(edge_factors[0], edge_factors[1] + 1, size=count)
    return [rmat(int(sc[i]), int(ef[i]), seed=seed * 1000 + i, threads=threads)
            for i in range(count)]


def disjoint_union(graphs) -> tuple:
    """Block-diagonal union: vertex v of graph i becomes vbase[i] + v. Returns the union
    (weights concatenated when every graph has them) and vbase (uint32, len + 1)."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    ms = np.array([g.m for g in graphs], dtype=np.int64)
    vbase = np.zeros(len(graphs) + 1, dtype=np.int64)
    vbase[1:] = np.cumsum(ns)
    ebase = np.zeros(len(graphs) + 1, dtype=np.int64)
    ebase[1:] = np.cumsum(ms)
    if vbase[-1] >= 2**31:
        raise ValueError("union too large for 31-bit vertex ids")
    off = np.empty(int(vbase[-1]) + 1, dtype=np.int64)
    cols = np.empty(int(ebase[-1]), dtype=np.uint32)
    weighted = all(g.weights is not None for g in graphs) and len(graphs) > 0
    w = np.empty(int(ebase[-1]), dtype=np.uint32) if weighted else None
    for i, g in enumerate(graphs):
        v0, e0 = int(vbase[i]), int(ebase[i])
        off[v0:v0 + g.n] = np.asarray(g.offsets[:-1]) + e0
        cols[e0:e0 + g.m] = np.asarray(g.cols[:g.m]) + np.uint32(v0)
        if weighted:
            w[e0:e0 + g.m] = g.weights[:g.m]
    off[-1] = ebase[-1]
    u = Csr(int(vbase[-1]), off, cols, w,
            dict(generator="disjoint_union", parts=[g.recipe for g in graphs]))
    return u, vbase.astype(np.uint32)


# ---- small structured graphs used by closed-form tests (plain constructions) -------------

def from_edges(n: int, edges, symmetric: bool = True, w=None) -> Csr:
    """CSR from an edge list (u, v[, w]); symmetrises when asked; drops duplicates and
    self-loops; neighbours in ascending order."""
    adj = [dict() for _ in range(n)]
    for k, e in enumerate(edges):
        u, v = int(e[0]), int(e[1])
        wt = None if w is None else int(w[k])
        if u == v:
            continue
        adj[u].setdefault(v, wt)
        if symmetric:
            adj[v].setdefault(u, wt)
    off = np.zeros(n + 1, dtype=np.int64)
    cols, ws = [], []
    for u in range(n):
        nb = sorted(adj[u])
        off[u + 1] = off[u] + len(nb)
        cols.extend(nb)
        if w is not None:
            ws.extend(adj[u][v] for v in nb)
    g = Csr(n, off, np.array(cols, dtype=np.uint32))
    if w is not None:
        g.weights = np.array(ws, dtype=np.uint32)
    return g


def path(n: int) -> Csr:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n: int, directed: bool = False) -> Csr:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], symmetric=not directed)


def grid(w: int, h: int) -> Csr:
    e = []
    for y in range(h):
        for x in range(w):
            v = y * w + x
            if x + 1 < w:
                e.append((v, v + 1))
            if y + 1 < h:
                e.append((v, v + w))
    return from_edges(w * h, e)


def star(k: int) -> Csr:
    """Centre 0 joined to leaves 1..k."""
    return from_edges(k + 1, [(0, i) for i in range(1, k + 1)])


def complete(n: int) -> Csr:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def erdos_renyi(n: int, p: float, seed: int, symmetric: bool = True) -> Csr:
    rng = np.random.default_rng(seed)
    e = [(i, j) for i in range(n) for j in range(n) if i != j and rng.random() < p]
    return from_edges(n, e, symmetric=symmetric)
