"""GB300 BSP graph library: Python binding of the C ABI in include/graph.h.

The functions below have the names of the C entry points and only marshal arguments:
every step (load validation, partitioning, BFS, SSSP, PageRank, exchange, collect) runs in
the CUDA library. PyTorch supplies device memory (its caching allocator, through the
allocator hooks of graph_runtime) and the stream. There is no CPU fallback: if the
compiled library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from ._lib import (GRAPH_BFS_AUTO, GRAPH_BFS_BOTTOMUP, GRAPH_BFS_TOPDOWN, GRAPH_INF,
                   GRAPH_MEM_DEVICE, GRAPH_MEM_HOST, GRAPH_PART_DEGREE, GRAPH_PART_EXPLICIT,
                   GRAPH_PART_NONE, GRAPH_PR_FP16, GRAPH_PR_FP32, GRAPH_PR_FP64, GraphError)

__all__ = ["graph_load_csr", "graph_partition", "graph_get_partition_info",
           "graph_export_partition", "bfs", "bfs_batch", "sssp", "sssp_batch", "betweenness",
           "connected_components", "pagerank", "pagerank_hybrid", "pagerank_multi",
           "bfs_csr_noalloc", "Server", "graph_free", "Graph", "GraphError", "INF",
           "library_path"]

INF = GRAPH_INF
_PREC = {"fp32": GRAPH_PR_FP32, "fp64": GRAPH_PR_FP64, "fp16": GRAPH_PR_FP16}
_DIR = {"auto": GRAPH_BFS_AUTO, "topdown": GRAPH_BFS_TOPDOWN, "bottomup": GRAPH_BFS_BOTTOMUP}


def library_path() -> str:
    return _lib.lib_path()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device available: this library has no CPU path")
    return torch


def _ptr(a):
    """Data pointer and memory kind of a numpy array or a torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data, GRAPH_MEM_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (GRAPH_MEM_DEVICE if a.is_cuda else GRAPH_MEM_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


@dataclass
class Graph:
    """Owns a graph_t handle and the allocator callbacks it uses."""
    handle: int
    n: int
    m: int
    stream: int
    keep: list = field(default_factory=list)

    def free(self):
        if self.handle:
            _lib.load().graph_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _torch_runtime(torch, stream):
    dev = torch.cuda.current_device()

    @_lib.ALLOC_FN
    def alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=stream)
        except Exception:
            return None

    @_lib.FREE_FN
    def free(ptr, nbytes, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    rt = _lib.graph_runtime(alloc, free, None, stream)
    return rt, [alloc, free]


def graph_load_csr(offsets, cols, weights=None, *, n: int | None = None, stream=None,
                   allocator: str = "torch") -> Graph:
    """Copy a CSR graph (int64 offsets[n+1], uint32 cols[m], optional uint32 weights[m])
    from host numpy arrays or device tensors into the library. allocator: "torch" (the
    caching allocator) or "cuda" (cudaMalloc inside the library)."""
    torch = _torch()
    if isinstance(offsets, np.ndarray):
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.uint32)
        if weights is not None:
            weights = np.ascontiguousarray(weights, dtype=np.uint32)
    nn = (len(offsets) - 1) if n is None else n
    m = int(offsets[-1]) if isinstance(offsets, np.ndarray) else int(offsets[-1].item())
    po, mem = _ptr(offsets)
    pc, memc = _ptr(cols)
    pw, memw = _ptr(weights)
    if memc != mem or (weights is not None and memw != mem):
        raise ValueError("offsets, cols and weights must live in the same memory")
    s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
    keep = []
    if allocator == "torch":
        rt, keep = _torch_runtime(torch, s)
    elif allocator == "cuda":
        rt = _lib.graph_runtime(_lib.ALLOC_FN(), _lib.FREE_FN(), None, s)
    else:
        raise ValueError("allocator must be 'torch' or 'cuda'")
    out = C.c_void_p(0)
    st = _lib.load().graph_load_csr(nn, m, po, pc, pw, mem, C.byref(rt), C.byref(out))
    _lib.check(st, "graph_load_csr")
    return Graph(out.value, nn, m, s, keep)


def graph_partition(g: Graph, strategy: str = "degree", *, degree_threshold: int = 2048,
                    edge_share: float = 0.0, assignment=None) -> dict:
    """strategy: "none" (one partition), "degree" (HIGH: partition 0 = degree >= T; T from
    degree_threshold, or from edge_share when > 0), "explicit" (uint8 assignment per vertex,
    e.g. a seeded random split)."""
    attr = _lib.graph_partition_attr()
    attr.strategy = {"none": GRAPH_PART_NONE, "degree": GRAPH_PART_DEGREE,
                     "explicit": GRAPH_PART_EXPLICIT}[strategy]
    attr.degree_threshold = int(degree_threshold)
    attr.edge_share = float(edge_share)
    keep = None
    if assignment is not None:
        keep = np.ascontiguousarray(assignment, dtype=np.uint8)
        attr.assignment = keep.ctypes.data
    _lib.check(_lib.load().graph_partition(g.handle, C.byref(attr)), "graph_partition")
    return graph_get_partition_info(g)


def graph_get_partition_info(g: Graph) -> dict:
    info = _lib.graph_partition_info()
    _lib.check(_lib.load().graph_get_partition_info(g.handle, C.byref(info)),
               "graph_get_partition_info")
    return dict(n=info.n, m=info.m, threshold=info.threshold, nv=list(info.nv),
                ne=list(info.ne), nout=list(info.nout),
                cls_end=[np.array(list(info.cls_end[p]), dtype=np.uint32) for p in (0, 1)],
                bytes_graph=info.bytes_graph)


def graph_export_partition(g: Graph, p: int, weights: bool = False) -> dict:
    info = graph_get_partition_info(g)
    nv, ne, nout = info["nv"][p], info["ne"][p], info["nout"][p]
    l2g = np.zeros(max(nv, 1), np.uint32)
    off = np.zeros(nv + 1, np.int64)
    E = np.zeros(max(ne, 1), np.uint32)
    W = np.zeros(max(ne, 1), np.uint32) if weights else None
    ob = np.zeros(max(nout, 1), np.uint32)
    g2l = np.zeros(g.n, np.uint32)
    st = _lib.load().graph_export_partition(g.handle, p, l2g.ctypes.data, off.ctypes.data,
                                            E.ctypes.data,
                                            None if W is None else W.ctypes.data,
                                            ob.ctypes.data, g2l.ctypes.data)
    _lib.check(st, "graph_export_partition")
    return dict(nv=nv, ne=ne, l2g=l2g[:nv], off=off, E=E[:ne],
                W=None if W is None else W[:ne], outbox=ob[:nout],
                cls_end=info["cls_end"][p], g2l=g2l)


_EDGE_PARTS = {"part0": 1, "part1": 2, "input": 4}


def graph_set_edge_memory(g: Graph, which, mem: str):
    """Moves edge arrays to page-locked host memory ("host"; kernels read them over the host
    link) or back to device memory ("device"). which: "part0", "part1", "input" or a list
    of them."""
    if isinstance(which, str):
        which = [which]
    mask = 0
    for w in which:
        mask |= _EDGE_PARTS[w]
    memv = {"host": GRAPH_MEM_HOST, "device": GRAPH_MEM_DEVICE}[mem]
    _lib.check(_lib.load().graph_set_edge_memory(g.handle, mask, memv), "graph_set_edge_memory")


def graph_get_edge_memory(g: Graph) -> dict:
    """{"part0": "host"|"device", "part1": ..., "input": ...}"""
    v = C.c_int(0)
    _lib.check(_lib.load().graph_get_edge_memory(g.handle, C.byref(v)), "graph_get_edge_memory")
    return {k: ("host" if v.value & b else "device") for k, b in _EDGE_PARTS.items()}


def _out_u32(torch, n, out, given):
    if given is not None:
        return given
    if out == "device":
        return torch.empty(n, dtype=torch.int32, device="cuda")
    return np.empty(n, dtype=np.uint32)


def as_numpy_u32(a) -> np.ndarray:
    if isinstance(a, np.ndarray):
        return a.view(np.uint32)
    return a.cpu().numpy().view(np.uint32)


def bfs(g: Graph, source: int, levels=None, parents=None, *, want_parents: bool = True,
        direction: str = "auto", alpha: float = 0.0, beta: float = 0.0, out: str = "device",
        max_supersteps: int = 0, timing: bool = False):
    """Levels and parents (uint32, INF unreached) in global vertex order, and stats."""
    torch = _torch()
    levels = _out_u32(torch, g.n, out, levels)
    if want_parents:
        parents = _out_u32(torch, g.n, out, parents)
    pl, mem = _ptr(levels)
    pp, memp = _ptr(parents) if want_parents else (None, mem)
    if memp != mem:
        raise ValueError("levels and parents must live in the same memory")
    attr = _lib.bfs_attr(mem, _DIR[direction], alpha, beta, max_supersteps, int(timing))
    stats = _lib.graph_stats()
    st = _lib.load().bfs(g.handle, int(source), pl, pp, C.byref(attr), C.byref(stats))
    _lib.check(st, "bfs")
    return levels, (parents if want_parents else None), stats.as_dict()


def bfs_batch(g: Graph, sources, levels=None, *, direction: str = "auto", alpha: float = 0.0,
              out: str = "device", max_supersteps: int = 0, timing: bool = False):
    """k = len(sources) <= BATCH_MAX searches in one pass of supersteps; levels [k, n]
    uint32 (row s for sources[s], INF unreached) and stats."""
    torch = _torch()
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64))
    if src.ndim != 1 or np.any(src < 0) or np.any(src >= 2**32):
        raise ValueError("sources must be a 1-D list of vertex ids")
    src = src.astype(np.uint32)
    k = len(src)
    if levels is None:
        levels = (torch.empty((k, g.n), dtype=torch.int32, device="cuda") if out == "device"
                  else np.empty((k, g.n), dtype=np.uint32))
    pl, mem = _ptr(levels)
    attr = _lib.bfs_attr(mem, _DIR[direction], alpha, 0.0, max_supersteps, int(timing))
    stats = _lib.graph_stats()
    st = _lib.load().bfs_batch(g.handle, src.ctypes.data, k, pl, C.byref(attr), C.byref(stats))
    _lib.check(st, "bfs_batch")
    return levels, stats.as_dict()


def sssp(g: Graph, source: int, dist=None, *, out: str = "device", max_supersteps: int = 0,
         timing: bool = False, delta: int = 0):
    """Shortest distances (uint32, INF unreachable) in global vertex order, and stats.
    delta = 0: plain active-set rounds (Figure 20); delta > 0: near-far order."""
    torch = _torch()
    dist = _out_u32(torch, g.n, out, dist)
    pd, mem = _ptr(dist)
    attr = _lib.sssp_attr(mem, max_supersteps, int(timing), int(delta))
    stats = _lib.graph_stats()
    st = _lib.load().sssp(g.handle, int(source), pd, C.byref(attr), C.byref(stats))
    _lib.check(st, "sssp")
    return dist, stats.as_dict()


def bfs_hybrid(g: Graph, source: int, levels=None, parents=None, *, cpu_threads: int = 0,
               want_parents: bool = True, out: str = "device", max_supersteps: int = 0):
    """BFS with partition 0 expanded on cpu_threads host threads and partition 1 on the GPU
    (the paper's hybrid placement, top-down). Returns (levels, parents, stats);
    stats["hybrid"] holds the per-processor sizes and times."""
    torch = _torch()
    levels = _out_u32(torch, g.n, out, levels)
    if want_parents:
        parents = _out_u32(torch, g.n, out, parents)
    pl, mem = _ptr(levels)
    pp, memp = _ptr(parents) if want_parents else (None, mem)
    if memp != mem:
        raise ValueError("levels and parents must live in the same memory")
    attr = _lib.bfs_attr(mem, _DIR["topdown"], 0.0, 0.0, max_supersteps, 0)
    stats = _lib.graph_stats()
    info = _lib.pagerank_hybrid_info()
    st = _lib.load().bfs_hybrid(g.handle, int(source), pl, pp, C.byref(attr), int(cpu_threads),
                                C.byref(stats), C.byref(info))
    _lib.check(st, "bfs_hybrid")
    d = stats.as_dict()
    d["hybrid"] = info.as_dict()
    return levels, (parents if want_parents else None), d


def sssp_hybrid(g: Graph, source: int, dist=None, *, cpu_threads: int = 0, out: str = "device",
                max_supersteps: int = 0):
    """SSSP (plain Bellman-Ford rounds) with partition 0 on cpu_threads host threads and
    partition 1 on the GPU. Returns (distances, stats); stats["hybrid"] as for bfs_hybrid."""
    torch = _torch()
    dist = _out_u32(torch, g.n, out, dist)
    pd, mem = _ptr(dist)
    attr = _lib.sssp_attr(mem, max_supersteps, 0, 0)
    stats = _lib.graph_stats()
    info = _lib.pagerank_hybrid_info()
    st = _lib.load().sssp_hybrid(g.handle, int(source), pd, C.byref(attr), int(cpu_threads),
                                 C.byref(stats), C.byref(info))
    _lib.check(st, "sssp_hybrid")
    d = stats.as_dict()
    d["hybrid"] = info.as_dict()
    return dist, d


def sssp_batch(g: Graph, sources, dist=None, *, out: str = "device", max_supersteps: int = 0,
               timing: bool = False, delta: int = 0):
    """k = len(sources) <= SSSP_BATCH_MAX shortest-path searches in one pass of Bellman-Ford
    supersteps (delta > 0: near-far order with one threshold for all searches); distances
    [k, n] uint32 (row s for sources[s], INF unreachable) and stats."""
    torch = _torch()
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64))
    if src.ndim != 1 or np.any(src < 0) or np.any(src >= 2**32):
        raise ValueError("sources must be a 1-D list of vertex ids")
    src = src.astype(np.uint32)
    k = len(src)
    if dist is None:
        dist = (torch.empty((k, g.n), dtype=torch.int32, device="cuda") if out == "device"
                else np.empty((k, g.n), dtype=np.uint32))
    pd, mem = _ptr(dist)
    attr = _lib.sssp_attr(mem, max_supersteps, int(timing), int(delta))
    stats = _lib.graph_stats()
    st = _lib.load().sssp_batch(g.handle, src.ctypes.data, k, pd, C.byref(attr),
                                C.byref(stats))
    _lib.check(st, "sssp_batch")
    return dist, stats.as_dict()


def betweenness(g: Graph, sources, scores=None, *, out: str = "device", timing: bool = False):
    """Betweenness centrality summed over the sources (FP64, global order), and stats."""
    torch = _torch()
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64))
    if src.ndim != 1 or np.any(src < 0) or np.any(src >= 2**32):
        raise ValueError("sources must be a 1-D list of vertex ids")
    src = src.astype(np.uint32)
    if scores is None:
        scores = (torch.empty(g.n, dtype=torch.float64, device="cuda") if out == "device"
                  else np.empty(g.n, dtype=np.float64))
    ps, mem = _ptr(scores)
    attr = _lib.bc_attr(mem, int(timing))
    stats = _lib.graph_stats()
    st = _lib.load().betweenness(g.handle, src.ctypes.data, len(src), ps, C.byref(attr),
                                 C.byref(stats))
    _lib.check(st, "betweenness")
    return scores, stats.as_dict()


def connected_components(g: Graph, labels=None, *, out: str = "device", max_supersteps: int = 0,
                         timing: bool = False):
    """Component labels (the smallest vertex id of each component, uint32) and stats."""
    torch = _torch()
    labels = _out_u32(torch, g.n, out, labels)
    pl, mem = _ptr(labels)
    attr = _lib.cc_attr(mem, int(max_supersteps), int(timing))
    stats = _lib.graph_stats()
    st = _lib.load().connected_components(g.handle, pl, C.byref(attr), C.byref(stats))
    _lib.check(st, "connected_components")
    return labels, stats.as_dict()


_METHOD = {"auto": 0, "gather": 1, "segmented": 2}


def pagerank(g: Graph, *, damping: float = 0.85, max_iter: int = 20, tol: float = 0.0,
             precision: str = "fp32", dangling: bool = True, ranks=None, out: str = "device",
             timing: bool = False, method: str = "auto", seg_log2: int = 0,
             seg_chunk: int = 0, seg_bin: int = 0):
    """FP64 ranks in global vertex order, and stats (residual = last L1 change).
    method: 'auto' (= 'gather'), 'gather' or 'segmented' (FP32 / FP16); seg_* are the
    segmented layout's parameters (0 = default)."""
    torch = _torch()
    if ranks is None:
        ranks = (torch.empty(g.n, dtype=torch.float64, device="cuda") if out == "device"
                 else np.empty(g.n, dtype=np.float64))
    pr_, mem = _ptr(ranks)
    attr = _lib.pagerank_attr(float(damping), int(max_iter), float(tol), _PREC[precision],
                              int(bool(dangling)), mem, int(timing), _METHOD[method],
                              int(seg_log2), int(seg_chunk), int(seg_bin))
    stats = _lib.graph_stats()
    st = _lib.load().pagerank(g.handle, C.byref(attr), pr_, C.byref(stats))
    _lib.check(st, "pagerank")
    return ranks, stats.as_dict()


def pagerank_plan(g: Graph) -> dict:
    """Layout of the segmented plan of g's current partition (all zero before one is built)."""
    info = _lib.pagerank_plan_info()
    _lib.check(_lib.load().pagerank_plan_get(g.handle, C.byref(info)), "pagerank_plan_get")
    return info.as_dict()


def pagerank_hybrid(g: Graph, *, cpu_threads: int = 0, damping: float = 0.85,
                    max_iter: int = 20, tol: float = 0.0, precision: str = "fp32",
                    dangling: bool = True, ranks=None, out: str = "device",
                    timing: bool = False):
    """PageRank with partition 0 updated on cpu_threads host threads and partition 1 on
    the GPU (the paper's hybrid placement). Returns (FP64 ranks in global order, stats);
    stats["hybrid"] holds the per-processor sizes and times."""
    torch = _torch()
    if ranks is None:
        ranks = (torch.empty(g.n, dtype=torch.float64, device="cuda") if out == "device"
                 else np.empty(g.n, dtype=np.float64))
    pr_, mem = _ptr(ranks)
    attr = _lib.pagerank_attr(float(damping), int(max_iter), float(tol), _PREC[precision],
                              int(bool(dangling)), mem, int(timing))
    stats = _lib.graph_stats()
    info = _lib.pagerank_hybrid_info()
    st = _lib.load().pagerank_hybrid(g.handle, C.byref(attr), int(cpu_threads), pr_,
                                     C.byref(stats), C.byref(info))
    _lib.check(st, "pagerank_hybrid")
    d = stats.as_dict()
    d["hybrid"] = info.as_dict()
    return ranks, d


def pagerank_multi(g: Graph, vbase, *, damping: float = 0.85, max_iter: int = 30,
                   precision: str = "fp32", dangling: bool = True, ranks=None,
                   out: str = "device", timing: bool = False):
    """PageRank of each component [vbase[c], vbase[c+1]) of the loaded union, max_iter
    iterations in one replayed CUDA graph. Returns (FP64 ranks in global order, per-component
    residual of the last iteration, stats)."""
    torch = _torch()
    vb = np.ascontiguousarray(np.asarray(vbase, dtype=np.int64))
    if vb.ndim != 1 or len(vb) < 2 or np.any(vb < 0) or np.any(vb >= 2**32):
        raise ValueError("vbase must be a 1-D list of at least two vertex ids")
    vb = vb.astype(np.uint32)
    G = len(vb) - 1
    if ranks is None:
        ranks = (torch.empty(g.n, dtype=torch.float64, device="cuda") if out == "device"
                 else np.empty(g.n, dtype=np.float64))
    pr_, mem = _ptr(ranks)
    res = np.zeros(G, dtype=np.float64)
    attr = _lib.pagerank_attr(float(damping), int(max_iter), 0.0, _PREC[precision],
                              int(bool(dangling)), mem, int(timing))
    stats = _lib.graph_stats()
    st = _lib.load().pagerank_multi(g.handle, G, vb.ctypes.data, C.byref(attr), pr_,
                                    res.ctypes.data, C.byref(stats))
    _lib.check(st, "pagerank_multi")
    return ranks, res, stats.as_dict()


class Server:
    """Continuous-batching query server on a resident, partitioned graph (graph_server_*):
    BFS queries share the lanes of one multi-source search, SSSP queries run on job slots
    sized by a device-memory budget. Outputs are caller arrays of n uint32 (host: numpy,
    pinned for speed; device: torch tensors) kept alive here until their query completes."""

    KINDS = {"bfs": _lib.GRAPH_QUERY_BFS, "sssp": _lib.GRAPH_QUERY_SSSP}

    def __init__(self, g: Graph, *, mem_budget: int = 0, bfs_lanes: int = 0, max_sssp: int = 0,
                 out: str = "device", sssp_delta: int = 0, sssp_batch: bool = False):
        _torch()
        self.g = g
        self.out = out
        mem = GRAPH_MEM_DEVICE if out == "device" else GRAPH_MEM_HOST
        attr = _lib.graph_server_attr(int(mem_budget), int(bfs_lanes), int(max_sssp), mem,
                                      int(sssp_delta), int(bool(sssp_batch)))
        h = C.c_void_p(0)
        _lib.check(_lib.load().graph_server_create(g.handle, C.byref(attr), C.byref(h)),
                   "graph_server_create")
        self.handle = h.value
        self._outs = {}

    def submit(self, kind: str, source: int, out) -> int:
        ptr, mem = _ptr(out)
        if mem != (GRAPH_MEM_DEVICE if self.out == "device" else GRAPH_MEM_HOST):
            raise ValueError("output array in the wrong memory for this server")
        t = C.c_uint64(0)
        _lib.check(_lib.load().graph_server_submit(self.handle, self.KINDS[kind], int(source),
                                                   ptr, C.byref(t)), "graph_server_submit")
        self._outs[t.value] = out
        return t.value

    def poll(self, cap: int = 256, wait_ms: int = 0) -> list:
        buf = (_lib.graph_completion * cap)()
        k = C.c_uint32(0)
        _lib.check(_lib.load().graph_server_poll(self.handle, buf, cap, C.byref(k), int(wait_ms)),
                   "graph_server_poll")
        res = []
        for c in buf[:k.value]:
            d = {f: getattr(c, f) for f, _ in c._fields_}
            d["kind"] = "bfs" if c.kind == _lib.GRAPH_QUERY_BFS else "sssp"
            d["out"] = self._outs.pop(c.ticket, None)
            res.append(d)
        return res

    def info(self) -> dict:
        i = _lib.graph_server_info()
        _lib.check(_lib.load().graph_server_info_get(self.handle, C.byref(i)),
                   "graph_server_info_get")
        return i.as_dict()

    def close(self):
        if self.handle:
            _lib.check(_lib.load().graph_server_destroy(self.handle), "graph_server_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def bfs_csr_noalloc(offsets, cols, source: int, levels=None, parents=None, *, stream=None,
                    want_parents: bool = True):
    """Allocation-free BFS on a CSR already in device memory (torch CUDA tensors: int64
    offsets[n+1], 32-bit cols[m]). For callers that cannot allocate device memory when they
    search: the library keeps its scratch in one fixed device array of 17.0 MB (16.25 MiB)
    and allocates nothing; pass preallocated `levels`/`parents` (32-bit CUDA tensors of
    length n) to keep this wrapper allocation-free as well. n is limited to 2^21 vertices.
    Calls share the scratch array and must not overlap on the GPU; the first call on a
    device should come before any stream capture. The call waits for the device after the
    CSR check and after every level, so it returns with the search complete.

    Raises ValueError before any device work unless offsets is a contiguous int64 tensor,
    cols, levels and parents contiguous 32-bit integer tensors of the right lengths, and all
    of them on one CUDA device; the call then runs with that device current."""
    torch = _torch()
    i32 = (torch.int32, getattr(torch, "uint32", torch.int32))

    def need(t, name, dtypes, length):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor (got {t.device})")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} has dtype {t.dtype}; expected one of {dtypes}")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 1-D tensor")
        if length is not None and t.numel() != length:
            raise ValueError(f"{name} has {t.numel()} elements; expected {length}")
        if t.device != offsets.device:
            raise ValueError(f"{name} is on {t.device}, offsets on {offsets.device}")

    need(offsets, "offsets", (torch.int64,), None)
    n = offsets.numel() - 1
    if n < 1:
        raise ValueError("offsets must hold n + 1 >= 2 entries")
    need(cols, "cols", i32, None)
    m = cols.numel()
    with torch.cuda.device(offsets.device):
        if levels is None:
            levels = torch.empty(n, dtype=torch.int32, device=offsets.device)
        if want_parents and parents is None:
            parents = torch.empty(n, dtype=torch.int32, device=offsets.device)
        need(levels, "levels", i32, n)
        if want_parents:
            need(parents, "parents", i32, n)
        s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
        st = _lib.load().bfs_csr_noalloc(n, m, offsets.data_ptr(),
                                         cols.data_ptr() if m > 0 else None, int(source),
                                         levels.data_ptr(),
                                         parents.data_ptr() if want_parents else None, s)
    _lib.check(st, "bfs_csr_noalloc")
    return levels, (parents if want_parents else None)


def graph_free(g: Graph) -> None:
    g.free()
