"""ctypes declarations mirroring include/graph.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

GRAPH_OK = 0
GRAPH_EINVAL = -1
GRAPH_ENOMEM = -2
GRAPH_ECUDA = -3
GRAPH_ETIMEOUT = -4
GRAPH_ERANGE = -5
GRAPH_ESTATE = -6
GRAPH_INF = 0xFFFFFFFF
GRAPH_MEM_HOST = 0
GRAPH_MEM_DEVICE = 1
GRAPH_PART_NONE = 0
GRAPH_PART_DEGREE = 1
GRAPH_PART_EXPLICIT = 2
GRAPH_BFS_AUTO = 0
GRAPH_BFS_TOPDOWN = 1
GRAPH_BFS_BOTTOMUP = 2
GRAPH_PR_FP32 = 0
GRAPH_PR_FP64 = 1
GRAPH_PR_FP16 = 2
GRAPH_NOALLOC_MAX_VERTICES = 1 << 21
GRAPH_BATCH_MAX = 64
GRAPH_SSSP_BATCH_MAX = 8
GRAPH_QUERY_BFS = 0
GRAPH_QUERY_SSSP = 1

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class graph_runtime(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p),
                ("stream", C.c_void_p)]


class graph_partition_attr(C.Structure):
    _fields_ = [("strategy", C.c_int), ("degree_threshold", C.c_uint32),
                ("edge_share", C.c_double), ("assignment", C.c_void_p)]


class graph_partition_info(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m", C.c_int64), ("threshold", C.c_uint32),
                ("nv", C.c_uint32 * 2), ("ne", C.c_int64 * 2), ("nout", C.c_uint32 * 2),
                ("cls_end", (C.c_uint32 * 34) * 2), ("bytes_graph", C.c_int64)]


class bc_attr(C.Structure):
    _fields_ = [("out_mem", C.c_int), ("timing", C.c_int)]


class cc_attr(C.Structure):
    _fields_ = [("out_mem", C.c_int), ("max_supersteps", C.c_int), ("timing", C.c_int)]


class graph_server_attr(C.Structure):
    _fields_ = [("mem_budget", C.c_uint64), ("bfs_lanes", C.c_uint32), ("max_sssp", C.c_uint32),
                ("out_mem", C.c_int), ("sssp_delta", C.c_uint32), ("sssp_batch", C.c_uint32)]


class graph_completion(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("kind", C.c_int), ("status", C.c_int),
                ("source", C.c_uint32), ("supersteps", C.c_int), ("t_submit_ms", C.c_double),
                ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double)]


class graph_server_info(C.Structure):
    _fields_ = [("bfs_lanes", C.c_uint32), ("sssp_slots", C.c_uint32),
                ("bytes_lanes", C.c_uint64), ("bytes_per_sssp", C.c_uint64),
                ("mem_budget", C.c_uint64), ("submitted", C.c_uint64),
                ("completed", C.c_uint64), ("pending", C.c_uint64),
                ("max_lanes_busy", C.c_uint32), ("max_slots_busy", C.c_uint32),
                ("bfs_supersteps", C.c_uint64), ("sssp_batch_slots", C.c_uint32),
                ("max_batch_busy", C.c_uint32), ("bytes_per_sssp_batch", C.c_uint64),
                ("sssp_batched", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class graph_stats(C.Structure):
    _fields_ = [("supersteps", C.c_int), ("topdown_steps", C.c_int),
                ("bottomup_steps", C.c_int), ("edges_traversed", C.c_int64),
                ("edges_inspected", C.c_int64), ("messages", C.c_int64),
                ("residual", C.c_double), ("ms_total", C.c_double),
                ("ms_compute", C.c_double), ("ms_exchange", C.c_double),
                ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bfs_attr(C.Structure):
    _fields_ = [("out_mem", C.c_int), ("direction", C.c_int), ("alpha", C.c_double),
                ("beta", C.c_double), ("max_supersteps", C.c_int), ("timing", C.c_int)]


class sssp_attr(C.Structure):
    _fields_ = [("out_mem", C.c_int), ("max_supersteps", C.c_int), ("timing", C.c_int),
                ("delta", C.c_uint32)]


class pagerank_attr(C.Structure):
    _fields_ = [("damping", C.c_double), ("max_iter", C.c_int), ("tol", C.c_double),
                ("precision", C.c_int), ("dangling", C.c_int), ("out_mem", C.c_int),
                ("timing", C.c_int), ("method", C.c_int), ("seg_log2", C.c_int),
                ("seg_chunk", C.c_int), ("seg_bin", C.c_int)]


GRAPH_PR_AUTO, GRAPH_PR_GATHER, GRAPH_PR_SEGMENTED = 0, 1, 2


class pagerank_plan_info(C.Structure):
    _fields_ = [("built", C.c_int), ("usable", C.c_int), ("seg_log2", C.c_int),
                ("seg_chunk", C.c_int), ("seg_bin", C.c_int), ("partials", C.c_uint64),
                ("chunks", C.c_uint32), ("bins", C.c_uint32), ("build_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pagerank_hybrid_info(C.Structure):
    _fields_ = [("cpu_threads", C.c_int), ("cpu_vertices", C.c_uint32),
                ("gpu_vertices", C.c_uint32), ("cpu_edges", C.c_int64),
                ("gpu_edges", C.c_int64), ("ms_cpu_compute", C.c_double),
                ("ms_gpu_compute", C.c_double), ("ms_exchange", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


GRAPH_HYBRID_MAX_THREADS = 1024

# Every symbol include/graph.h declares, with (restype, argtypes).
_vp, _u32, _i64, _int = C.c_void_p, C.c_uint32, C.c_int64, C.c_int
SIGNATURES = {
    "graph_load_csr": (_int, [_u32, _i64, _vp, _vp, _vp, _int, C.POINTER(graph_runtime),
                              C.POINTER(_vp)]),
    "graph_partition": (_int, [_vp, C.POINTER(graph_partition_attr)]),
    "graph_get_partition_info": (_int, [_vp, C.POINTER(graph_partition_info)]),
    "graph_export_partition": (_int, [_vp, _int, _vp, _vp, _vp, _vp, _vp, _vp]),
    "graph_set_edge_memory": (_int, [_vp, _int, _int]),
    "graph_get_edge_memory": (_int, [_vp, C.POINTER(_int)]),
    "bfs": (_int, [_vp, _u32, _vp, _vp, C.POINTER(bfs_attr), C.POINTER(graph_stats)]),
    "bfs_batch": (_int, [_vp, _vp, _u32, _vp, C.POINTER(bfs_attr), C.POINTER(graph_stats)]),
    "sssp": (_int, [_vp, _u32, _vp, C.POINTER(sssp_attr), C.POINTER(graph_stats)]),
    "sssp_batch": (_int, [_vp, _vp, _u32, _vp, C.POINTER(sssp_attr), C.POINTER(graph_stats)]),
    "betweenness": (_int, [_vp, _vp, _u32, _vp, C.POINTER(bc_attr), C.POINTER(graph_stats)]),
    "connected_components": (_int, [_vp, _vp, C.POINTER(cc_attr), C.POINTER(graph_stats)]),
    "pagerank": (_int, [_vp, C.POINTER(pagerank_attr), _vp, C.POINTER(graph_stats)]),
    "pagerank_plan_get": (_int, [_vp, C.POINTER(pagerank_plan_info)]),
    "pagerank_multi": (_int, [_vp, _u32, _vp, C.POINTER(pagerank_attr), _vp, _vp,
                              C.POINTER(graph_stats)]),
    "pagerank_hybrid": (_int, [_vp, C.POINTER(pagerank_attr), _int, _vp, C.POINTER(graph_stats),
                               C.POINTER(pagerank_hybrid_info)]),
    "bfs_hybrid": (_int, [_vp, _u32, _vp, _vp, C.POINTER(bfs_attr), _int, C.POINTER(graph_stats),
                          C.POINTER(pagerank_hybrid_info)]),
    "sssp_hybrid": (_int, [_vp, _u32, _vp, C.POINTER(sssp_attr), _int, C.POINTER(graph_stats),
                           C.POINTER(pagerank_hybrid_info)]),
    "bfs_csr_noalloc": (_int, [_u32, _i64, _vp, _vp, _u32, _vp, _vp, _vp]),
    "graph_server_create": (_int, [_vp, C.POINTER(graph_server_attr), C.POINTER(_vp)]),
    "graph_server_submit": (_int, [_vp, _int, _u32, _vp, C.POINTER(C.c_uint64)]),
    "graph_server_poll": (_int, [_vp, C.POINTER(graph_completion), _u32, C.POINTER(_u32),
                                 _int]),
    "graph_server_info_get": (_int, [_vp, C.POINTER(graph_server_info)]),
    "graph_server_destroy": (_int, [_vp]),
    "graph_free": (None, [_vp]),
    "graph_strerror": (C.c_char_p, [_int]),
    "graph_last_error": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The loaded library. Raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                if build_if_missing:
                    _build.build()
                else:
                    raise RuntimeError(
                        f"CUDA library {path} is not built; run "
                        "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class GraphError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.graph_strerror(status).decode()
        detail = lib.graph_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}): {detail}")
        self.status = status


def check(status: int, where: str):
    if status != GRAPH_OK:
        raise GraphError(status, where)
